"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares.  CPU only: no compute call is made."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2103_07537_gb300 import bamg, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:long\s+|unsigned\s+)*\w+[\s\*]+(\w+)\s*\(", text,
                                 flags=re.M)))


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ["amg_setup", "amg_apply", "fgmres_solve", "amg_destroy", "amg_stats", "amg_strerror",
                 "bsr_spmv", "amg_solve_host", "amg_setup_fields", "amg_level_fields"]:
        assert name in fns


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    assert sorted(bamg.EXPORTS) == sorted(declared_functions())
    lib = bamg.load()
    for f in declared_functions():
        assert hasattr(lib, f)


def test_host_side_validation_without_gpu():
    # argument checks that return before any CUDA call
    lib = bamg.load()
    h = ctypes.c_void_p()
    fm = np.zeros(3, np.int32)
    assert lib.amg_setup(None, None, None, 1, 1, 3, fm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), None, None,
                         ctypes.byref(h)) == bamg.BAMG_EINVAL
    assert lib.amg_apply(None, None, None, None) == bamg.BAMG_EINVAL
    assert lib.amg_destroy(None) == bamg.BAMG_OK
    assert bamg.amg_strerror(bamg.BAMG_ESINGULAR_COARSE) == "singular coarsest operator"
    # fields on node sets: bad ranges, parameters the mode excludes, a null handle
    ip = ctypes.POINTER(ctypes.c_int)
    dummy = ctypes.c_void_p(16)
    for off, kw in (([0, 0, 10], {}), ([0, 4, 9], {}), ([1, 4, 10], {}), ([0, 6, 4, 10], {}),
                    ([0, 4, 10], dict(smooth_p=1)), ([0] + list(range(1, 10)) + [10], {})):
        o = np.array(off, np.int32)
        prm = bamg.amg_default_params(**kw)
        assert lib.amg_setup_fields(dummy, dummy, dummy, 10, 10, 3, len(off) - 1, o.ctypes.data_as(ip),
                                    ctypes.byref(prm), None, ctypes.byref(h)) == bamg.BAMG_EINVAL
        assert not h.value
    assert lib.amg_level_fields(None, 0, None, None) == bamg.BAMG_EINVAL
    p = bamg.amg_default_params()
    assert (p.max_levels, p.max_coarse, p.n_pre, p.n_post, p.omega, p.cycle_prec) == (10, 2500, 1, 1, 0.5, 64)


def test_oracle_is_not_linked_into_the_library():
    out = subprocess.run(["nm", "-D", build.LIB_PATH], capture_output=True, text=True, check=True).stdout
    assert "oracle_" not in out


def test_no_cpu_fallback():
    # the binding computes nothing on the host: CPU tensors are refused before
    # any call into the library, for every solver class
    torch = pytest.importorskip("torch")
    from paper_2103_07537_gb300 import problems as P

    s = P.mhd2d_q2q1(2, 1)
    rp, ci = torch.from_numpy(s.row_ptr), torch.from_numpy(s.col_idx)
    va = torch.from_numpy(s.vals.reshape(-1))
    with pytest.raises(ValueError, match="CUDA"):
        bamg.Solver(rp, ci, va, 3, [0, 0, 0])
    with pytest.raises(ValueError, match="CUDA"):
        bamg.FieldSolver(s.node_field_off, rp, ci, va, 3)
    with pytest.raises(ValueError, match="CUDA"):
        bamg.BatchSolver([0, s.n_nodes], rp, ci, va, 3, [0, 0, 0])


def test_params_struct_layout_matches_the_header(tmp_path):
    # the binding's ctypes amg_params against the C compiler's layout of the
    # header's struct: every field at the same offset, the same total size
    fields = [name for name, _ in bamg.AmgParams._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "bamg.h"', 'int main(void) {',
             '    printf("size %zu\\n", sizeof(amg_params));']
    lines += ['    printf("%s %%zu\\n", offsetof(amg_params, %s));' % (f, f) for f in fields]
    lines += ['    return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    assert int(got["size"]) == ctypes.sizeof(bamg.AmgParams)
    for f in fields:
        assert int(got[f]) == getattr(bamg.AmgParams, f).offset, f


def test_parameter_and_field_map_refusals_without_gpu():
    # refusals of amg_setup that return before any CUDA call: inner sweeps out
    # of range or with another sub-solver, autotune out of range, field maps
    # that skip a field or start above 0, fields of unequal size with the
    # options built on one field width, and a padded block wider than 8
    lib = bamg.load()
    ip = ctypes.POINTER(ctypes.c_int)
    dummy = ctypes.c_void_p(16)
    h = ctypes.c_void_p()

    def setup(fmap, **kw):
        fm = np.array(fmap, np.int32)
        prm = bamg.amg_default_params(**kw)
        st = lib.amg_setup(dummy, dummy, dummy, 10, 10, len(fmap), fm.ctypes.data_as(ip), ctypes.byref(prm), None,
                           ctypes.byref(h))
        assert not h.value
        return st

    for kw in (dict(inner_sweeps=65), dict(inner_sweeps=-1), dict(inner_sweeps=2, sub_solver=1),
               dict(inner_sweeps=2, sub_solver=2), dict(autotune=9), dict(coarse_tc=2)):
        assert setup([0, 0, 0, 0], **kw) == bamg.BAMG_EINVAL, kw
    for fmap in ([0, 0, 2, 2], [1, 1, 0, 0], [0, 1, 0, 1]):
        assert setup(fmap) == bamg.BAMG_EINVAL, fmap
    for fmap, kw in (([0, 0, 1], dict(smooth_p=1)), ([0, 0, 1], dict(sub_solver=1)),
                     ([0, 0, 1], dict(sub_solver=2)), ([0, 0, 0, 1, 1, 1, 2], {})):
        assert setup(fmap, **kw) == bamg.BAMG_EUNSUPPORTED, (fmap, kw)
    assert lib.amg_block_size(None) == bamg.BAMG_EINVAL
