"""The allocation-free colouring entry point (amg_colour_noalloc).

Callers that may not allocate at call time (stream capture, real-time paths,
pre-reserved memory) get the finest-level colouring from a fixed device array
inside the library.  This checks, through the C ABI, that it gives exactly the
colouring that amg_setup computes for level 0 (colourings are compared bit for
bit, as everywhere in these tests), on two calls in a row that share the
scratch array.  The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _level0_colours(s):
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    va = torch.from_numpy(np.ascontiguousarray(s.vals.reshape(-1))).cuda()
    g = bamg.Solver(rp, ci, va, s.b, s.field_of_dof, max_levels=2, max_coarse=0)
    L0 = g.level(0)
    return rp, ci, L0["colour"], L0["n_colours"]


@pytest.mark.parametrize("system", ["mhd2d_40", "stokes3d_9"])
def test_noalloc_colouring_equals_setup_colouring_on_two_calls(system):
    assert torch.cuda.is_available()
    s = P.mhd2d(40, 2) if system == "mhd2d_40" else P.stokes3d(9, 1)
    rp, ci, ref_colour, ref_nc = _level0_colours(s)
    lib = bamg.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        colour = torch.full((s.n_nodes,), -7, dtype=torch.int32, device="cuda")
        nc = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        st = lib.amg_colour_noalloc(rp.data_ptr(), ci.data_ptr(), s.n_nodes, colour.data_ptr(), nc.data_ptr(),
                                    ctypes.c_void_p(stream))
        assert st == bamg.BAMG_OK, (call, bamg.amg_strerror(st))
        torch.cuda.synchronize()
        assert int(nc.item()) == ref_nc, call
        assert np.array_equal(colour.cpu().numpy(), ref_colour), call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = bamg.load()
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = lib.amg_colour_noalloc(d.data_ptr(), d.data_ptr(), 40001, d.data_ptr(), d.data_ptr(), None)
    assert st == bamg.BAMG_EUNSUPPORTED
