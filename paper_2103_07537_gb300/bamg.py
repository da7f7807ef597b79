"""Python binding of the bamg C ABI (include/bamg.h, include/bamg_fields.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
arguments are torch CUDA tensors (their storage is passed as a raw pointer),
host arguments numpy arrays.  Every step of the solve runs in the CUDA
library; if that library cannot be loaded these functions raise, there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import threading

import numpy as np

from . import build as _build

BAMG_OK, BAMG_NOT_CONVERGED = 0, 1
BAMG_EINVAL, BAMG_ECUDA, BAMG_ESINGULAR_BLOCK, BAMG_ESINGULAR_COARSE = -1, -2, -3, -4
BAMG_ENAN, BAMG_ETIMEOUT, BAMG_EUNSUPPORTED = -5, -6, -7

#: every symbol the C header declares
EXPORTS = ["amg_default_params", "amg_setup", "amg_apply", "fgmres_solve", "amg_solve_host", "amg_solve_batched_host",
           "amg_solve_fields_host", "bsr_spmv",
           "amg_num_levels", "amg_level_info", "amg_level_copy", "amg_level_ilu", "amg_stats", "amg_destroy", "amg_strerror",
           "amg_profile", "amg_profile_read", "amg_profile_read_level", "amg_launch_count", "amg_colour_noalloc", "amg_setup_batched",
           "fgmres_solve_batched", "amg_num_systems", "amg_level_systems", "amg_features", "mlp_pack",
           "mlp_forward", "mlp_grad", "mlp_adam", "mlp_clip", "amg_set_omega", "amg_select", "amg_level_omega",
           "amg_level_p", "amg_setup_fields", "amg_level_fields", "amg_dense_inverse_f32", "amg_gemm_tc_f32",
           "amg_block_size"]

#: network sizes (include/bamg.h)
NFEAT, MLP_H, MLP_OUT = 8, 64, 2
MLP_NTRAIN = MLP_H * NFEAT + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT
MLP_NPARAMS = MLP_NTRAIN + 2 * NFEAT

#: kernel kinds of amg_profile_read
KERNEL_KINDS = ["smooth", "residual", "restrict", "prolong", "coarse", "spmv", "krylov", "cast", "tail"]

_lock = threading.Lock()
_lib = None


class AmgParams(C.Structure):
    _fields_ = [("max_levels", C.c_int), ("max_coarse", C.c_int), ("n_pre", C.c_int), ("n_post", C.c_int),
                ("omega", C.c_double), ("cycle_prec", C.c_int), ("use_graph", C.c_int), ("tail_dofs", C.c_int),
                ("autotune", C.c_int), ("smooth_p", C.c_int), ("omega_p", C.c_double),
                ("omega_s_arr", C.POINTER(C.c_double)), ("omega_s_len", C.c_longlong),
                ("omega_p_arr", C.POINTER(C.c_double)), ("omega_p_len", C.c_longlong),
                ("mlp", C.POINTER(C.c_float)), ("pr_storage", C.c_int), ("mlp_levels", C.c_int),
                ("use_pdl", C.c_int), ("coarse_prec", C.c_int), ("tail_grid", C.c_int),
                ("value_layout", C.c_int), ("sweep", C.c_int), ("sub_solver", C.c_int),
                ("schwarz_overlap", C.c_int), ("ortho", C.c_int), ("coarse_tc", C.c_int),
                ("inner_sweeps", C.c_int)]


class BamgError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {amg_strerror(status)} (status {status})")
        self.status = status


_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)
_vp = C.c_void_p


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libbamg.so (building it in-tree if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"bamg CUDA library not built: {path}")
            _build.build()
        lib = C.CDLL(path)
        lib.amg_default_params.argtypes = [C.POINTER(AmgParams)]
        lib.amg_default_params.restype = None
        lib.amg_setup.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _ip, C.POINTER(AmgParams), _vp,
                                  C.POINTER(_vp)]
        lib.amg_apply.argtypes = [_vp, _vp, _vp, _vp]
        lib.fgmres_solve.argtypes = [_vp, _vp, _vp, C.c_double, C.c_int, C.c_int, _ip, _dp, _vp]
        lib.amg_solve_host.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _ip, C.POINTER(AmgParams), _vp,
                                       _vp, C.c_double, C.c_int, C.c_int, _ip, _dp, _vp]
        lib.amg_solve_batched_host.argtypes = [C.c_int, _ip, _vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _ip,
                                               C.POINTER(AmgParams), _vp, _vp, C.c_double, C.c_int, C.c_int, _ip,
                                               _dp, _vp]
        lib.amg_solve_fields_host.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _ip,
                                              C.POINTER(AmgParams), _vp, _vp, C.c_double, C.c_int, C.c_int, _ip, _dp,
                                              _vp]
        lib.bsr_spmv.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp]
        lib.amg_num_levels.argtypes = [_vp]
        lib.amg_block_size.argtypes = [_vp]
        lib.amg_level_info.argtypes = [_vp, C.c_int, _ip, _ip, _ip, _ip]
        lib.amg_level_copy.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp]
        lib.amg_level_ilu.argtypes = [_vp, C.c_int, _vp]
        lib.amg_stats.argtypes = [_vp, C.c_char_p, C.c_int]
        lib.amg_destroy.argtypes = [_vp]
        lib.amg_strerror.argtypes = [C.c_int]
        lib.amg_strerror.restype = C.c_char_p
        lib.amg_profile.argtypes = [_vp, C.c_int]
        lib.amg_profile_read.argtypes = [_vp, C.c_int, _dp, C.POINTER(C.c_longlong), _dp, _dp]
        lib.amg_profile_read_level.argtypes = [_vp, C.c_int, C.c_int, _dp, C.POINTER(C.c_longlong), _dp, _dp]
        lib.amg_launch_count.argtypes = []
        lib.amg_launch_count.restype = C.c_longlong
        lib.amg_colour_noalloc.argtypes = [_vp, _vp, C.c_int, _vp, _vp, _vp]
        lib.amg_dense_inverse_f32.argtypes = [C.c_int, _vp, _vp, C.c_int, _vp]
        lib.amg_gemm_tc_f32.argtypes = [C.c_int, C.c_int, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp]
        lib.amg_setup_batched.argtypes = [C.c_int, _ip, _vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _ip,
                                          C.POINTER(AmgParams), _vp, C.POINTER(_vp)]
        lib.fgmres_solve_batched.argtypes = [_vp, _vp, _vp, C.c_double, C.c_int, C.c_int, _ip, _dp, _vp]
        lib.amg_num_systems.argtypes = [_vp]
        lib.amg_level_systems.argtypes = [_vp, C.c_int, _ip]
        lib.amg_features.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, _ip, _vp, C.c_int, C.c_int, _vp, _vp, _vp]
        lib.mlp_pack.argtypes = [_vp, _vp, _vp]
        lib.mlp_forward.argtypes = [_vp, _vp, C.c_int, _vp, _vp]
        lib.mlp_grad.argtypes = [_vp, _vp, _vp, _vp, C.c_int, _vp, _vp, _vp]
        lib.mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, _vp]
        lib.mlp_clip.argtypes = [C.c_int, C.c_double]
        lib.mlp_clip.restype = C.c_double
        lib.amg_set_omega.argtypes = [_vp, C.c_int, _vp, _vp]
        lib.amg_select.argtypes = [_vp, _vp, _vp, C.c_double, C.c_int, C.c_int, _ip, _ip, _ip, _vp]
        lib.amg_level_omega.argtypes = [_vp, C.c_int, _vp, _vp]
        lib.amg_level_p.argtypes = [_vp, C.c_int, _ip, _vp, _vp, _vp]
        lib.amg_setup_fields.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _ip,
                                         C.POINTER(AmgParams), _vp, C.POINTER(_vp)]
        lib.amg_level_fields.argtypes = [_vp, C.c_int, _ip, _ip]
        _lib = lib
        return lib


def _ptr(t) -> int:
    """Raw device pointer of a contiguous torch CUDA tensor."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _hp(a: np.ndarray) -> int:
    return a.ctypes.data


def amg_strerror(status: int) -> str:
    return load().amg_strerror(int(status)).decode()


def amg_default_params(**overrides) -> AmgParams:
    """Defaults with overrides; the host arrays omega_s_arr, omega_p_arr
    (float64) and mlp (float32, MLP_NPARAMS) are given as numpy arrays and
    kept alive by the returned structure."""
    p = AmgParams()
    load().amg_default_params(C.byref(p))
    keep = []
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        if k in ("omega_s_arr", "omega_p_arr") and v is not None:
            a = np.ascontiguousarray(v, dtype=np.float64).ravel()
            keep.append(a)
            setattr(p, k, a.ctypes.data_as(C.POINTER(C.c_double)))
            setattr(p, k.replace("_arr", "_len"), a.size)
        elif k == "mlp" and v is not None:
            a = np.ascontiguousarray(v, dtype=np.float32).ravel()
            if a.size != MLP_NPARAMS:
                raise ValueError(f"mlp needs {MLP_NPARAMS} parameters")
            keep.append(a)
            p.mlp = a.ctypes.data_as(C.POINTER(C.c_float))
        elif v is not None:
            setattr(p, k, v)
    p._keep = keep
    return p


def amg_setup(row_ptr, col_idx, vals, n_nodes: int, nnzb: int, b: int, field_of_dof, params=None,
              stream=None) -> int:
    """Returns the handle (an int); device tensors row_ptr/col_idx (int32), vals (float64)."""
    fm = np.ascontiguousarray(field_of_dof, dtype=np.int32)
    h = _vp()
    st = load().amg_setup(_ptr(row_ptr), _ptr(col_idx), _ptr(vals), int(n_nodes), int(nnzb), int(b),
                          fm.ctypes.data_as(_ip), C.byref(params) if params is not None else None,
                          _stream(stream), C.byref(h))
    if st != BAMG_OK:
        raise BamgError(st, "amg_setup")
    return h.value


def amg_apply(handle: int, r, z, stream=None) -> None:
    st = load().amg_apply(handle, _ptr(r), _ptr(z), _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "amg_apply")


def fgmres_solve(handle: int, b, x, tol=1e-8, restart=30, max_iter=10000, stream=None):
    """Returns (status, iterations, true relative residual); x updated in place."""
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = load().fgmres_solve(handle, _ptr(b), _ptr(x), float(tol), int(restart), int(max_iter), C.byref(it),
                             C.byref(rr), _stream(stream))
    if st < 0:
        raise BamgError(st, "fgmres_solve")
    return st, it.value, rr.value


def amg_solve_host(row_ptr: np.ndarray, col_idx: np.ndarray, vals: np.ndarray, n_nodes: int, nnzb: int, b: int,
                   field_of_dof, rhs: np.ndarray, x: np.ndarray, tol=1e-8, restart=30, max_iter=10000,
                   params=None, stream=None):
    """Host arrays in, solution written to x (float64, in place)."""
    fm = np.ascontiguousarray(field_of_dof, dtype=np.int32)
    for a, dt in ((row_ptr, np.int32), (col_idx, np.int32), (vals, np.float64), (rhs, np.float64),
                  (x, np.float64)):
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous int32 / float64")
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = load().amg_solve_host(_hp(row_ptr), _hp(col_idx), _hp(vals), int(n_nodes), int(nnzb), int(b),
                               fm.ctypes.data_as(_ip), C.byref(params) if params is not None else None,
                               _hp(rhs), _hp(x), float(tol), int(restart), int(max_iter), C.byref(it),
                               C.byref(rr), _stream(stream))
    if st < 0:
        raise BamgError(st, "amg_solve_host")
    return st, it.value, rr.value


def _host_arrays(*arrs):
    for a, dt in arrs:
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous int32 / float64")


def amg_solve_batched_host(sys_node_off, row_ptr: np.ndarray, col_idx: np.ndarray, vals: np.ndarray, n_nodes: int,
                           nnzb: int, b: int, field_of_dof, rhs: np.ndarray, x: np.ndarray, tol=1e-8, restart=30,
                           max_iter=10000, params=None, stream=None):
    """A batch end to end from host arrays; x (float64) updated in place.
    Returns (status, iterations[nsys], true relative residuals[nsys])."""
    off = np.ascontiguousarray(sys_node_off, dtype=np.int32)
    fm = np.ascontiguousarray(field_of_dof, dtype=np.int32)
    _host_arrays((row_ptr, np.int32), (col_idx, np.int32), (vals, np.float64), (rhs, np.float64), (x, np.float64))
    ns = off.size - 1
    it = np.zeros(ns, np.int32)
    rr = np.zeros(ns)
    st = load().amg_solve_batched_host(ns, off.ctypes.data_as(_ip), _hp(row_ptr), _hp(col_idx), _hp(vals),
                                       int(n_nodes), int(nnzb), int(b), fm.ctypes.data_as(_ip),
                                       C.byref(params) if params is not None else None, _hp(rhs), _hp(x), float(tol),
                                       int(restart), int(max_iter), it.ctypes.data_as(_ip),
                                       rr.ctypes.data_as(_dp), _stream(stream))
    if st < 0:
        raise BamgError(st, "amg_solve_batched_host")
    return st, it, rr


def amg_solve_fields_host(field_node_off, row_ptr: np.ndarray, col_idx: np.ndarray, vals: np.ndarray,
                          n_nodes: int, nnzb: int, b: int, rhs: np.ndarray, x: np.ndarray, tol=1e-8, restart=30,
                          max_iter=10000, params=None, stream=None):
    """A system with fields on node sets end to end from host arrays; x
    updated in place.  Returns (status, iterations, true relative residual)."""
    off = np.ascontiguousarray(field_node_off, dtype=np.int32)
    _host_arrays((row_ptr, np.int32), (col_idx, np.int32), (vals, np.float64), (rhs, np.float64), (x, np.float64))
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = load().amg_solve_fields_host(_hp(row_ptr), _hp(col_idx), _hp(vals), int(n_nodes), int(nnzb), int(b),
                                      off.size - 1, off.ctypes.data_as(_ip),
                                      C.byref(params) if params is not None else None, _hp(rhs), _hp(x), float(tol),
                                      int(restart), int(max_iter), C.byref(it), C.byref(rr), _stream(stream))
    if st < 0:
        raise BamgError(st, "amg_solve_fields_host")
    return st, it.value, rr.value


def bsr_spmv(row_ptr, col_idx, vals, n_nodes: int, b: int, x, y, stream=None) -> None:
    st = load().bsr_spmv(_ptr(row_ptr), _ptr(col_idx), _ptr(vals), int(n_nodes), int(b), _ptr(x), _ptr(y),
                         _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "bsr_spmv")


def amg_num_levels(handle: int) -> int:
    n = load().amg_num_levels(handle)
    if n < 0:
        raise BamgError(n, "amg_num_levels")
    return n


def amg_block_size(handle: int) -> int:
    """Dofs per node of the hierarchy's levels (the padded size for fields of unequal size)."""
    b = load().amg_block_size(handle)
    if b < 0:
        raise BamgError(b, "amg_block_size")
    return b


def amg_level_info(handle: int, level: int):
    n, nnz, nc, na = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    st = load().amg_level_info(handle, level, C.byref(n), C.byref(nnz), C.byref(nc), C.byref(na))
    if st != BAMG_OK:
        raise BamgError(st, "amg_level_info")
    return n.value, nnz.value, nc.value, na.value


def amg_level_copy(handle: int, level: int, b: int, F: int):
    """dict of host copies of one level (see include/bamg.h)."""
    n, nnz, ncol, nagg = amg_level_info(handle, level)
    coarsest = level == amg_num_levels(handle) - 1
    fb = b // F
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(nnz, np.int32)
    v = np.zeros((nnz, b, b))
    agg = None if coarsest else np.zeros(n, np.int32)
    col = None if coarsest else np.zeros(n, np.int32)
    dinv = None if coarsest else np.zeros((n, F, fb, fb))
    st = load().amg_level_copy(handle, level, _hp(rp), _hp(ci), _hp(v), _hp(agg) if agg is not None else None,
                               _hp(col) if col is not None else None, _hp(dinv) if dinv is not None else None)
    if st != BAMG_OK:
        raise BamgError(st, "amg_level_copy")
    return dict(n=n, nnzb=nnz, n_colours=ncol, n_agg=nagg, row_ptr=rp, col_idx=ci, vals=v, agg=agg,
                colour=col, dinv=dinv)


def amg_level_ilu(handle: int, level: int, b: int, F: int):
    """Host copy of one level's ILU(0) factors, shape (F, nnzb, fb, fb)."""
    _, nnz, _, _ = amg_level_info(handle, level)
    fb = b // F
    lu = np.zeros((F, nnz, fb, fb))
    st = load().amg_level_ilu(handle, level, _hp(lu))
    if st != BAMG_OK:
        raise BamgError(st, "amg_level_ilu")
    return lu


def amg_stats(handle: int) -> dict:
    buf = C.create_string_buffer(1 << 16)
    n = load().amg_stats(handle, buf, len(buf))
    if n < 0:
        raise BamgError(n, "amg_stats")
    return json.loads(buf.value.decode())


def amg_destroy(handle: int) -> None:
    load().amg_destroy(handle)


def amg_profile(handle: int, enable: bool) -> None:
    st = load().amg_profile(handle, 1 if enable else 0)
    if st != BAMG_OK:
        raise BamgError(st, "amg_profile")


def amg_profile_read(handle: int, kind) -> dict:
    """{'ms', 'launches', 'bytes', 'flops'} for one kernel kind since the last read."""
    k = KERNEL_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    ms, n, by, fl = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
    st = load().amg_profile_read(handle, k, C.byref(ms), C.byref(n), C.byref(by), C.byref(fl))
    if st != BAMG_OK:
        raise BamgError(st, "amg_profile_read")
    return dict(ms=ms.value, launches=n.value, bytes=by.value, flops=fl.value)


def amg_profile_read_level(handle: int, kind, level: int) -> dict:
    """As amg_profile_read for the launches of one level (-1: the outer FGMRES kernels)."""
    k = KERNEL_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    ms, n, by, fl = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
    st = load().amg_profile_read_level(handle, k, int(level), C.byref(ms), C.byref(n), C.byref(by), C.byref(fl))
    if st != BAMG_OK:
        raise BamgError(st, "amg_profile_read_level")
    return dict(ms=ms.value, launches=n.value, bytes=by.value, flops=fl.value)


def amg_launch_count() -> int:
    return int(load().amg_launch_count())


def amg_dense_inverse_f32(a, inv, method: int = 1, stream=None) -> None:
    """inv = a^-1 for a square contiguous FP32 device tensor a (row-major) by LU
    with partial pivoting; method 1 = tensor cores, 0 = CUDA cores."""
    nd = int(a.shape[0])
    st = load().amg_dense_inverse_f32(nd, _ptr(a), _ptr(inv), int(method), _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "amg_dense_inverse_f32")


def amg_gemm_tc_f32(A, B, C_, stream=None) -> None:
    """C_ += A @ B on the tensor cores (contiguous row-major FP32 device tensors)."""
    m, k = int(A.shape[0]), int(A.shape[1])
    n = int(B.shape[1])
    st = load().amg_gemm_tc_f32(m, n, k, _ptr(A), k, _ptr(B), n, _ptr(C_), n, _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "amg_gemm_tc_f32")


def amg_colour_noalloc(row_ptr, col_idx, n_nodes: int, colour, n_colours, stream=None) -> None:
    """Colours of the pattern into device int32 tensors colour[n_nodes] and
    n_colours[1] (-1 on failure), without any allocation in the library."""
    st = load().amg_colour_noalloc(_ptr(row_ptr), _ptr(col_idx), int(n_nodes), _ptr(colour), _ptr(n_colours),
                                   _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "amg_colour_noalloc")


def amg_setup_batched(sys_node_off, row_ptr, col_idx, vals, n_nodes: int, nnzb: int, b: int, field_of_dof,
                      params=None, stream=None) -> int:
    off = np.ascontiguousarray(sys_node_off, dtype=np.int32)
    fm = np.ascontiguousarray(field_of_dof, dtype=np.int32)
    h = _vp()
    st = load().amg_setup_batched(int(off.shape[0] - 1), off.ctypes.data_as(_ip), _ptr(row_ptr), _ptr(col_idx),
                                  _ptr(vals), int(n_nodes), int(nnzb), int(b), fm.ctypes.data_as(_ip),
                                  C.byref(params) if params is not None else None, _stream(stream), C.byref(h))
    if st != BAMG_OK:
        raise BamgError(st, "amg_setup_batched")
    return h.value


def amg_setup_fields(field_node_off, row_ptr, col_idx, vals, n_nodes: int, nnzb: int, b: int, params=None,
                     stream=None) -> int:
    """Hierarchy of a system whose fields live on disjoint node sets
    (include/bamg_fields.h); field g owns nodes field_node_off[g]..[g+1]-1."""
    off = np.ascontiguousarray(field_node_off, dtype=np.int32)
    h = _vp()
    st = load().amg_setup_fields(_ptr(row_ptr), _ptr(col_idx), _ptr(vals), int(n_nodes), int(nnzb), int(b),
                                 int(off.shape[0] - 1), off.ctypes.data_as(_ip),
                                 C.byref(params) if params is not None else None, _stream(stream), C.byref(h))
    if st != BAMG_OK:
        raise BamgError(st, "amg_setup_fields")
    return h.value


def amg_level_fields(handle: int, level: int, n_fields: int):
    """(node_off[n_fields+1], colour_off[n_fields+1]) of one level."""
    no = np.zeros(n_fields + 1, np.int32)
    co = np.zeros(n_fields + 1, np.int32)
    st = load().amg_level_fields(handle, level, no.ctypes.data_as(_ip), co.ctypes.data_as(_ip))
    if st < 0:
        raise BamgError(st, "amg_level_fields")
    return no, co


def fgmres_solve_batched(handle: int, b, x, tol=1e-8, restart=30, max_iter=10000, stream=None):
    """Returns (status, iterations[nsys], true relative residuals[nsys])."""
    ns = amg_num_systems(handle)
    it = np.zeros(ns, np.int32)
    rr = np.zeros(ns)
    st = load().fgmres_solve_batched(handle, _ptr(b), _ptr(x), float(tol), int(restart), int(max_iter),
                                     it.ctypes.data_as(_ip), rr.ctypes.data_as(_dp), _stream(stream))
    if st < 0:
        raise BamgError(st, "fgmres_solve_batched")
    return st, it, rr


def amg_num_systems(handle: int) -> int:
    n = load().amg_num_systems(handle)
    if n < 0:
        raise BamgError(n, "amg_num_systems")
    return n


def amg_level_systems(handle: int, level: int) -> np.ndarray:
    off = np.zeros(amg_num_systems(handle) + 1, np.int32)
    st = load().amg_level_systems(handle, level, off.ctypes.data_as(_ip))
    if st != BAMG_OK:
        raise BamgError(st, "amg_level_systems")
    return off


def amg_features(row_ptr, col_idx, vals, n_nodes: int, b: int, field_of_dof, agg, n_agg: int, level: int,
                 node_feat, agg_feat=None, stream=None) -> None:
    fm = np.ascontiguousarray(field_of_dof, dtype=np.int32)
    st = load().amg_features(_ptr(row_ptr), _ptr(col_idx), _ptr(vals), int(n_nodes), int(b), fm.ctypes.data_as(_ip),
                             _ptr(agg), int(n_agg), int(level), _ptr(node_feat),
                             _ptr(agg_feat) if agg_feat is not None else None, _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "amg_features")


def mlp_pack(params, params16, stream=None) -> None:
    st = load().mlp_pack(_ptr(params), _ptr(params16), _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "mlp_pack")


def mlp_forward(params16, x, n: int, y, stream=None) -> None:
    st = load().mlp_forward(_ptr(params16), _ptr(x), int(n), _ptr(y), _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "mlp_forward")


def mlp_grad(params16, x, t, head, n: int, grad, loss, stream=None) -> None:
    st = load().mlp_grad(_ptr(params16), _ptr(x), _ptr(t), _ptr(head), int(n), _ptr(grad), _ptr(loss),
                         _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "mlp_grad")


def mlp_adam(params, params16, grad, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    st = load().mlp_adam(_ptr(params), _ptr(params16), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr), float(beta1),
                         float(beta2), float(eps), _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "mlp_adam")


def mlp_clip(head: int, w: float) -> float:
    return float(load().mlp_clip(int(head), float(w)))


def amg_set_omega(handle: int, level: int, omega_s, stream=None) -> None:
    st = load().amg_set_omega(handle, int(level), _ptr(omega_s), _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "amg_set_omega")


def amg_select(learned: int, plain: int, b, tol=1e-8, restart=30, max_iter=10000, stream=None):
    """Returns (choice, iterations learned, iterations plain); choice 0 keeps the learned hierarchy."""
    ch, il, ip = C.c_int(), C.c_int(), C.c_int()
    st = load().amg_select(learned, plain, _ptr(b), float(tol), int(restart), int(max_iter), C.byref(ch),
                           C.byref(il), C.byref(ip), _stream(stream))
    if st != BAMG_OK:
        raise BamgError(st, "amg_select")
    return ch.value, il.value, ip.value


def amg_level_omega(handle: int, level: int, F: int):
    """(omega_s[n, F], omega_p[n_agg, F]) host copies of one level."""
    n, _, _, nagg = amg_level_info(handle, level)
    ws = np.zeros((n, F))
    wp = np.zeros((max(nagg, 0), F))
    st = load().amg_level_omega(handle, level, _hp(ws), _hp(wp) if wp.size else None)
    if st != BAMG_OK:
        raise BamgError(st, "amg_level_omega")
    return ws, wp


def amg_level_p(handle: int, level: int, F: int, fb: int):
    """(p_rp, p_ci, p_v[nnz, F, fb, fb]) of a level with a smoothed P, else None."""
    nnz = C.c_int()
    st = load().amg_level_p(handle, level, C.byref(nnz), None, None, None)
    if st != BAMG_OK:
        raise BamgError(st, "amg_level_p")
    if nnz.value == 0:
        return None
    n = amg_level_info(handle, level)[0]
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(nnz.value, np.int32)
    v = np.zeros((nnz.value, F, fb, fb))
    st = load().amg_level_p(handle, level, C.byref(nnz), _hp(rp), _hp(ci), _hp(v))
    if st != BAMG_OK:
        raise BamgError(st, "amg_level_p")
    return rp, ci, v


class Solver:
    """Owns one hierarchy built from a block system held in device tensors."""

    def __init__(self, row_ptr, col_idx, vals, b: int, field_of_dof, stream=None, **params):
        self.b = int(b)
        self.F = int(max(field_of_dof)) + 1
        self.n = int(row_ptr.shape[0]) - 1
        self.row_ptr, self.col_idx, self.vals = row_ptr, col_idx, vals
        self.params = amg_default_params(**params)
        self.handle = amg_setup(row_ptr, col_idx, vals, self.n, int(col_idx.shape[0]), self.b, field_of_dof,
                                self.params, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                amg_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def num_levels(self) -> int:
        return amg_num_levels(self.handle)

    def level(self, l: int) -> dict:
        # the levels of a system with fields of unequal size are the padded system's
        return amg_level_copy(self.handle, l, amg_block_size(self.handle), self.F)

    def ilu(self, l: int):
        return amg_level_ilu(self.handle, l, self.b, self.F)

    def apply(self, r, z, stream=None):
        amg_apply(self.handle, r, z, stream)
        return z

    def solve(self, b, x, tol=1e-8, restart=30, max_iter=10000, stream=None):
        return fgmres_solve(self.handle, b, x, tol, restart, max_iter, stream)

    def stats(self) -> dict:
        return amg_stats(self.handle)

    def omega(self, l: int):
        return amg_level_omega(self.handle, l, self.F)

    def prolongator(self, l: int):
        return amg_level_p(self.handle, l, self.F, self.b // self.F)

    def set_omega(self, l: int, omega_s, stream=None):
        amg_set_omega(self.handle, l, omega_s, stream)


class FieldSolver(Solver):
    """Owns one hierarchy of a system whose fields live on disjoint node sets
    (field g owns nodes field_node_off[g]..[g+1]-1, every dof of a node in its
    node's field): separate aggregation per field block."""

    def __init__(self, field_node_off, row_ptr, col_idx, vals, b: int, stream=None, **params):
        self.b = int(b)
        self.F = 1
        self.n = int(row_ptr.shape[0]) - 1
        self.n_fields = len(field_node_off) - 1
        self.row_ptr, self.col_idx, self.vals = row_ptr, col_idx, vals
        self.params = amg_default_params(**params)
        self.handle = amg_setup_fields(field_node_off, row_ptr, col_idx, vals, self.n, int(col_idx.shape[0]),
                                       self.b, self.params, stream)

    def fields(self, l: int):
        return amg_level_fields(self.handle, l, self.n_fields)


class BatchSolver(Solver):
    """Owns one hierarchy for a batch of independent systems (block-diagonal
    device BSR with the node range of every system in sys_node_off)."""

    def __init__(self, sys_node_off, row_ptr, col_idx, vals, b: int, field_of_dof, stream=None, **params):
        self.b = int(b)
        self.F = int(max(field_of_dof)) + 1
        self.n = int(row_ptr.shape[0]) - 1
        self.row_ptr, self.col_idx, self.vals = row_ptr, col_idx, vals
        self.params = amg_default_params(**params)
        self.handle = amg_setup_batched(sys_node_off, row_ptr, col_idx, vals, self.n, int(col_idx.shape[0]),
                                        self.b, field_of_dof, self.params, stream)

    @property
    def num_systems(self) -> int:
        return amg_num_systems(self.handle)

    def level_systems(self, l: int) -> np.ndarray:
        return amg_level_systems(self.handle, l)

    def solve(self, b, x, tol=1e-8, restart=30, max_iter=10000, stream=None):
        return fgmres_solve_batched(self.handle, b, x, tol, restart, max_iter, stream)
