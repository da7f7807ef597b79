"""ctypes view of the FP64 C oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
import this package.  The CUDA library neither links nor calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bamg_oracle.c")
_HDR = os.path.join(_HERE, "bamg_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbamg_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ESINGULAR_BLOCK, ESINGULAR_COARSE, NOT_CONVERGED = 0, -1, -2, -3, -4, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fused multiply-add)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest_src = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest_src:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)


class Params(C.Structure):
    _fields_ = [("max_levels", C.c_int), ("max_coarse", C.c_int), ("n_pre", C.c_int),
                ("n_post", C.c_int), ("omega", C.c_double)]


def _declare(L):
    L.oracle_spmv.argtypes = [C.c_int, C.c_int, _ip, _ip, _dp, _dp, _dp]
    L.oracle_aggregate.argtypes = [C.c_int, _ip, _ip, _ip, _ip]
    L.oracle_colour.argtypes = [C.c_int, _ip, _ip, _ip]
    L.oracle_rap_tentative.argtypes = [C.c_int, C.c_int, _ip, _ip, _dp, _ip, C.c_int, _ip, _ip, _dp]
    L.oracle_block_inverse.argtypes = [C.c_int, _dp, _dp]
    L.oracle_lu_factor.argtypes = [C.c_int, _dp, _ip]
    L.oracle_lu_solve.argtypes = [C.c_int, _dp, _ip, _dp, _dp]
    L.oracle_setup.argtypes = [C.c_int, C.c_int, C.c_int, _ip, _ip, _dp, _ip, C.POINTER(Params),
                               C.POINTER(C.c_void_p)]
    L.oracle_free.argtypes = [C.c_void_p]
    L.oracle_free.restype = None
    L.oracle_num_levels.argtypes = [C.c_void_p]
    L.oracle_level_sizes.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _ip, _ip]
    L.oracle_level_get.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _dp, _ip, _ip, _dp]
    L.oracle_bgs.argtypes = [C.c_void_p, C.c_int, _dp, _dp, C.c_int]
    L.oracle_vcycle.argtypes = [C.c_void_p, _dp, _dp]
    L.oracle_fgmres.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, C.c_int, C.c_int, _ip, _dp]


def _i(a):
    return a.ctypes.data_as(_ip)


def _d(a):
    return a.ctypes.data_as(_dp)


def _int32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def spmv(row_ptr, col_idx, vals, x):
    rp, ci, v, x = _int32(row_ptr), _int32(col_idx), _f64(vals), _f64(x)
    n = rp.shape[0] - 1
    b = int(round((v.size // max(ci.size, 1)) ** 0.5)) if ci.size else 1
    y = np.zeros(n * b)
    lib().oracle_spmv(n, b, _i(rp), _i(ci), _d(v), _d(x), _d(y))
    return y


def aggregate(row_ptr, col_idx):
    """Returns (agg, is_root, n_agg)."""
    rp, ci = _int32(row_ptr), _int32(col_idx)
    n = rp.shape[0] - 1
    agg = np.zeros(n, np.int32)
    root = np.zeros(n, np.int32)
    nagg = lib().oracle_aggregate(n, _i(rp), _i(ci), _i(agg), _i(root))
    if nagg < 0:
        raise OracleError(nagg, "aggregate")
    return agg, root.astype(bool), nagg


def colour(row_ptr, col_idx):
    rp, ci = _int32(row_ptr), _int32(col_idx)
    n = rp.shape[0] - 1
    col = np.zeros(n, np.int32)
    nc = lib().oracle_colour(n, _i(rp), _i(ci), _i(col))
    if nc < 0:
        raise OracleError(nc, "colour")
    return col, nc


def rap_tentative(row_ptr, col_idx, vals, b, agg, nc):
    rp, ci, v, ag = _int32(row_ptr), _int32(col_idx), _f64(vals), _int32(agg)
    n = rp.shape[0] - 1
    rpc = np.zeros(nc + 1, np.int32)
    nnz = lib().oracle_rap_tentative(n, b, _i(rp), _i(ci), _d(v), _i(ag), nc, _i(rpc), None, None)
    if nnz < 0:
        raise OracleError(nnz, "rap symbolic")
    cic = np.zeros(nnz, np.int32)
    vc = np.zeros((nnz, b, b))
    st = lib().oracle_rap_tentative(n, b, _i(rp), _i(ci), _d(v), _i(ag), nc, _i(rpc), _i(cic), _d(vc))
    if st < 0:
        raise OracleError(st, "rap numeric")
    return rpc, cic, vc


def block_inverse(a):
    a = _f64(a)
    m = a.shape[0]
    out = np.zeros_like(a)
    st = lib().oracle_block_inverse(m, _d(a), _d(out))
    if st:
        raise OracleError(st, "block_inverse")
    return out


def lu_factor(a):
    a = _f64(a).copy()
    n = a.shape[0]
    piv = np.zeros(n, np.int32)
    st = lib().oracle_lu_factor(n, _d(a), _i(piv))
    if st:
        raise OracleError(st, "lu_factor")
    return a, piv


def lu_solve(lu, piv, rhs):
    lu, piv, rhs = _f64(lu), _int32(piv), _f64(rhs)
    x = np.zeros_like(rhs)
    lib().oracle_lu_solve(lu.shape[0], _d(lu), _i(piv), _d(rhs), _d(x))
    return x


class Hierarchy:
    """The oracle's AMG hierarchy for one block system."""

    def __init__(self, row_ptr, col_idx, vals, b, field_of_dof, max_levels=10, max_coarse=2500,
                 n_pre=1, n_post=1, omega=0.5):
        self.rp, self.ci, self.v = _int32(row_ptr), _int32(col_idx), _f64(vals)
        self.b = int(b)
        self.n = self.rp.shape[0] - 1
        fm = _int32(field_of_dof)
        self.F = int(fm.max()) + 1
        self.fb = self.b // self.F
        self.params = Params(max_levels, max_coarse, n_pre, n_post, omega)
        h = C.c_void_p()
        st = lib().oracle_setup(self.n, self.ci.shape[0], self.b, _i(self.rp), _i(self.ci), _d(self.v),
                                _i(fm), C.byref(self.params), C.byref(h))
        if st:
            raise OracleError(st, "setup")
        self._h = h

    @classmethod
    def from_system(cls, sys, **kw):
        return cls(sys.row_ptr, sys.col_idx, sys.vals, sys.b, sys.field_of_dof, **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().oracle_free(h)
            self._h = None

    @property
    def num_levels(self):
        return lib().oracle_num_levels(self._h)

    def level_sizes(self, l):
        n, nnz, ncol, nagg = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        st = lib().oracle_level_sizes(self._h, l, C.byref(n), C.byref(nnz), C.byref(ncol), C.byref(nagg))
        if st:
            raise OracleError(st, "level_sizes")
        return n.value, nnz.value, ncol.value, nagg.value

    def level(self, l):
        """dict with row_ptr, col_idx, vals[nnzb,b,b], agg, colour, dinv[n,F,fb,fb]."""
        n, nnz, ncol, nagg = self.level_sizes(l)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros((nnz, self.b, self.b))
        coarsest = l == self.num_levels - 1
        agg = None if coarsest else np.zeros(n, np.int32)
        col = None if coarsest else np.zeros(n, np.int32)
        dinv = None if coarsest else np.zeros((n, self.F, self.fb, self.fb))
        lib().oracle_level_get(self._h, l, _i(rp), _i(ci), _d(v),
                               _i(agg) if agg is not None else None,
                               _i(col) if col is not None else None,
                               _d(dinv) if dinv is not None else None)
        return dict(n=n, nnzb=nnz, n_colours=ncol, n_agg=nagg, row_ptr=rp, col_idx=ci, vals=v,
                    agg=agg, colour=col, dinv=dinv)

    def bgs(self, l, x, rhs, sweeps=1):
        x = _f64(x).copy()
        rhs = _f64(rhs)
        st = lib().oracle_bgs(self._h, l, _d(x), _d(rhs), sweeps)
        if st:
            raise OracleError(st, "bgs")
        return x

    def vcycle(self, r):
        r = _f64(r)
        z = np.zeros_like(r)
        st = lib().oracle_vcycle(self._h, _d(r), _d(z))
        if st:
            raise OracleError(st, "vcycle")
        return z

    def fgmres(self, b, x0=None, tol=1e-8, restart=30, max_iter=1000, prec=0):
        """Returns (x, iterations, true relative residual, converged)."""
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        it = C.c_int()
        rr = C.c_double()
        st = lib().oracle_fgmres(self._h, _d(b), _d(x), tol, restart, max_iter, prec,
                                 C.byref(it), C.byref(rr))
        if st < 0:
            raise OracleError(st, "fgmres")
        return x, it.value, rr.value, st == OK
