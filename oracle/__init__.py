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
_SRC2 = os.path.join(_HERE, "learned_oracle.c")
_HDR = os.path.join(_HERE, "bamg_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbamg_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ESINGULAR_BLOCK, ESINGULAR_COARSE, NOT_CONVERGED = 0, -1, -2, -3, -4, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fused multiply-add)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest_src = max(os.path.getmtime(f) for f in (_SRC, _SRC2, _HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest_src:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, _SRC2, "-lm"]
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
                ("n_post", C.c_int), ("omega", C.c_double), ("smooth_p", C.c_int), ("omega_p", C.c_double),
                ("omega_s_arr", _dp), ("omega_s_len", C.c_longlong), ("omega_p_arr", _dp),
                ("omega_p_len", C.c_longlong), ("mlp", _dp), ("mlp_levels", C.c_int), ("sub_ilu", C.c_int),
                ("n_node_fields", C.c_int), ("node_field_off", _ip), ("sub_schwarz", C.c_int),
                ("schwarz_overlap", C.c_int), ("inner_sweeps", C.c_int)]


NFEAT, MLP_H, MLP_OUT = 8, 64, 2
MLP_NTRAIN = MLP_H * NFEAT + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT
MLP_NPARAMS = MLP_NTRAIN + 2 * NFEAT


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
    L.oracle_ilu0_field.argtypes = [C.c_int, C.c_int, _ip, _ip, _ip, _dp, C.c_int, _dp]
    L.oracle_ilu0_solve.argtypes = [C.c_int, C.c_int, _ip, _ip, _dp, _dp, _dp]
    L.oracle_ilu0_field_ordered.argtypes = [C.c_int, C.c_int, _ip, _ip, _ip, _dp, C.c_int, _ip, _dp]
    L.oracle_ilu0_solve_ordered.argtypes = [C.c_int, C.c_int, _ip, _ip, _ip, _dp, _dp, _dp]
    L.oracle_free.restype = None
    L.oracle_level_fields.argtypes = [C.c_void_p, C.c_int, _ip, _ip]
    L.oracle_num_levels.argtypes = [C.c_void_p]
    L.oracle_level_sizes.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _ip, _ip]
    L.oracle_level_get.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _dp, _ip, _ip, _dp]
    L.oracle_bgs.argtypes = [C.c_void_p, C.c_int, _dp, _dp, C.c_int]
    L.oracle_vcycle.argtypes = [C.c_void_p, _dp, _dp]
    L.oracle_fgmres.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, C.c_int, C.c_int, _ip, _dp]
    L.oracle_prolongator.argtypes = [C.c_int, C.c_int, _ip, _ip, _ip, _dp, _ip, C.c_int, _dp, _ip, _ip, _dp]
    L.oracle_rap_general.argtypes = [C.c_int, C.c_int, _ip, _ip, _ip, _dp, C.c_int, _ip, _ip, _dp, _ip, _ip, _dp]
    L.oracle_level_p_nnz.argtypes = [C.c_void_p, C.c_int]
    L.oracle_level_get_p.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _dp]
    L.oracle_level_omega.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
    L.oracle_features.argtypes = [C.c_int, C.c_int, _ip, _ip, _ip, _dp, _ip, C.c_int, C.c_int, _dp, _dp]
    L.oracle_mlp_forward.argtypes = [_dp, _dp, C.c_int, _dp]
    L.oracle_mlp_grad.argtypes = [_dp, _dp, _dp, _ip, C.c_int, _dp, _dp]
    L.oracle_adam.argtypes = [_dp, _dp, _dp, _dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
    L.oracle_mlp_clip.argtypes = [C.c_int, C.c_double]
    L.oracle_mlp_clip.restype = C.c_double


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


def ilu0_field(row_ptr, col_idx, vals, b, field_of_dof, f, pos=None):
    """ILU(0) factors of the field-f part A_ff, [nnzb, fb, fb] (see
    oracle_ilu0_field); pos: elimination position of every node (None: natural)."""
    rp, ci, v = _int32(row_ptr), _int32(col_idx), _f64(vals)
    fm = _int32(field_of_dof)
    fb = int(b) // (int(fm.max()) + 1)
    n = rp.shape[0] - 1
    lu = np.zeros((ci.size, fb, fb))
    ps = None if pos is None else _int32(pos)
    st = lib().oracle_ilu0_field_ordered(n, int(b), _i(fm), _i(rp), _i(ci), _d(v), int(f),
                                         None if ps is None else _i(ps), _d(lu))
    if st:
        raise OracleError(st, "ilu0_field")
    return lu


def ilu0_solve(row_ptr, col_idx, lu, r, pos=None):
    """(L U)^{-1} r for the factors of ilu0_field (same pos)."""
    rp, ci, lu = _int32(row_ptr), _int32(col_idx), _f64(lu)
    n, fb = rp.shape[0] - 1, lu.shape[1]
    x = np.zeros(n * fb)
    ps = None if pos is None else _int32(pos)
    st = lib().oracle_ilu0_solve_ordered(n, fb, _i(rp), _i(ci), None if ps is None else _i(ps), _d(lu),
                                         _d(_f64(r)), _d(x))
    if st:
        raise OracleError(st, "ilu0_solve")
    return x


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


def _fields(field_of_dof):
    fm = _int32(field_of_dof)
    F = int(fm.max()) + 1
    return fm, F, fm.size // F


def prolongator(row_ptr, col_idx, vals, field_of_dof, agg, nc, omega_p):
    """Smoothed prolongator: (p_rp, p_ci, p_v[nnz, F, fb, fb]); omega_p[nc, F]."""
    rp, ci, v, ag = _int32(row_ptr), _int32(col_idx), _f64(vals), _int32(agg)
    fm, F, fb = _fields(field_of_dof)
    n, b = rp.shape[0] - 1, fm.size
    om = _f64(np.broadcast_to(np.asarray(omega_p, dtype=np.float64), (nc, F)))
    prp = np.zeros(n + 1, np.int32)
    nnz = lib().oracle_prolongator(n, b, _i(fm), _i(rp), _i(ci), _d(v), _i(ag), nc, _d(om), _i(prp), None, None)
    if nnz < 0:
        raise OracleError(nnz, "prolongator symbolic")
    pci = np.zeros(nnz, np.int32)
    pv = np.zeros((nnz, F, fb, fb))
    st = lib().oracle_prolongator(n, b, _i(fm), _i(rp), _i(ci), _d(v), _i(ag), nc, _d(om), _i(prp), _i(pci),
                                  _d(pv))
    if st < 0:
        raise OracleError(st, "prolongator")
    return prp, pci, pv


def rap_general(row_ptr, col_idx, vals, field_of_dof, nc, p_rp, p_ci, p_v):
    """A_c = P^T A P with a field-block-diagonal P: (rp_c, ci_c, vals_c[nnz, b, b])."""
    rp, ci, v = _int32(row_ptr), _int32(col_idx), _f64(vals)
    fm, F, fb = _fields(field_of_dof)
    prp, pci, pv = _int32(p_rp), _int32(p_ci), _f64(p_v)
    n, b = rp.shape[0] - 1, fm.size
    rpc = np.zeros(nc + 1, np.int32)
    nnz = lib().oracle_rap_general(n, b, _i(fm), _i(rp), _i(ci), _d(v), nc, _i(prp), _i(pci), _d(pv), _i(rpc),
                                   None, None)
    if nnz < 0:
        raise OracleError(nnz, "rap_general symbolic")
    cic = np.zeros(nnz, np.int32)
    vc = np.zeros((nnz, b, b))
    st = lib().oracle_rap_general(n, b, _i(fm), _i(rp), _i(ci), _d(v), nc, _i(prp), _i(pci), _d(pv), _i(rpc),
                                  _i(cic), _d(vc))
    if st < 0:
        raise OracleError(st, "rap_general")
    return rpc, cic, vc


def features(row_ptr, col_idx, vals, field_of_dof, agg, nc, level):
    """(node_feat[n, F, NFEAT], agg_feat[nc, F, NFEAT])."""
    rp, ci, v, ag = _int32(row_ptr), _int32(col_idx), _f64(vals), _int32(agg)
    fm, F, _ = _fields(field_of_dof)
    n = rp.shape[0] - 1
    nf = np.zeros((n, F, NFEAT))
    af = np.zeros((nc, F, NFEAT))
    st = lib().oracle_features(n, fm.size, _i(fm), _i(rp), _i(ci), _d(v), _i(ag), nc, level, _d(nf), _d(af))
    if st:
        raise OracleError(st, "features")
    return nf, af


def mlp_forward(params, x):
    p, x = _f64(params), _f64(x).reshape(-1, NFEAT)
    assert p.size == MLP_NPARAMS
    y = np.zeros((x.shape[0], MLP_OUT))
    lib().oracle_mlp_forward(_d(p), _d(x), x.shape[0], _d(y))
    return y


def mlp_grad(params, x, t, head):
    """(loss, grad[MLP_NTRAIN]) of the mean squared error of the selected heads."""
    p, x, t, hd = _f64(params), _f64(x).reshape(-1, NFEAT), _f64(t), _int32(head)
    assert p.size == MLP_NPARAMS and t.size == x.shape[0] == hd.size
    g = np.zeros(MLP_NTRAIN)
    loss = C.c_double()
    st = lib().oracle_mlp_grad(_d(p), _d(x), _d(t), _i(hd), x.shape[0], _d(g), C.byref(loss))
    if st:
        raise OracleError(st, "mlp_grad")
    return loss.value, g


def adam(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on params[:MLP_NTRAIN], m, v (float64 arrays)."""
    st = lib().oracle_adam(_d(params), _d(_f64(grad)), _d(m), _d(v), t, lr, beta1, beta2, eps)
    if st:
        raise OracleError(st, "adam")


def mlp_clip(head, w):
    return np.vectorize(lambda z: lib().oracle_mlp_clip(head, float(z)))(np.asarray(w, dtype=np.float64))


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
                 n_pre=1, n_post=1, omega=0.5, smooth_p=0, omega_p=0.0, omega_s_arr=None, omega_p_arr=None,
                 mlp=None, mlp_levels=0, sub_ilu=0, node_field_off=None, sub_schwarz=0, schwarz_overlap=1,
                 inner_sweeps=1):
        """``node_field_off``: node ranges of fields on disjoint node sets
        (non-co-located fields; every dof of a node in the node's field, so
        ``field_of_dof`` is all zero); None for co-located fields."""
        self.rp, self.ci, self.v = _int32(row_ptr), _int32(col_idx), _f64(vals)
        self.b = int(b)
        self.n = self.rp.shape[0] - 1
        fm = _int32(field_of_dof)
        self.F = int(fm.max()) + 1
        self.fsize = [int((fm == f).sum()) for f in range(self.F)]  # dofs per field (may differ)
        self.fb = max(self.fsize)
        # keep the weight arrays alive for the duration of the setup call
        self._ws = None if omega_s_arr is None else _f64(omega_s_arr).ravel()
        self._wp = None if omega_p_arr is None else _f64(omega_p_arr).ravel()
        self._mlp = None if mlp is None else _f64(mlp).ravel()
        if self._mlp is not None:
            assert self._mlp.size == MLP_NPARAMS
        self.params = Params(max_levels, max_coarse, n_pre, n_post, omega, int(smooth_p), float(omega_p),
                             None if self._ws is None else _d(self._ws),
                             0 if self._ws is None else self._ws.size,
                             None if self._wp is None else _d(self._wp),
                             0 if self._wp is None else self._wp.size,
                             None if self._mlp is None else _d(self._mlp), int(mlp_levels), int(sub_ilu),
                             0, None, int(sub_schwarz), int(schwarz_overlap), int(inner_sweeps))
        self._foff = None if node_field_off is None else _int32(node_field_off)
        self.NF = 1
        if self._foff is not None:
            self.NF = self._foff.size - 1
            self.params.n_node_fields = self.NF
            self.params.node_field_off = _i(self._foff)
        h = C.c_void_p()
        st = lib().oracle_setup(self.n, self.ci.shape[0], self.b, _i(self.rp), _i(self.ci), _d(self.v),
                                _i(fm), C.byref(self.params), C.byref(h))
        if st:
            raise OracleError(st, "setup")
        self._h = h

    @classmethod
    def from_system(cls, sys, **kw):
        if getattr(sys, "node_field_off", None) is not None:
            kw.setdefault("node_field_off", sys.node_field_off)
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
        """dict with row_ptr, col_idx, vals[nnzb,b,b], agg, colour, dinv[n,F,fb,fb]
        (fields of unequal size: dinv a list over the fields of [n,fs,fs])."""
        n, nnz, ncol, nagg = self.level_sizes(l)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros((nnz, self.b, self.b))
        coarsest = l == self.num_levels - 1
        agg = None if coarsest else np.zeros(n, np.int32)
        col = None if coarsest else np.zeros(n, np.int32)
        dinv = None if coarsest else np.zeros((n, sum(fs * fs for fs in self.fsize)))
        lib().oracle_level_get(self._h, l, _i(rp), _i(ci), _d(v),
                               _i(agg) if agg is not None else None,
                               _i(col) if col is not None else None,
                               _d(dinv) if dinv is not None else None)
        if dinv is not None:
            if len(set(self.fsize)) == 1:
                dinv = dinv.reshape(n, self.F, self.fb, self.fb)
            else:
                parts, o = [], 0
                for fs in self.fsize:
                    parts.append(dinv[:, o:o + fs * fs].reshape(n, fs, fs))
                    o += fs * fs
                dinv = parts
        return dict(n=n, nnzb=nnz, n_colours=ncol, n_agg=nagg, row_ptr=rp, col_idx=ci, vals=v,
                    agg=agg, colour=col, dinv=dinv)

    def fields(self, l):
        """(node_off[NF+1], colour_off[NF+1]) of level l; colour_off is None
        on the coarsest level."""
        no = np.zeros(self.NF + 1, np.int32)
        co = np.zeros(self.NF + 1, np.int32)
        st = lib().oracle_level_fields(self._h, l, _i(no), _i(co))
        if st < 0:
            raise OracleError(st, "level_fields")
        return no, (None if l == self.num_levels - 1 else co)

    def prolongator(self, l):
        """(p_rp, p_ci, p_v[nnz, F, fb, fb]) of a level coarsened with smooth_p = 1."""
        n = self.level_sizes(l)[0]
        nnz = lib().oracle_level_p_nnz(self._h, l)
        if nnz <= 0:
            raise OracleError(nnz, "level_p")
        prp = np.zeros(n + 1, np.int32)
        pci = np.zeros(nnz, np.int32)
        pv = np.zeros((nnz, self.F, self.fb, self.fb))
        st = lib().oracle_level_get_p(self._h, l, _i(prp), _i(pci), _d(pv))
        if st:
            raise OracleError(st, "level_get_p")
        return prp, pci, pv

    def omega(self, l):
        """(omega_s[n, F], omega_p[n_agg, F]) of a level with a smoother."""
        n, _, _, nagg = self.level_sizes(l)
        ws = np.zeros((n, self.F))
        wp = np.zeros((max(nagg, 0), self.F))
        st = lib().oracle_level_omega(self._h, l, _d(ws), _d(wp))
        if st:
            raise OracleError(st, "level_omega")
        return ws, wp

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
