"""FP32 coarsest solve of FP32 cycles (amg_params.coarse_prec = 32).

The LU with partial pivoting of the coarsest matrix rounded to FP32 is
backward stable: the computed solution of A z = r has a relative error of at
most about c * nd * u * kappa(A) (u = 2^-24, modest growth), which the
one-level tests below check against an FP64 dense solve, on matrices of the
shared-memory size (nd <= 223) and of the cooperative size.  On multilevel
hierarchies the FP32 coarse solve must leave the FGMRES iteration count to
1e-8 within one of the FP64 coarse solve's.
"""
import numpy as np
import pytest

from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bamg.load()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_solver(s, **kw):
    return bamg.Solver(dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b, s.field_of_dof, **kw)


def dense(s):
    nd = s.n_nodes * s.b
    a = np.zeros((nd, nd))
    for i in range(s.n_nodes):
        for k in range(s.row_ptr[i], s.row_ptr[i + 1]):
            j = s.col_idx[k]
            a[i * s.b:(i + 1) * s.b, j * s.b:(j + 1) * s.b] = s.vals[k]
    return a


@pytest.mark.parametrize("s_fn", [lambda: P.random_block_system(6, 6, [0] * 6, seed=3),       # nd 216: one CTA
                                  lambda: P.random_block_system(8, 4, [0, 0, 1, 1], seed=4),   # nd 256: cooperative
                                  lambda: P.poisson_block(14, 2),                              # nd 450
                                  lambda: P.mhd2d(12, 5)])                                     # nd 1014
def test_fp32_coarse_solve_within_lu_bound(s_fn):
    s = s_fn()
    a = dense(s)
    nd = a.shape[0]
    g = make_solver(s, max_levels=1, cycle_prec=32, coarse_prec=32)
    st = g.stats()
    assert st["coarse_prec"] == 32 and st["coarse_unknowns"] == nd
    r = P.uniform_pm1(21, 0, nd)
    z = torch.empty(nd, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    zs = np.linalg.solve(a, r)
    err = np.abs(z.cpu().numpy() - zs).max() / np.abs(zs).max()
    kappa = np.linalg.cond(a, np.inf)
    assert err <= 4.0 * nd * U32 * kappa, (err, kappa)
    # the FP64 coarse solve of the same hierarchy is far more accurate: the
    # FP32 path is the one that ran
    g64 = make_solver(s, max_levels=1, cycle_prec=32, coarse_prec=64)
    assert g64.stats()["coarse_prec"] == 64


@pytest.mark.parametrize("s_fn,levels", [(lambda: P.mhd2d(41, 3), 4), (lambda: P.mhd2d(40, 4), 2),
                                         (lambda: P.stokes3d(12, 1), 2)])
def test_fp32_coarse_keeps_iterations(s_fn, levels):
    s = s_fn()
    its = {}
    for cp in (64, 32):
        g = make_solver(s, max_levels=levels, max_coarse=0, cycle_prec=32, coarse_prec=cp)
        assert g.stats()["coarse_prec"] == cp
        b = dev(s.rhs)
        x = torch.zeros_like(b)
        st, it, rr = g.solve(b, x, tol=1e-8, restart=30, max_iter=1000)
        assert st == bamg.BAMG_OK and rr <= 1e-8
        its[cp] = it
    assert abs(its[32] - its[64]) <= 1, its


def test_coarse_prec_validation():
    s = P.mhd2d(8, 1)
    for kw in (dict(coarse_prec=32, cycle_prec=64), dict(coarse_prec=16, cycle_prec=32)):
        with pytest.raises(bamg.BamgError) as e:
            make_solver(s, max_levels=2, max_coarse=0, **kw)
        assert e.value.status == bamg.BAMG_EINVAL


@pytest.mark.parametrize("coarse_tc", [1, 0])
def test_fp32_coarse_tensor_core_switch(coarse_tc):
    """Coarsest matrices above the one-CTA size go to the tensor-core LU by
    default (coarse_tc 1); coarse_tc 0 keeps the CUDA-core LU.  Both stay within
    the LU bound."""
    s = P.mhd2d(12, 5)  # nd 1014
    a = dense(s)
    nd = a.shape[0]
    g = make_solver(s, max_levels=1, cycle_prec=32, coarse_prec=32, coarse_tc=coarse_tc)
    st = g.stats()
    assert st["coarse_tc"] == coarse_tc
    r = P.uniform_pm1(22, 0, nd)
    z = torch.empty(nd, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    zs = np.linalg.solve(a, r)
    err = np.abs(z.cpu().numpy() - zs).max() / np.abs(zs).max()
    assert err <= 4.0 * nd * U32 * np.linalg.cond(a, np.inf)
    small = make_solver(P.random_block_system(6, 6, [0] * 6, seed=3), max_levels=1, cycle_prec=32, coarse_prec=32)
    assert small.stats()["coarse_tc"] == 0  # 216 unknowns: the one-CTA LU
