"""Restricted Schwarz on aggregates as the sub-solve of Algorithm 1 on the GPU
(Sec. 5: one Schwarz iteration with overlap one per field block; subdomains
= the level's aggregates, the reading of the oracle's sub_schwarz = 2),
against the oracle.

Bars: the FP64 V-cycle within 1e-12 of the oracle relative to its largest
entry (the GPU applies the own rows of each local inverse, formed at setup
from the same LU with partial pivoting; the oracle solves with the LU, so the
two differ by rounding only); FGMRES iteration counts within +-1 at 1e-8;
overlap 0 (block Jacobi over the aggregates) likewise; the FP32 cycle reaches
the FP64 residual 1e-8.
"""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "stokes2d_32": lambda: (P.stokes2d(32, 1), dict(max_levels=3, max_coarse=0)),
    "mhd2d_16": lambda: (P.mhd2d(16, 2), dict(max_levels=3, max_coarse=0)),
    "mhd2d_41_ragged": lambda: (P.mhd2d(41, 3), dict(max_levels=4, max_coarse=0)),
    "random_b4_f2": lambda: (P.random_block_system(23, 4, [0, 0, 1, 1], seed=5), dict(max_levels=3, max_coarse=0)),
    "poisson_b1": lambda: (P.poisson_block(50, 1), dict(max_levels=4, max_coarse=0)),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bamg.load()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_solver(s, **kw):
    return bamg.Solver(dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b, s.field_of_dof, **kw)


def rel_max(a, ref):
    scale = np.abs(ref).max()
    return np.abs(a - ref).max() / (scale if scale > 0 else 1.0)


@pytest.mark.parametrize("overlap", [1, 0])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_schwarz_vcycle_fp64_matches_oracle(name, overlap):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, sub_solver=2, schwarz_overlap=overlap, **kw)
    o = oracle.Hierarchy.from_system(s, sub_schwarz=2, schwarz_overlap=overlap, **kw)
    r = np.random.default_rng(7).standard_normal(s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("variant", [dict(n_pre=0, n_post=2), dict(n_pre=2, n_post=1, omega=0.6)])
def test_schwarz_cycle_variants_match_oracle(variant):
    s = P.mhd2d(12, 4)
    kw = dict(max_levels=3, max_coarse=0)
    kw.update(variant)
    g = make_solver(s, sub_solver=2, **kw)
    o = oracle.Hierarchy.from_system(s, sub_schwarz=2, **kw)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(s.rhs), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(s.rhs)) <= 1e-12


@pytest.mark.parametrize("name,restart", [("mhd2d_16", 30), ("mhd2d_41_ragged", 10)])
def test_schwarz_fgmres_iterations_match_oracle(name, restart):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, sub_solver=2, **kw)
    o = oracle.Hierarchy.from_system(s, sub_schwarz=2, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=restart, max_iter=3000)
    _, it_o, _, _ = o.fgmres(s.rhs, tol=1e-8, restart=restart, max_iter=3000)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    assert abs(it - it_o) <= 1, (it, it_o)


def test_schwarz_fp32_cycle_reaches_fp64_residual():
    s = P.mhd2d(48, 2)
    g = make_solver(s, sub_solver=2, cycle_prec=32, max_levels=4, max_coarse=0)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=3000)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    res = s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(s.rhs) <= 1e-8


@pytest.mark.parametrize("N", [12, 21])
def test_schwarz_on_fields_on_node_sets_matches_oracle(N):
    s = P.mhd2d_q2q1(N, 1)
    kw = dict(max_levels=4, max_coarse=0, omega=0.6)
    g = bamg.FieldSolver(s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b,
                         sub_solver=2, **kw)
    o = oracle.Hierarchy.from_system(s, sub_schwarz=2, **kw)
    r = np.random.default_rng(3).standard_normal(s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= 1e-12
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=3000)
    _, it_o, _, _ = o.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=3000)
    assert st == bamg.BAMG_OK and abs(it - it_o) <= 1, (it, it_o)


def test_schwarz_needs_fewer_iterations_than_the_sweep_on_mixed_elements():
    s = P.mhd2d_q2q1(16, 1)
    kw = dict(max_levels=4, max_coarse=0, omega=0.6)
    its = []
    for sub in (0, 2):
        g = bamg.FieldSolver(s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b,
                             sub_solver=sub, **kw)
        x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
        st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=3000)
        assert st == bamg.BAMG_OK
        its.append(it)
    assert 2 * its[1] < its[0], its


def test_schwarz_rejects_subdomains_beyond_its_size():
    s = P.stokes3d(8, 1)  # 5^3-node subdomains of 4 dofs: 500 unknowns
    with pytest.raises(bamg.BamgError) as e:
        make_solver(s, sub_solver=2, max_levels=3, max_coarse=0)
    assert e.value.status == bamg.BAMG_EUNSUPPORTED
