"""Several multicolour Gauss-Seidel sweeps of the sub-solve A_ff x~ = r_f in
each field step of Algorithm 1 (amg_params.inner_sweeps) against the oracle's
iterated sub-solve (oracle inner_sweeps).

Bars: the FP64 V-cycle within 1e-12 of the oracle relative to its largest
entry; FGMRES iteration counts within +-1 at 1e-8; inner_sweeps 1 (and 0, read
as 1) bit for bit the default cycle.  On the saddle-point field blocks of the
Stokes and MHD systems the sweep on A_ff alone diverges (spectral radius of its
iteration above 1), so a V-cycle there still has a definite value to compare,
but the iteration counts are checked on systems whose field blocks the sweep
converges on (block Poisson, a diagonally dominant random system).
"""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "poisson_b1": lambda: (P.poisson_block(50, 1), dict(max_levels=4, max_coarse=0)),
    "poisson_b2_ragged": lambda: (P.poisson_block(37, 2), dict(max_levels=4, max_coarse=0)),
    "random_b4_f2": lambda: (P.random_block_system(23, 4, [0, 0, 1, 1], seed=5), dict(max_levels=3, max_coarse=0)),
    "mhd2d_16": lambda: (P.mhd2d(16, 2), dict(max_levels=3, max_coarse=0)),
    "stokes3d_9": lambda: (P.stokes3d(9, 1), dict(max_levels=3, max_coarse=0)),
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


def apply(g, r):
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("k", [2, 3, 5])
def test_inner_sweeps_vcycle_fp64_matches_oracle(name, k):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, inner_sweeps=k, **kw)
    assert g.stats()["inner_sweeps"] == k
    o = oracle.Hierarchy.from_system(s, inner_sweeps=k, **kw)
    r = np.random.default_rng(11).standard_normal(s.n_unknowns)
    assert rel_max(apply(g, r), o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("variant", [dict(n_pre=0, n_post=2), dict(n_pre=2, n_post=1, omega=0.7),
                                     dict(n_pre=1, n_post=0), dict(cycle_prec=64, use_graph=0, use_pdl=0)])
def test_inner_sweeps_cycle_variants_match_oracle(variant):
    s = P.random_block_system(31, 4, [0, 0, 1, 1], seed=8)
    kw = dict(max_levels=3, max_coarse=0)
    kw.update(variant)
    okw = {k: v for k, v in kw.items() if k not in ("cycle_prec", "use_graph", "use_pdl")}
    g = make_solver(s, inner_sweeps=4, **kw)
    o = oracle.Hierarchy.from_system(s, inner_sweeps=4, **okw)
    assert rel_max(apply(g, s.rhs), o.vcycle(s.rhs)) <= 1e-12


@pytest.mark.parametrize("at", [0, 2, 4, 6])
def test_inner_sweeps_do_not_depend_on_the_row_mapping(at):
    # the inner sweeps run one kernel whatever mapping the single sweep would
    # take; the field residual before them follows the level's SpMV mapping
    s, kw = SYSTEMS["poisson_b2_ragged"]()
    o = oracle.Hierarchy.from_system(s, inner_sweeps=3, **kw)
    g = make_solver(s, inner_sweeps=3, autotune=at, **kw)
    r = np.random.default_rng(5).standard_normal(s.n_unknowns)
    assert rel_max(apply(g, r), o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("k", [0, 1])
def test_one_inner_sweep_is_the_default_cycle_bitwise(k):
    s = P.mhd2d(20, 3)
    kw = dict(max_levels=4, max_coarse=0, autotune=0)
    r = np.random.default_rng(2).standard_normal(s.n_unknowns)
    z0 = apply(make_solver(s, **kw), r)
    g = make_solver(s, inner_sweeps=k, **kw)
    assert g.stats()["inner_sweeps"] == 1
    assert np.array_equal(apply(g, r), z0)


@pytest.mark.parametrize("name,restart", [("poisson_b1", 30), ("poisson_b2_ragged", 10), ("random_b4_f2", 30)])
@pytest.mark.parametrize("k", [2, 4])
def test_inner_sweeps_fgmres_iterations_match_oracle(name, restart, k):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, inner_sweeps=k, **kw)
    o = oracle.Hierarchy.from_system(s, inner_sweeps=k, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=restart, max_iter=500)
    _, it_o, _, _ = o.fgmres(s.rhs, tol=1e-8, restart=restart, max_iter=500)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    assert abs(it - it_o) <= 1, (it, it_o)


def test_more_inner_sweeps_fewer_iterations_on_block_poisson():
    # the sweep on A_ff converges on these blocks: the sub-solve tends to the
    # exact field solve and the outer iteration count drops
    s = P.poisson_block(64, 2)
    its = []
    for k in (1, 2, 4, 8):
        g = make_solver(s, inner_sweeps=k, max_levels=4, max_coarse=0)
        x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
        st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=500)
        assert st == bamg.BAMG_OK and rr <= 1e-8
        its.append(it)
    assert its[0] > its[1] > its[2] > its[3], its


def test_inner_sweeps_fp32_cycle_reaches_fp64_residual():
    s = P.poisson_block(80, 2)
    g = make_solver(s, inner_sweeps=3, cycle_prec=32, max_levels=4, max_coarse=0)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=500)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    res = s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(s.rhs) <= 1e-8


def test_inner_sweeps_on_a_batch_match_each_system_alone():
    members = [P.poisson_block(N, 2) for N in (19, 30, 24)]
    bt = P.concatenate(members)
    s = bt.system
    kw = dict(max_levels=3, max_coarse=0)
    g = bamg.BatchSolver(bt.sys_node_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b,
                         s.field_of_dof, inner_sweeps=3, **kw)
    r = np.random.default_rng(9).standard_normal(s.n_unknowns)
    zg = apply(g, r)
    off = bt.sys_node_off * s.b
    for q, m in enumerate(bt.members):
        o = oracle.Hierarchy.from_system(m, inner_sweeps=3, **kw)
        if o.num_levels != g.num_levels:
            continue  # a member that coarsens differently alone is not comparable level by level
        zo = o.vcycle(r[off[q]:off[q + 1]])
        assert rel_max(zg[off[q]:off[q + 1]], zo) <= 1e-12, q


@pytest.mark.parametrize("bad", [dict(inner_sweeps=65), dict(inner_sweeps=-1), dict(inner_sweeps=2, sub_solver=1),
                                 dict(inner_sweeps=2, sub_solver=2)])
def test_inner_sweeps_validation(bad):
    s = P.poisson_block(12, 2)
    with pytest.raises(bamg.BamgError) as e:
        make_solver(s, **bad)
    assert e.value.status == bamg.BAMG_EINVAL


def test_inner_sweeps_need_dof_fields():
    s = P.mhd2d_q2q1(12, 1)
    with pytest.raises(bamg.BamgError) as e:
        bamg.FieldSolver(s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b,
                         inner_sweeps=2, max_levels=3, max_coarse=0)
    assert e.value.status == bamg.BAMG_EINVAL
