"""The persistent multicolour sweep (every colour of a field step of
Algorithm 1 in one launch, tiles waiting on per-tile flags) against the
per-colour launches and the oracle.

Bars: bit for bit equal to the per-colour thread-per-row (sweep = 2) and
four-lanes-per-row (sweep = 3) kernels, whose sums it repeats in the same
order, in FP64 and FP32, over repeated launches (the flags carry an epoch and
are never cleared); FP64 V-cycle within 1e-12 of the oracle; FGMRES iteration
counts within +-1 of the oracle; fields on node sets and batches bit for bit
against their per-colour cycles.
"""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "stokes2d_32": lambda: (P.stokes2d(32, 1), dict(max_levels=3, max_coarse=0)),
    "mhd2d_41_ragged": lambda: (P.mhd2d(41, 3), dict(max_levels=4, max_coarse=0)),
    "stokes3d_9": lambda: (P.stokes3d(9, 1), dict(max_levels=3, max_coarse=0)),
    "stokes3d_24": lambda: (P.stokes3d(24, 2), dict(max_levels=3, max_coarse=0)),
    "random_b4_f2": lambda: (P.random_block_system(23, 4, [0, 0, 1, 1], seed=5), dict(max_levels=3, max_coarse=0)),
    "random_b6_f1": lambda: (P.random_block_system(19, 6, [0] * 6, seed=6), dict(max_levels=3, max_coarse=0)),
    "poisson_b1": lambda: (P.poisson_block(50, 1), dict(max_levels=4, max_coarse=0)),
    "poisson_b2": lambda: (P.poisson_block(30, 2), dict(max_levels=10, max_coarse=100)),
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


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("g4", [0, 1])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_sweep_equals_per_colour_kernels_bitwise(name, g4, prec):
    s, kw = SYSTEMS[name]()
    at = 4 if g4 else 2  # the per-colour kernel with the same lanes per row
    per_colour = make_solver(s, autotune=at, sweep=1, cycle_prec=prec, **kw)
    swept = make_solver(s, autotune=at, sweep=3 if g4 else 2, cycle_prec=prec, **kw)
    levels = swept.stats()["levels"][:-1]
    assert all(lv["smoother_mapping"] == ("sweep-split" if g4 else "sweep") for lv in levels), levels
    assert all(lv["sweep_tiles"] > 0 for lv in levels)
    r = dev(np.random.default_rng(21).standard_normal(s.n_unknowns))
    z0, z1 = torch.empty_like(r), torch.empty_like(r)
    per_colour.apply(r, z0)
    swept.apply(r, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)
    # every further launch finds the flags of the previous one: same bits
    for _ in range(3):
        z2 = torch.empty_like(r)
        swept.apply(r, z2)
        torch.cuda.synchronize()
        assert torch.equal(z2, z0)


@pytest.mark.parametrize("sweep", [2, 3])
@pytest.mark.parametrize("name", ["stokes2d_32", "mhd2d_41_ragged", "stokes3d_9", "random_b4_f2", "poisson_b2"])
def test_sweep_vcycle_fp64_matches_oracle(name, sweep):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, autotune=0, sweep=sweep, **kw)
    o = oracle.Hierarchy.from_system(s, **kw)
    r = np.random.default_rng(7).standard_normal(s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("variant", [dict(n_pre=0, n_post=2), dict(n_pre=2, n_post=3, omega=0.6)])
def test_sweep_cycle_variants_match_oracle(variant):
    s = P.mhd2d(12, 4)
    kw = dict(max_levels=3, max_coarse=0)
    kw.update(variant)
    g = make_solver(s, autotune=0, sweep=2, **kw)
    o = oracle.Hierarchy.from_system(s, **kw)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(s.rhs), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(s.rhs)) <= 1e-12


@pytest.mark.parametrize("name,restart", [("mhd2d_41_ragged", 10), ("stokes3d_9", 30)])
def test_sweep_fgmres_iterations_match_oracle(name, restart):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, autotune=0, sweep=3, **kw)
    o = oracle.Hierarchy.from_system(s, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=restart, max_iter=3000)
    _, it_o, rr_o, _ = o.fgmres(s.rhs, tol=1e-8, restart=restart, max_iter=3000)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    assert abs(it - it_o) <= 1, (it, it_o)


def test_sweep_fp32_cycle_reaches_fp64_residual_3d():
    s = P.stokes3d(24, 2)
    g = make_solver(s, max_levels=10, max_coarse=2500, cycle_prec=32, coarse_prec=32, autotune=0, sweep=3)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=50, max_iter=3000)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    # the true residual, with the oracle's SpMV
    res = s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(s.rhs) <= 1e-8


def test_sweep_on_fields_on_node_sets_bitwise():
    s = P.mhd2d_q2q1(16, 1)
    kw = dict(max_levels=4, max_coarse=0, omega=0.6)
    args = (s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b)
    per_colour = bamg.FieldSolver(*args, autotune=2, sweep=1, **kw)
    swept = bamg.FieldSolver(*args, autotune=2, sweep=2, **kw)
    r = dev(np.random.default_rng(5).standard_normal(s.n_unknowns))
    z0, z1 = torch.empty_like(r), torch.empty_like(r)
    per_colour.apply(r, z0)
    swept.apply(r, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)


def test_sweep_on_a_batch_bitwise():
    bt = P.mhd2d_batch(6, 3, nmin=8, nmax=24)
    s = bt.system
    args = (bt.sys_node_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.n_nodes, s.nnzb, s.b,
            s.field_of_dof)
    kw = dict(max_levels=4, max_coarse=0, cycle_prec=32)
    hs = [bamg.amg_setup_batched(*args, bamg.amg_default_params(autotune=2, sweep=sw, **kw)) for sw in (1, 2)]
    try:
        r = dev(np.random.default_rng(2).standard_normal(s.n_unknowns))
        zs = []
        for h in hs:
            z = torch.empty_like(r)
            bamg.amg_apply(h, r, z)
            zs.append(z)
        torch.cuda.synchronize()
        assert torch.equal(zs[0], zs[1])
        # the same cycle bit for bit: the same per-system FGMRES histories
        res = []
        for h in hs:
            x = torch.zeros_like(r)
            st, its, rrs = bamg.fgmres_solve_batched(h, dev(s.rhs), x, 1e-8, 30, 600)
            assert st in (bamg.BAMG_OK, bamg.BAMG_NOT_CONVERGED)
            res.append((its.copy(), rrs.copy()))
        assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    finally:
        for h in hs:
            bamg.amg_destroy(h)


def test_sweep_parameter_is_validated():
    s = P.stokes2d(8, 1)
    with pytest.raises(bamg.BamgError) as e:
        make_solver(s, sweep=4, max_levels=2, max_coarse=0)
    assert e.value.status == bamg.BAMG_EINVAL


def test_tuning_is_reused_for_the_same_level_shape():
    s = P.stokes3d(24, 3)
    kw = dict(max_levels=3, max_coarse=0, cycle_prec=32)
    g1 = make_solver(s, **kw)
    g2 = make_solver(s, **kw)
    l1, l2 = g1.stats()["levels"][:-1], g2.stats()["levels"][:-1]
    assert all(lv["tune_cached"] == 1 for lv in l2)
    for a, b in zip(l1, l2):
        assert a["smoother_mapping"] == b["smoother_mapping"] and a["residual_mapping"] == b["residual_mapping"]
        assert a["tune_us"] == b["tune_us"]
    r = dev(np.random.default_rng(4).standard_normal(s.n_unknowns))
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    g1.apply(r, z1)
    g2.apply(r, z2)
    torch.cuda.synchronize()
    assert torch.equal(z1, z2)
    # a forced launch mode is not overridden by an earlier tuning of the shape
    g3 = make_solver(s, sweep=2, **kw)
    assert all(lv["smoother_mapping"] == "sweep" for lv in g3.stats()["levels"][:-1])
