"""Block shapes beyond the configured workloads: 5 x 5, 7 x 7 and 8 x 8 node
blocks of one field, 8 dofs in two fields of 4 and in four fields of 2, and 6
dofs in three fields of 2.  For each: the hierarchy bit for bit against the
oracle, the FP64 V-cycle within 1e-12 of the oracle under every smoother row
mapping, FGMRES iteration counts within +-1 at 1e-8, and the FP32 cycle
reaching the FP64 residual 1e-8.  The inputs are seeded random stencil
systems with a strengthened diagonal (problems.random_block_system)."""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SHAPES = {
    "b5_f1": (5, [0] * 5),
    "b7_f1": (7, [0] * 7),
    "b8_f1": (8, [0] * 8),
    "b8_f2": (8, [0] * 4 + [1] * 4),
    "b8_f4": (8, [0, 0, 1, 1, 2, 2, 3, 3]),
    "b6_f3": (6, [0, 0, 1, 1, 2, 2]),
}
KW = dict(max_levels=3, max_coarse=0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bamg.load()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def system(name):
    b, fm = SHAPES[name]
    return P.random_block_system(21, b, fm, seed=40 + b + len(set(fm)))  # 441 nodes: several CTAs, ragged tail


def make_solver(s, **kw):
    return bamg.Solver(dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b, s.field_of_dof, **kw)


def rel_max(a, ref):
    scale = np.abs(ref).max()
    return np.abs(a - ref).max() / (scale if scale > 0 else 1.0)


@pytest.mark.parametrize("name", list(SHAPES))
def test_shape_hierarchy_matches_oracle(name):
    s = system(name)
    g = make_solver(s, **KW)
    o = oracle.Hierarchy.from_system(s, **KW)
    assert g.num_levels == o.num_levels
    for l in range(o.num_levels):
        Lg, Lo = g.level(l), o.level(l)
        assert np.array_equal(Lg["row_ptr"], Lo["row_ptr"]) and np.array_equal(Lg["col_idx"], Lo["col_idx"])
        assert np.array_equal(Lg["vals"], Lo["vals"]), l
        if l < o.num_levels - 1:
            assert np.array_equal(Lg["agg"], Lo["agg"]) and np.array_equal(Lg["colour"], Lo["colour"])
            assert rel_max(Lg["dinv"].reshape(-1), Lo["dinv"].reshape(-1)) <= 1e-12


@pytest.mark.parametrize("mapping", [dict(autotune=0), dict(autotune=2), dict(autotune=4), dict(autotune=5),
                                     dict(autotune=7), dict(autotune=8),
                                     dict(autotune=0, sweep=2), dict(autotune=0, tail_dofs=1 << 30)])
@pytest.mark.parametrize("name", list(SHAPES))
def test_shape_vcycle_fp64_matches_oracle(name, mapping):
    s = system(name)
    g = make_solver(s, **mapping, **KW)
    o = oracle.Hierarchy.from_system(s, **KW)
    r = np.random.default_rng(5).standard_normal(s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("sub", [1, 2])
@pytest.mark.parametrize("name", ["b5_f1", "b8_f2", "b6_f3"])
def test_shape_sub_solvers_match_oracle(name, sub):
    s = system(name)
    g = make_solver(s, sub_solver=sub, **KW)
    o = oracle.Hierarchy.from_system(s, sub_ilu=2 if sub == 1 else 0, sub_schwarz=2 if sub == 2 else 0, **KW)
    r = np.random.default_rng(6).standard_normal(s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("name", list(SHAPES))
def test_shape_fgmres_iterations_and_fp32_cycle(name):
    s = system(name)
    o = oracle.Hierarchy.from_system(s, **KW)
    _, it_o, _, _ = o.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=2000)
    for prec in (64, 32):
        g = make_solver(s, cycle_prec=prec, **KW)
        x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
        st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=2000)
        assert st == bamg.BAMG_OK and rr <= 1e-8, (prec, st, rr)
        if prec == 64:
            assert abs(it - it_o) <= 1, (it, it_o)
