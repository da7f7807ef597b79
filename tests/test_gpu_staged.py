"""The colour step with every node's row staged in shared memory by bulk
copies (autotune = 5) against the four-lanes-per-row kernel whose lanes and
sums it repeats (autotune = 4): the same V-cycle bit for bit in FP64 and FP32,
over repeated cycles, with one field, with the field-major layout of several
fields, and on the 3D system with its 27-block rows; the FP64 cycle within
1e-12 of the oracle; where the layout would stage blocks the step does not
read (several fields, block-major values) the mapping falls back to the
four-lanes kernel."""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "stokes2d_32": lambda: (P.stokes2d(32, 1), dict(max_levels=3, max_coarse=0)),
    "stokes3d_9": lambda: (P.stokes3d(9, 1), dict(max_levels=3, max_coarse=0)),
    "stokes3d_24": lambda: (P.stokes3d(24, 2), dict(max_levels=3, max_coarse=0)),
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


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_staged_equals_four_lanes_bitwise(name, prec):
    s, kw = SYSTEMS[name]()
    ref = make_solver(s, autotune=4, cycle_prec=prec, **kw)
    stg = make_solver(s, autotune=5, cycle_prec=prec, **kw)
    assert all(lv["smoother_mapping"] == "staged" for lv in stg.stats()["levels"][:-1])
    r = dev(np.random.default_rng(31).standard_normal(s.n_unknowns))
    z0, z1 = torch.empty_like(r), torch.empty_like(r)
    ref.apply(r, z0)
    for _ in range(3):
        stg.apply(r, z1)
        torch.cuda.synchronize()
        assert torch.equal(z0, z1)


@pytest.mark.parametrize("name", ["mhd2d_41", "random_b4_f2"])
def test_staged_with_field_major_values_bitwise(name):
    s = P.mhd2d(41, 3) if name == "mhd2d_41" else P.random_block_system(23, 4, [0, 0, 1, 1], seed=5)
    kw = dict(max_levels=3, max_coarse=0, cycle_prec=32, value_layout=2)
    ref = make_solver(s, autotune=4, **kw)
    stg = make_solver(s, autotune=5, **kw)
    assert all(lv["smoother_mapping"] == "staged" for lv in stg.stats()["levels"][:-1])
    r = dev(np.random.default_rng(32).standard_normal(s.n_unknowns))
    z0, z1 = torch.empty_like(r), torch.empty_like(r)
    ref.apply(r, z0)
    stg.apply(r, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)


def test_staged_falls_back_where_it_would_read_unused_blocks():
    s = P.mhd2d(16, 2)  # two fields, block-major values
    g = make_solver(s, autotune=5, cycle_prec=64, max_levels=3, max_coarse=0)
    assert all(lv["smoother_mapping"] == "thread-split" for lv in g.stats()["levels"][:-1])


@pytest.mark.parametrize("name", ["stokes2d_32", "stokes3d_9", "poisson_b2"])
def test_staged_vcycle_fp64_matches_oracle(name):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, autotune=5, **kw)
    o = oracle.Hierarchy.from_system(s, **kw)
    r = np.random.default_rng(7).standard_normal(s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    ref = o.vcycle(r)
    assert np.abs(z.cpu().numpy() - ref).max() / np.abs(ref).max() <= 1e-12


def test_staged_fp32_3d_solve_reaches_fp64_residual():
    s = P.stokes3d(24, 2)
    g = make_solver(s, max_levels=10, max_coarse=2500, cycle_prec=32, coarse_prec=32, autotune=5)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=50, max_iter=3000)
    assert st == bamg.BAMG_OK and rr <= 1e-8
