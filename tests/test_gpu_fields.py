"""GPU parity of fields on disjoint node sets (separate aggregation per field
block, Sec. 4.3.1; the mixed Q2/Q1 example of Sec. 5) through the C ABI
(amg_setup_fields) against the FP64 oracle.

Bars, as for co-located fields: aggregates, colourings, field ranges and
every level's pattern and Galerkin values bit for bit; FP64 V-cycle within
1e-12 of the oracle relative to its largest entry; FGMRES iterations within
+-1 at a relative residual of 1e-8.
"""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P
from test_oracle_fields import two_field_system

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

VCYCLE_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bamg.load()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_max(a, ref):
    scale = np.abs(ref).max()
    return np.abs(a - ref).max() / (scale if scale > 0 else 1.0)


def three_field_system(sizes, b, seed):
    """Random two-field system split further: field ranges of ``sizes``."""
    rp, ci, vals, _ = two_field_system(sizes[0] + sizes[1], sizes[2], b, seed, 0.06, 0.04)
    off = np.concatenate([[0], np.cumsum(sizes)]).tolist()
    return rp, ci, vals, off


def q2q1(N, seed):
    s = P.mhd2d_q2q1(N, seed)
    return s.row_ptr, s.col_idx, s.vals, s.node_field_off


SYSTEMS = {
    "q2q1_12": lambda: (q2q1(12, 1), dict(max_levels=3, max_coarse=0)),
    "q2q1_21_ragged": lambda: (q2q1(21, 2), dict(max_levels=4, max_coarse=0)),
    "two_field_b2": lambda: (two_field_system(70, 45, 2, 3, 0.06, 0.03), dict(max_levels=3, max_coarse=0)),
    # ragged ranges, one field of three nodes
    "three_field_b4": lambda: (three_field_system([60, 41, 3], 4, 8), dict(max_levels=3, max_coarse=0)),
}


def rhs_of(vals, n, seed=7):
    return np.random.default_rng(seed).standard_normal(n * vals.shape[1])


def make(sysdef, **kw):
    (rp, ci, vals, off), base = sysdef
    okw = {k: v for k, v in dict(base, **kw).items() if k in ("max_levels", "max_coarse", "n_pre", "n_post", "omega")}
    g = bamg.FieldSolver(off, dev(rp), dev(ci), dev(vals.reshape(-1)), vals.shape[1], **dict(base, **kw))
    o = oracle.Hierarchy(rp, ci, vals, vals.shape[1], [0] * vals.shape[1], node_field_off=off, **okw)
    return g, o, (rp, ci, vals, off)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_field_hierarchy_matches_oracle(name):
    g, o, _ = make(SYSTEMS[name]())
    assert g.num_levels == o.num_levels
    for l in range(o.num_levels):
        Lg, Lo = g.level(l), o.level(l)
        assert (Lg["n"], Lg["nnzb"]) == (Lo["n"], Lo["nnzb"]), l
        assert np.array_equal(Lg["row_ptr"], Lo["row_ptr"]), l
        assert np.array_equal(Lg["col_idx"], Lo["col_idx"]), l
        assert np.array_equal(Lg["vals"], Lo["vals"]), (l, rel_max(Lg["vals"], Lo["vals"]))
        no_g, co_g = g.fields(l)
        no_o, co_o = o.fields(l)
        assert np.array_equal(no_g, no_o), l
        if l < o.num_levels - 1:
            assert Lg["n_colours"] == Lo["n_colours"] and Lg["n_agg"] == Lo["n_agg"]
            assert np.array_equal(Lg["agg"], Lo["agg"]), l
            assert np.array_equal(Lg["colour"], Lo["colour"]), l
            assert np.array_equal(co_g, co_o), l
            assert rel_max(Lg["dinv"].reshape(-1), Lo["dinv"].reshape(-1)) <= 1e-12
    st = g.stats()
    assert st["node_fields"] == len(SYSTEMS[name]()[0][3]) - 1
    assert st["levels"][0]["field_nodes"] == np.diff(SYSTEMS[name]()[0][3]).tolist()


@pytest.mark.parametrize("mapping", [dict(autotune=0), dict(autotune=2), dict(autotune=3), dict(autotune=4),
                                     dict(autotune=6), dict(autotune=7), dict(autotune=8)])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_field_vcycle_fp64_matches_oracle(name, mapping):
    g, o, (rp, ci, vals, off) = make(SYSTEMS[name](), **mapping)
    r = rhs_of(vals, len(rp) - 1)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= VCYCLE_TOL


@pytest.mark.parametrize("variant", [dict(n_pre=0, n_post=2), dict(n_pre=2, n_post=0), dict(omega=0.8),
                                     dict(n_pre=2, n_post=3, omega=0.6), dict(max_levels=1),
                                     dict(use_graph=0)])
def test_field_vcycle_variants_match_oracle(variant):
    g, o, (rp, ci, vals, off) = make(SYSTEMS["q2q1_12"](), **variant)
    r = rhs_of(vals, len(rp) - 1, 3)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    z2 = torch.empty_like(z)
    g.apply(dev(r), z2)
    torch.cuda.synchronize()
    assert torch.equal(z, z2)
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= VCYCLE_TOL


def test_one_field_equals_colocated_setup():
    s = P.mhd2d_q2q1(10, 3)
    kw = dict(max_levels=3, max_coarse=0, autotune=0)
    gf = bamg.FieldSolver([0, s.n_nodes], dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), 3, **kw)
    gc = bamg.Solver(dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), 3, [0, 0, 0], **kw)
    r = dev(s.rhs)
    zf = torch.empty_like(r)
    zc = torch.empty_like(r)
    gf.apply(r, zf)
    gc.apply(r, zc)
    torch.cuda.synchronize()
    assert torch.equal(zf, zc)
    assert gc.stats()["node_fields"] == 1


@pytest.mark.parametrize("N,restart", [(16, 30), (32, 30), (21, 10)])
def test_field_fgmres_iterations_match_oracle(N, restart):
    s = P.mhd2d_q2q1(N, 1)
    kw = dict(max_levels=4, max_coarse=0, omega=0.6)
    g = bamg.FieldSolver(s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), 3, **kw)
    o = oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, 3, [0, 0, 0], node_field_off=s.node_field_off, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=restart, max_iter=3000)
    _, it_ref, _, conv = o.fgmres(s.rhs, tol=1e-8, restart=restart, max_iter=3000)
    assert conv and st == bamg.BAMG_OK
    assert abs(it - it_ref) <= 1, (it, it_ref)
    xs = x.cpu().numpy()
    true_rel = np.linalg.norm(s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, xs)) / np.linalg.norm(s.rhs)
    assert true_rel <= 1e-8 and rr <= 1e-8


def test_field_fp32_cycle_solves():
    s = P.mhd2d_q2q1(32, 2)
    kw = dict(max_levels=4, max_coarse=0, omega=0.6)
    g64 = bamg.FieldSolver(s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), 3, **kw)
    g32 = bamg.FieldSolver(s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), 3,
                           cycle_prec=32, coarse_prec=32, **kw)
    r = dev(s.rhs)
    z64 = torch.empty_like(r)
    z32 = torch.empty_like(r)
    g64.apply(r, z64)
    g32.apply(r, z32)
    torch.cuda.synchronize()
    assert float((z32 - z64).norm() / z64.norm()) < 1e-4
    its = {}
    for p, g in ((64, g64), (32, g32)):
        x = torch.zeros_like(r)
        st, it, rr = g.solve(r, x, tol=1e-8, restart=30, max_iter=3000)
        xs = x.cpu().numpy()
        true_rel = np.linalg.norm(s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, xs)) / np.linalg.norm(s.rhs)
        assert st == bamg.BAMG_OK and true_rel <= 1e-8
        its[p] = it
    assert abs(its[32] - its[64]) <= max(2, its[64] // 20), its


def test_field_vcycle_full_size_q2q1_64():
    # the Q2/Q1 system of 64 x 64 cells (20,866 nodes, 62,598 unknowns), four levels
    s = P.mhd2d_q2q1(64, 1)
    kw = dict(max_levels=4, max_coarse=0, omega=0.6)
    g = bamg.FieldSolver(s.node_field_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), 3, **kw)
    o = oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, 3, [0, 0, 0], node_field_off=s.node_field_off, **kw)
    for l in range(o.num_levels):
        assert np.array_equal(g.fields(l)[0], o.fields(l)[0])
    r = dev(s.rhs)
    z = torch.empty_like(r)
    g.apply(r, z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(s.rhs)) <= VCYCLE_TOL


def test_field_invalid_inputs_are_rejected():
    s = P.mhd2d_q2q1(4, 1)
    args = (dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), 3)
    n = s.n_nodes
    for off, kw in (([0, 0, n], {}), ([0, 10, n - 1], {}), ([0, 30, 20, n], {}), ([0, 81, n], dict(smooth_p=1))):
        with pytest.raises(bamg.BamgError) as e:
            bamg.FieldSolver(off, *args, max_levels=2, max_coarse=0, **kw)
        assert e.value.status == bamg.BAMG_EINVAL


@pytest.mark.parametrize("at", [0, 6])
@pytest.mark.parametrize("sub", [0, 1, 2])
@pytest.mark.parametrize("prec", [64, 32])
def test_programmatic_launches_give_identical_node_field_cycles(prec, sub, at):
    # the other fields' nodes are copied by a kernel of the cycle, so the
    # cycle runs with programmatic dependent launches: same bits as without
    # (the row mapping fixed: warp per node, or four warps per node; the
    # autotuner could pick mappings with another summation order for the two)
    (rp, ci, vals, off), kw = SYSTEMS["q2q1_21_ragged"]()
    kw = dict(kw, autotune=at)
    args = (off, dev(rp), dev(ci), dev(vals.reshape(-1)), vals.shape[1])
    zs = []
    n, b = len(rp) - 1, vals.shape[1]
    r = dev(np.random.default_rng(17).standard_normal(n * b))
    for pdl in (0, 1):
        g = bamg.FieldSolver(*args, use_pdl=pdl, cycle_prec=prec, sub_solver=sub, **kw)
        z = torch.empty_like(r)
        g.apply(r, z)
        g.apply(r, z)
        zs.append(z)
    torch.cuda.synchronize()
    assert torch.equal(zs[0], zs[1])


def test_fields_host_entry_point_matches_device_path():
    (rp, ci, vals, off), kw = SYSTEMS["q2q1_12"]()
    kw = dict(kw, autotune=0)
    n, b = len(rp) - 1, vals.shape[1]
    rhs = np.random.default_rng(23).standard_normal(n * b)
    g = bamg.FieldSolver(off, dev(rp), dev(ci), dev(vals.reshape(-1)), b, **kw)
    x = torch.zeros(n * b, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(rhs), x, tol=1e-8, restart=30, max_iter=3000)
    xh = np.zeros(n * b)
    sth, ith, rrh = bamg.amg_solve_fields_host(off, np.ascontiguousarray(rp), np.ascontiguousarray(ci),
                                               np.ascontiguousarray(vals.reshape(-1)), n, len(ci), b, rhs, xh, 1e-8,
                                               30, 3000, bamg.amg_default_params(**kw))
    assert st == sth == bamg.BAMG_OK and it == ith and rr == rrh
    assert np.array_equal(x.cpu().numpy(), xh)
