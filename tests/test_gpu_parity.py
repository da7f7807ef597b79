"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars (stated per test): bit-exact aggregates, colourings, every level's
sparsity pattern and the Galerkin values (both sides add the same FP64
numbers in the same order); node-block inverses within 1e-12; FP64 V-cycle
output within 1e-12 of the oracle relative to its largest entry; FGMRES
iteration counts within +-1 at a relative residual of 1e-8.
"""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

VCYCLE_TOL = 1e-12  # relative to max |z| of the oracle
DINV_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bamg.load()
    torch.cuda.set_device(0)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def device_system(s):
    return dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1))


def make_solver(s, **kw):
    rp, ci, va = device_system(s)
    return bamg.Solver(rp, ci, va, s.b, s.field_of_dof, **kw)


def make_oracle(s, **kw):
    okw = {k: kw[k] for k in ("max_levels", "max_coarse", "n_pre", "n_post", "omega") if k in kw}
    return oracle.Hierarchy.from_system(s, **okw)


def rel_max(a, ref):
    scale = np.abs(ref).max()
    return np.abs(a - ref).max() / (scale if scale > 0 else 1.0)


SYSTEMS = {
    "stokes2d_32": lambda: (P.stokes2d(32, 1), dict(max_levels=3, max_coarse=0)),
    "mhd2d_16": lambda: (P.mhd2d(16, 2), dict(max_levels=3, max_coarse=0)),
    "mhd2d_41_ragged": lambda: (P.mhd2d(41, 3), dict(max_levels=4, max_coarse=0)),
    "stokes3d_9": lambda: (P.stokes3d(9, 1), dict(max_levels=3, max_coarse=0)),
    "random_b4_f2": lambda: (P.random_block_system(23, 4, [0, 0, 1, 1], seed=5), dict(max_levels=3, max_coarse=0)),
    "random_b6_f1": lambda: (P.random_block_system(19, 6, [0] * 6, seed=6), dict(max_levels=3, max_coarse=0)),
    "poisson_b1": lambda: (P.poisson_block(50, 1), dict(max_levels=4, max_coarse=0)),
    "poisson_b2": lambda: (P.poisson_block(30, 2), dict(max_levels=10, max_coarse=100)),
}


# ---------------------------------------------------------------------------
# SpMV
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 6, 7, 8])
def test_bsr_spmv_matches_oracle(b):
    s = P.random_block_system(37, b, [0] * b, seed=40 + b)  # 1369 block rows: several CTAs and a ragged tail
    rp, ci, va = device_system(s)
    x = np.random.default_rng(b).standard_normal(s.n_unknowns)
    y = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    bamg.bsr_spmv(rp, ci, va, s.n_nodes, b, dev(x), y)
    torch.cuda.synchronize()
    ref = oracle.spmv(s.row_ptr, s.col_idx, s.vals, x)
    assert rel_max(y.cpu().numpy(), ref) <= 1e-14


def test_bsr_spmv_empty_and_single_node():
    s = P.random_block_system(1, 3, [0] * 3, seed=1)
    rp, ci, va = device_system(s)
    x = dev(np.ones(3))
    y = torch.empty(3, dtype=torch.float64, device="cuda")
    bamg.bsr_spmv(rp, ci, va, 1, 3, x, y)
    torch.cuda.synchronize()
    assert np.allclose(y.cpu().numpy(), s.vals[0] @ np.ones(3), rtol=1e-15)
    bamg.bsr_spmv(rp, ci, va, 0, 3, x, y)  # zero rows: no work, no error


# ---------------------------------------------------------------------------
# hierarchy structure
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_hierarchy_matches_oracle(name):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, **kw)
    o = make_oracle(s, **kw)
    assert g.num_levels == o.num_levels
    F = max(s.field_of_dof) + 1
    for l in range(o.num_levels):
        Lg, Lo = g.level(l), o.level(l)
        assert (Lg["n"], Lg["nnzb"]) == (Lo["n"], Lo["nnzb"]), l
        assert np.array_equal(Lg["row_ptr"], Lo["row_ptr"]), l
        assert np.array_equal(Lg["col_idx"], Lo["col_idx"]), l
        # Galerkin values: the same FP64 additions in the same order
        assert np.array_equal(Lg["vals"], Lo["vals"]), (l, rel_max(Lg["vals"], Lo["vals"]))
        if l < o.num_levels - 1:
            assert Lg["n_colours"] == Lo["n_colours"] and Lg["n_agg"] == Lo["n_agg"]
            assert np.array_equal(Lg["agg"], Lo["agg"]), l
            assert np.array_equal(Lg["colour"], Lo["colour"]), l
            assert rel_max(Lg["dinv"].reshape(-1), Lo["dinv"].reshape(-1)) <= DINV_TOL
            assert Lg["dinv"].shape[1] == F


# ---------------------------------------------------------------------------
# V-cycle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mapping", [dict(tail_dofs=0, autotune=0), dict(tail_dofs=65536, autotune=0),
                                     dict(tail_dofs=0, autotune=2), dict(tail_dofs=0, autotune=3),
                                     dict(tail_dofs=0, autotune=4), dict(tail_dofs=0, autotune=6),
                                     dict(tail_dofs=0, autotune=7), dict(tail_dofs=0, autotune=8)])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_vcycle_fp64_matches_oracle(name, mapping):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, **mapping, **kw)
    o = make_oracle(s, **kw)
    r = np.random.default_rng(7).standard_normal(s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= VCYCLE_TOL


@pytest.mark.parametrize("variant", [dict(n_pre=0, n_post=2), dict(n_pre=2, n_post=0), dict(omega=0.8),
                                     dict(n_pre=2, n_post=3, omega=0.6), dict(max_levels=1)])
def test_vcycle_variants_match_oracle(variant):
    s = P.mhd2d(12, 4)
    kw = dict(max_levels=3, max_coarse=0)
    kw.update(variant)
    g = make_solver(s, **kw)
    o = make_oracle(s, **kw)
    r = s.rhs
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), o.vcycle(r)) <= VCYCLE_TOL


@pytest.mark.parametrize("grid", [0, 1])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", ["stokes2d_32", "mhd2d_41_ragged", "stokes3d_9", "poisson_b2"])
def test_cluster_tail_equals_per_kernel_cycle_bitwise(name, prec, grid):
    s, kw = SYSTEMS[name]()
    # the tail (one cluster, or every SM with grid barriers) replays the
    # warp-per-row device functions: compare with that mapping
    with_tail = make_solver(s, tail_dofs=1 << 30, tail_grid=grid, cycle_prec=prec, autotune=0, **kw)
    some_tail = make_solver(s, tail_dofs=2000, tail_grid=grid, cycle_prec=prec, autotune=0, **kw)
    no_tail = make_solver(s, tail_dofs=0, cycle_prec=prec, autotune=0, **kw)
    st = with_tail.stats()
    assert st["tail_level"] == 0 and no_tail.stats()["tail_level"] == -1
    assert (st["tail_grid"] > 0) == bool(grid) and (st["tail_cluster"] > 0) == (not grid)
    r = dev(np.random.default_rng(3).standard_normal(s.n_unknowns))
    outs = []
    for g in (with_tail, some_tail, no_tail):
        z = torch.empty_like(r)
        g.apply(r, z)
        outs.append(z)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[2]) and torch.equal(outs[1], outs[2])
    # repeated launches reuse the barrier words: the same bits again, and a solve
    z = torch.empty_like(r)
    with_tail.apply(r, z)
    torch.cuda.synchronize()
    assert torch.equal(z, outs[2])
    x = torch.zeros_like(r)
    st_, it, rr = with_tail.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=3000)
    x0 = torch.zeros_like(r)
    _, it0, _ = no_tail.solve(dev(s.rhs), x0, tol=1e-8, restart=30, max_iter=3000)
    assert st_ == bamg.BAMG_OK and rr <= 1e-8 and it == it0


@pytest.mark.parametrize("name", ["mhd2d_41_ragged", "random_b4_f2", "mhd2d_16"])
def test_field_major_values_bitwise(name):
    # FP32 values stored field-major inside each block row: the same entries
    # in the same order, so the cycle is bitwise the block-major one, for every
    # row mapping of the smoother and the residual
    s, kw = SYSTEMS[name]()
    r = dev(np.random.default_rng(11).standard_normal(s.n_unknowns))
    for at in (0, 2, 3, 4, 7, 8):
        zs = []
        for layout in (1, 2):
            g = make_solver(s, cycle_prec=32, autotune=at, value_layout=layout, **kw)
            st = g.stats()["levels"]
            assert all(lv["field_major"] == (layout == 2) for lv in st[:-1])
            z = torch.empty_like(r)
            g.apply(r, z)
            zs.append(z)
        torch.cuda.synchronize()
        assert torch.equal(zs[0], zs[1]), at
    # and through the cluster tail (recorded residual and smoother phases)
    zt = []
    for layout in (1, 2):
        g = make_solver(s, cycle_prec=32, autotune=0, value_layout=layout, tail_dofs=1 << 30, **kw)
        z = torch.empty_like(r)
        g.apply(r, z)
        zt.append(z)
    torch.cuda.synchronize()
    assert torch.equal(zt[0], zt[1])


@pytest.mark.parametrize("tuned", [(2, "thread"), (4, "thread-split")])
@pytest.mark.parametrize("prec", [64, 32])
def test_row_mappings_agree_and_solve(prec, tuned):
    # warp-per-row and thread-per-row kernels: same cycle up to summation order
    s, kw = SYSTEMS["mhd2d_41_ragged"]()
    gw = make_solver(s, autotune=0, cycle_prec=prec, **kw)
    gt = make_solver(s, autotune=tuned[0], cycle_prec=prec, **kw)
    st = gt.stats()["levels"]
    assert all(lv["smoother_mapping"] == tuned[1] for lv in st[:-1])
    r = dev(np.random.default_rng(9).standard_normal(s.n_unknowns))
    zw, zt = torch.empty_like(r), torch.empty_like(r)
    gw.apply(r, zw)
    gt.apply(r, zt)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == 64 else 1e-5
    assert float((zw - zt).abs().max() / zw.abs().max()) <= tol
    x = torch.zeros_like(r)
    status, it, rr = gt.solve(r, x, tol=1e-8, restart=10, max_iter=2000)
    assert status == bamg.BAMG_OK and rr <= 1e-8


@pytest.mark.parametrize("name", ["stokes2d_32", "stokes3d_9", "random_b4_f2", "poisson_b1", "mhd2d_41_ragged"])
@pytest.mark.parametrize("at,mapping", [(7, "block-split16"), (8, "block-split8")])
@pytest.mark.parametrize("prec", [64, 32])
def test_block_split_mappings_agree_and_solve(name, at, mapping, prec):
    # lanes taking whole blocks: the warp mapping's cycle up to the order of
    # the row sums; blocks of more than 16 field-row values (b = 6 with fields
    # of 3) keep four lanes per row
    s, kw = SYSTEMS[name]()
    gw = make_solver(s, autotune=0, cycle_prec=prec, **kw)
    gb = make_solver(s, autotune=at, cycle_prec=prec, **kw)
    fb = s.b // (max(s.field_of_dof) + 1)
    want = mapping if fb * s.b <= 16 else "thread-split"
    assert all(lv["smoother_mapping"] == want for lv in gb.stats()["levels"][:-1])
    r = dev(np.random.default_rng(19).standard_normal(s.n_unknowns))
    zw, zb = torch.empty_like(r), torch.empty_like(r)
    gw.apply(r, zw)
    gb.apply(r, zb)
    zb2 = torch.empty_like(r)
    gb.apply(r, zb2)
    torch.cuda.synchronize()
    assert torch.equal(zb, zb2)  # a fixed order of the row sums: repeatable bit for bit
    tol = 1e-12 if prec == 64 else 1e-5
    assert float((zw - zb).abs().max() / zw.abs().max()) <= tol
    x = torch.zeros_like(r)
    status, it, rr = gb.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=2000)
    assert status == bamg.BAMG_OK and rr <= 1e-8


@pytest.mark.parametrize("name", ["stokes3d_9", "mhd2d_41_ragged", "random_b6_f1"])
def test_outer_spmv_mappings_agree(name):
    # the FP64 outer SpMV of FGMRES as warp per row (autotune 0), thread per
    # row (2) and four lanes per row (4): the same iterations up to rounding
    s, kw = SYSTEMS[name]()
    its = []
    for at, want in ((0, "warp"), (2, "thread"), (4, "thread-split")):
        g = make_solver(s, autotune=at, **kw)
        assert g.stats()["outer_mapping"] == want
        x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
        status, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=2000)
        assert status == bamg.BAMG_OK and rr <= 1e-8
        res = s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, x.cpu().numpy())
        assert np.linalg.norm(res) / np.linalg.norm(s.rhs) <= 1e-8
        its.append(it)
    assert max(its) - min(its) <= 1, its


def test_vcycle_graph_and_direct_launch_agree_bitwise_and_repeat():
    s = P.mhd2d(20, 5)
    kw = dict(max_levels=3, max_coarse=0)
    g1 = make_solver(s, use_graph=1, autotune=0, **kw)
    g0 = make_solver(s, use_graph=0, autotune=0, **kw)
    r = dev(s.rhs)
    z1 = torch.empty_like(r)
    z2 = torch.empty_like(r)
    z0 = torch.empty_like(r)
    g1.apply(r, z1)
    g1.apply(r, z2)
    g0.apply(r, z0)
    torch.cuda.synchronize()
    assert torch.equal(z1, z2) and torch.equal(z1, z0)


# ---------------------------------------------------------------------------
# FGMRES
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ortho", [0, 1])  # second projection where the DGKS test asks / at every step
@pytest.mark.parametrize("name,restart", [("stokes2d_32", 30), ("mhd2d_16", 30), ("mhd2d_41_ragged", 10),
                                          ("random_b4_f2", 5), ("stokes3d_9", 50)])
def test_fgmres_iterations_match_oracle(name, restart, ortho):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, ortho=ortho, **kw)
    o = make_oracle(s, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=restart, max_iter=3000)
    _, it_ref, rr_ref, conv = o.fgmres(s.rhs, tol=1e-8, restart=restart, max_iter=3000)
    assert conv and st == bamg.BAMG_OK
    assert abs(it - it_ref) <= 1, (it, it_ref)
    xs = x.cpu().numpy()
    true_rel = np.linalg.norm(s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, xs)) / np.linalg.norm(s.rhs)
    assert true_rel <= 1e-8 and rr <= 1e-8


def test_fgmres_not_converged_and_zero_rhs():
    s, kw = SYSTEMS["mhd2d_16"]()
    g = make_solver(s, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=3)
    assert st == bamg.BAMG_NOT_CONVERGED and it == 3 and rr > 1e-8
    zero = torch.zeros_like(x)
    x.fill_(1.0)
    st, it, rr = g.solve(zero, x)
    assert st == bamg.BAMG_OK and it == 0 and float(x.abs().max()) == 0.0


def test_fp32_cycle_reaches_fp64_residual():
    s, kw = SYSTEMS["mhd2d_41_ragged"]()
    g64 = make_solver(s, **kw)
    g32 = make_solver(s, cycle_prec=32, **kw)
    r = dev(s.rhs)
    z64 = torch.empty_like(r)
    z32 = torch.empty_like(r)
    g64.apply(r, z64)
    g32.apply(r, z32)
    torch.cuda.synchronize()
    err = float((z32 - z64).norm() / z64.norm())
    assert err < 1e-4, err
    x = torch.zeros_like(r)
    st, it, rr = g32.solve(r, x, tol=1e-8, restart=30, max_iter=3000)
    xs = x.cpu().numpy()
    true_rel = np.linalg.norm(s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, xs)) / np.linalg.norm(s.rhs)
    assert st == bamg.BAMG_OK and true_rel <= 1e-8


def test_host_entry_point_matches_device_path():
    s, kw = SYSTEMS["mhd2d_16"]()
    kw = dict(kw, autotune=0)  # both paths with the same row mapping: bitwise equal results
    g = make_solver(s, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x)
    xh = np.zeros(s.n_unknowns)
    p = bamg.amg_default_params(**kw)
    st2, it2, rr2 = bamg.amg_solve_host(s.row_ptr, s.col_idx, np.ascontiguousarray(s.vals.reshape(-1)),
                                        s.n_nodes, s.nnzb, s.b, s.field_of_dof, s.rhs, xh, params=p)
    assert st == st2 == 0 and it == it2
    assert np.array_equal(xh, x.cpu().numpy())


# ---------------------------------------------------------------------------
# errors reported as statuses (the device is never trapped)
# ---------------------------------------------------------------------------
def expect_status(status, fn):
    with pytest.raises(bamg.BamgError) as e:
        fn()
    assert e.value.status == status


def test_invalid_inputs_are_rejected():
    s = P.mhd2d(6, 1)
    rp, ci, va = device_system(s)
    kw = dict(max_levels=2, max_coarse=0)
    # bad field maps (fields of unequal size are valid: tests/test_gpu_unequal.py)
    expect_status(bamg.BAMG_EINVAL, lambda: bamg.Solver(rp, ci, va, 6, [0, 0, 2, 2, 2, 2], **kw))
    expect_status(bamg.BAMG_EINVAL, lambda: bamg.Solver(rp, ci, va, 6, [1, 1, 1, 0, 0, 0], **kw))
    # unsupported block shape for the smoother (three fields of one dof)
    s3 = P.random_block_system(5, 3, [0, 1, 2], seed=1)
    expect_status(bamg.BAMG_EUNSUPPORTED, lambda: make_solver(s3, **kw))
    # unsorted columns in one row
    ci_bad = s.col_idx.copy()
    k0 = s.row_ptr[7]
    ci_bad[k0], ci_bad[k0 + 1] = ci_bad[k0 + 1], ci_bad[k0]
    expect_status(bamg.BAMG_EINVAL, lambda: bamg.Solver(rp, dev(ci_bad), va, 6, s.field_of_dof, **kw))
    # a block stored on one side only (row 20 lists node 3 and node 45, and
    # neither lists 20 back): the pattern is not structurally symmetric
    for j in (3, 45):
        row = s.col_idx[s.row_ptr[20]:s.row_ptr[21]]
        pos = s.row_ptr[20] + int(np.searchsorted(row, j))
        ci_1 = np.insert(s.col_idx, pos, j).astype(np.int32)
        va_1 = np.insert(s.vals, pos, 0.0, axis=0)
        rp_1 = s.row_ptr.copy()
        rp_1[21:] += 1
        expect_status(bamg.BAMG_EINVAL, lambda: bamg.Solver(dev(rp_1), dev(ci_1), dev(va_1.reshape(-1)), 6,
                                                            s.field_of_dof, **kw))
    # singular node block of one field
    v_bad = s.vals.copy()
    diag = [k for k in range(s.row_ptr[9], s.row_ptr[10]) if s.col_idx[k] == 9][0]
    v_bad[diag, 3:, 3:] = 0.0
    expect_status(bamg.BAMG_ESINGULAR_BLOCK,
                  lambda: bamg.Solver(rp, ci, dev(v_bad.reshape(-1)), 6, s.field_of_dof, **kw))


def test_nonfinite_rhs_reported():
    s = P.mhd2d(6, 1)
    g = make_solver(s, max_levels=2, max_coarse=0)
    rhs = s.rhs.copy()
    rhs[5] = np.nan
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    expect_status(bamg.BAMG_ENAN, lambda: g.solve(dev(rhs), x))


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("at", [0, 6, 7])
def test_programmatic_dependent_launch_gives_identical_cycles(prec, at):
    """The V-cycle with programmatic dependent launches (default) and with
    ordinary launches: identical bits, replayed from the graph and direct."""
    s = P.mhd2d(41, 3)
    r = dev(P.uniform_pm1(5, 0, s.n_unknowns))
    outs = []
    for pdl in (1, 0):
        for graph in (1, 0):
            sol = make_solver(s, max_levels=4, max_coarse=0, cycle_prec=prec, use_pdl=pdl, use_graph=graph,
                              autotune=at)
            z = torch.empty_like(r)
            for _ in range(3):  # repeated cycles reuse every buffer
                sol.apply(r, z)
            torch.cuda.synchronize()
            outs.append(z.clone())
    for z in outs[1:]:
        assert torch.equal(z, outs[0])


@pytest.mark.parametrize("s_fn,levels", [(lambda: P.mhd2d(40, 4), 2), (lambda: P.stokes2d(40, 3), 2),
                                         (lambda: P.random_block_system(24, 4, [0, 0, 1, 1], seed=9), 2)])
def test_large_coarsest_factorisation(s_fn, levels):
    """Coarsest operators above the shared-memory LU size (the cooperative
    factorisation): V-cycle and FGMRES against the oracle's dense LU."""
    s = s_fn()
    kw = dict(max_levels=levels, max_coarse=0)
    ref = make_oracle(s, **kw)
    sol = make_solver(s, **kw)
    nc = sol.level(sol.num_levels - 1)["n"] * s.b
    assert 158 < nc <= 4096, nc
    r = P.uniform_pm1(15, 0, s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    sol.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), ref.vcycle(r)) <= 1e-12
    x = torch.zeros_like(z)
    st, it, rr = sol.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=500)
    _, it_o, _, ok = ref.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=500)
    assert st == 0 and ok and abs(it - it_o) <= 1


@pytest.mark.parametrize("n_side,seed", [(220, 1), (300, 2)])
def test_colouring_frontiers_on_permuted_graph(n_side, seed):
    """Graphs above the one-CTA worklist size are coloured by frontier rounds;
    on a randomly renumbered stencil graph (irregular lower/higher neighbour
    structure) the colours must equal the oracle's sequential first fit."""
    s = P.random_block_system(n_side, 1, [0], seed)
    n = s.n_nodes
    assert n > 40000
    perm = np.random.default_rng(seed).permutation(n)  # new index of old node i
    inv = np.argsort(perm)
    rows = []
    for new in range(n):
        old = inv[new]
        k0, k1 = s.row_ptr[old], s.row_ptr[old + 1]
        cols = perm[s.col_idx[k0:k1]]
        order = np.argsort(cols)
        rows.append((cols[order], s.vals[k0:k1][order]))
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(c) for c, _ in rows])
    ci = np.concatenate([c for c, _ in rows]).astype(np.int32)
    va = np.concatenate([v for _, v in rows])
    g = bamg.Solver(dev(rp), dev(ci), dev(np.ascontiguousarray(va).reshape(-1)), 1, [0], max_levels=3, max_coarse=0)
    want, _ = oracle.colour(rp, ci)
    assert np.array_equal(g.level(0)["colour"], want)
