"""GPU parity of the smoothed transfers, per-node damping and the learned
damping network (through the C ABI) against the FP64 oracle.

Bars: bit-exact aggregates, colourings and every pattern (levels, P);
prolongator and Galerkin values within 1e-13 / 1e-12 of the oracle relative
to the largest entry; FP64 V-cycle within 1e-12; FGMRES iterations within
+-1 at 1e-8.  Network: GPU forward (FP16 parameters, FP32 arithmetic) within
2e-5 of the FP64 oracle run on the same FP16-rounded parameters; gradient
within 1e-3 (norm-wise relative) of the oracle's.  Features within 2e-6.
The damping weights of every level come from the seeded generator, sized
from an oracle hierarchy (level sizes depend on patterns only).
"""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FM6 = [0, 0, 0, 1, 1, 1]


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


def make_solver(s, **kw):
    return bamg.Solver(dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b, s.field_of_dof, **kw)


def rel_max(a, ref):
    scale = np.abs(ref).max()
    return np.abs(a - ref).max() / (scale if scale > 0 else 1.0)


def weight_arrays(s, seed, levels, lo_s=0.35, hi_s=0.65, lo_p=0.05, hi_p=0.45):
    """Seeded per-level weights sized from a (constant-weight) oracle hierarchy."""
    F = max(s.field_of_dof) + 1
    h = oracle.Hierarchy.from_system(s, max_levels=levels, max_coarse=0, smooth_p=1, omega_p=0.2)
    sizes = [h.level_sizes(l) for l in range(h.num_levels - 1)]
    ns = sum(n for n, _, _, _ in sizes) * F
    na = sum(a for _, _, _, a in sizes) * F
    ws = lo_s + (hi_s - lo_s) * P.uniform01(seed, 0, ns)
    wp = lo_p + (hi_p - lo_p) * P.uniform01(seed, ns, na)
    return ws, wp


CASES = {
    "mhd2d_16": lambda: (P.mhd2d(16, 2), 3),
    "mhd2d_cells_33": lambda: (P.mhd2d_cells(33, 4), 3),
    "random_b4_f2": lambda: (P.random_block_system(21, 4, [0, 0, 1, 1], seed=7), 3),
    "stokes2d_16": lambda: (P.stokes2d(16, 2), 3),
    "poisson_b1": lambda: (P.poisson_block(40, 1), 4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_smoothed_hierarchy_and_vcycle_match_oracle(name):
    s, levels = CASES[name]()
    ws, wp = weight_arrays(s, 100 + len(name), levels)
    kw = dict(max_levels=levels, max_coarse=0, smooth_p=1, omega_s_arr=ws, omega_p_arr=wp)
    ref = oracle.Hierarchy.from_system(s, **kw)
    sol = make_solver(s, autotune=0, **kw)
    assert sol.num_levels == ref.num_levels
    F, fb = max(s.field_of_dof) + 1, s.b // (max(s.field_of_dof) + 1)
    for l in range(ref.num_levels):
        g, o = sol.level(l), ref.level(l)
        np.testing.assert_array_equal(g["row_ptr"], o["row_ptr"])
        np.testing.assert_array_equal(g["col_idx"], o["col_idx"])
        assert rel_max(g["vals"], o["vals"]) <= 1e-12, l
        if l < ref.num_levels - 1:
            np.testing.assert_array_equal(g["agg"], o["agg"])
            np.testing.assert_array_equal(g["colour"], o["colour"])
            gp = sol.prolongator(l)
            op = ref.prolongator(l)
            np.testing.assert_array_equal(gp[0], op[0])
            np.testing.assert_array_equal(gp[1], op[1])
            assert rel_max(gp[2], op[2]) <= 1e-13, l
            gs, gpw = sol.omega(l)
            os_, opw = ref.omega(l)
            np.testing.assert_array_equal(gs, os_)
            np.testing.assert_array_equal(gpw, opw)
    r = P.uniform_pm1(7, 0, s.n_unknowns)
    z = torch.empty(s.n_unknowns, dtype=torch.float64, device="cuda")
    sol.apply(dev(r), z)
    torch.cuda.synchronize()
    assert rel_max(z.cpu().numpy(), ref.vcycle(r)) <= 1e-12
    # FGMRES to 1e-8: iteration counts within one
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = sol.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=400)
    _, it_o, rr_o, ok = ref.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=400)
    assert st == bamg.BAMG_OK and ok
    assert abs(it - it_o) <= 1, (it, it_o)
    assert rr <= 1e-8


def test_smoothed_graph_replay_equals_direct_launches():
    s = P.mhd2d(24, 5)
    ws, wp = weight_arrays(s, 5, 3)
    kw = dict(max_levels=3, max_coarse=0, smooth_p=1, omega_s_arr=ws, omega_p_arr=wp, autotune=0)
    a = make_solver(s, use_graph=1, **kw)
    b = make_solver(s, use_graph=0, **kw)
    r = dev(P.uniform_pm1(8, 0, s.n_unknowns))
    za = torch.empty_like(r)
    zb = torch.empty_like(r)
    a.apply(r, za)
    b.apply(r, zb)
    torch.cuda.synchronize()
    assert torch.equal(za, zb)


@pytest.mark.parametrize("storage", [32, 16])
def test_smoothed_fp32_cycle_and_bf16_transfers(storage):
    """FP32 V-cycle (P and R in FP32 or BF16) inside FP64 FGMRES: the cycle's
    deviation from the FP64 cycle is reported against a bound, and the final
    true FP64 residual meets the tolerance."""
    s = P.mhd2d_cells(48, 6)
    ws, wp = weight_arrays(s, 9, 3)
    kw = dict(max_levels=3, max_coarse=0, smooth_p=1, omega_s_arr=ws, omega_p_arr=wp, autotune=0)
    s64 = make_solver(s, **kw)
    s32 = make_solver(s, cycle_prec=32, pr_storage=storage, **kw)
    r = dev(P.uniform_pm1(10, 0, s.n_unknowns))
    z64 = torch.empty_like(r)
    z32 = torch.empty_like(r)
    s64.apply(r, z64)
    s32.apply(r, z32)
    torch.cuda.synchronize()
    dev_rel = float((z32 - z64).norm() / z64.norm())
    assert dev_rel <= (1e-4 if storage == 32 else 3e-2), dev_rel
    x = torch.zeros_like(r)
    st, it, rr = s32.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=600)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    A = s.to_scipy()
    xr = x.cpu().numpy()
    assert np.linalg.norm(s.rhs - A @ xr) / np.linalg.norm(s.rhs) <= 1e-8


def test_per_node_damping_set_after_setup_matches_oracle():
    s = P.mhd2d(20, 7)
    sol = make_solver(s, max_levels=3, max_coarse=0, autotune=0)
    r = dev(P.uniform_pm1(11, 0, s.n_unknowns))
    z0 = torch.empty_like(r)
    z1 = torch.empty_like(r)
    sol.apply(r, z0)
    n0 = sol.level(0)["n"]
    sol.set_omega(0, torch.full((n0 * 2,), 0.5, dtype=torch.float64, device="cuda"))
    sol.apply(r, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)  # the same damping as an array: the same arithmetic
    w0 = 0.4 + 0.3 * P.uniform01(12, 0, n0 * 2)
    sol.set_omega(0, dev(w0))
    sol.apply(r, z1)
    torch.cuda.synchronize()
    ref_h = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0)
    n1 = ref_h.level_sizes(1)[0]
    ws = np.concatenate([w0, np.full(n1 * 2, 0.5)])
    ref = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, omega_s_arr=ws)
    assert rel_max(z1.cpu().numpy(), ref.vcycle(r.cpu().numpy())) <= 1e-12


def test_select_keeps_the_hierarchy_with_fewer_iterations():
    s = P.mhd2d(24, 8)
    good = make_solver(s, max_levels=3, max_coarse=0, omega=0.55)
    bad = make_solver(s, max_levels=3, max_coarse=0, omega=0.2)
    b = dev(s.rhs)
    ch, il, ip = bamg.amg_select(bad.handle, good.handle, b, 1e-8, 30, 500)
    assert il > ip and ch == 1
    ch, il, ip = bamg.amg_select(good.handle, bad.handle, b, 1e-8, 30, 500)
    assert il < ip and ch == 0
    ch, il, ip = bamg.amg_select(good.handle, good.handle, b, 1e-8, 30, 500)
    assert il == ip and ch == 0


# ----------------------------------------------------------------------------
# features and network
# ----------------------------------------------------------------------------

def test_features_match_oracle():
    for s in (P.random_block_system(31, 6, FM6, seed=21), P.mhd2d_cells(40, 3), P.stokes2d(20, 1)):
        agg, _, nc = oracle.aggregate(s.row_ptr, s.col_idx)
        F = max(s.field_of_dof) + 1
        nf = torch.empty((s.n_nodes, F, 8), dtype=torch.float32, device="cuda")
        af = torch.empty((nc, F, 8), dtype=torch.float32, device="cuda")
        bamg.amg_features(dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.n_nodes, s.b, s.field_of_dof,
                          dev(agg), nc, 1, nf, af)
        torch.cuda.synchronize()
        onf, oaf = oracle.features(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, 1)
        np.testing.assert_allclose(nf.cpu().numpy(), onf, rtol=2e-6, atol=2e-6)
        np.testing.assert_allclose(af.cpu().numpy(), oaf, rtol=2e-6, atol=2e-6)


def random_params(seed, scale=0.4):
    p = ((P.uniform01(seed, 0, bamg.MLP_NPARAMS) - 0.5) * 2 * scale).astype(np.float32)
    p[bamg.MLP_NTRAIN:bamg.MLP_NTRAIN + 8] = (P.uniform01(seed + 1, 0, 8) - 0.5).astype(np.float32)
    p[bamg.MLP_NTRAIN + 8:] = (0.5 + P.uniform01(seed + 2, 0, 8)).astype(np.float32)
    return p


def half_rounded(p32):
    """The FP16 parameters as the oracle sees them (round to nearest even)."""
    return p32.astype(np.float16).astype(np.float64)


def test_pack_rounds_to_nearest_even():
    p = random_params(30)
    p[:6] = [1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 65504.0, -0.0, 1e-8, 7e-5]
    p16 = torch.empty(bamg.MLP_NPARAMS, dtype=torch.int16, device="cuda")
    bamg.mlp_pack(dev(p), p16)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(p16.cpu().numpy().view(np.uint16), p.astype(np.float16).view(np.uint16))


@pytest.mark.parametrize("n", [1, 127, 5000])
def test_mlp_forward_matches_oracle(n):
    p = random_params(31 + n)
    x = (P.uniform_pm1(40 + n, 0, n * 8) * 3).astype(np.float32).reshape(n, 8)
    p16 = torch.empty(bamg.MLP_NPARAMS, dtype=torch.int16, device="cuda")
    bamg.mlp_pack(dev(p), p16)
    y = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    bamg.mlp_forward(p16, dev(x), n, y)
    torch.cuda.synchronize()
    ref = oracle.mlp_forward(half_rounded(p), x.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=0, atol=2e-5 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("n", [1, 64, 1000])
def test_mlp_gradient_matches_oracle(n):
    p = random_params(50 + n)
    x = (P.uniform_pm1(60 + n, 0, n * 8) * 2).astype(np.float32).reshape(n, 8)
    t = P.uniform_pm1(70 + n, 0, n).astype(np.float32)
    head = (P.uniform01(80 + n, 0, n) < 0.5).astype(np.int32)
    p16 = torch.empty(bamg.MLP_NPARAMS, dtype=torch.int16, device="cuda")
    bamg.mlp_pack(dev(p), p16)
    g = torch.empty(bamg.MLP_NTRAIN, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    bamg.mlp_grad(p16, dev(x), dev(t), dev(head), n, g, loss)
    torch.cuda.synchronize()
    lo, go = oracle.mlp_grad(half_rounded(p), x.astype(np.float64), t.astype(np.float64), head)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - go) <= 1e-3 * np.linalg.norm(go)
    assert abs(float(loss.item()) - lo) <= 1e-4 * max(lo, 1e-6)


def test_adam_step_matches_oracle():
    p = random_params(90)
    g = P.uniform_pm1(91, 0, bamg.MLP_NTRAIN).astype(np.float32)
    m = (0.1 * P.uniform_pm1(92, 0, bamg.MLP_NTRAIN)).astype(np.float32)
    v = (0.1 * P.uniform01(93, 0, bamg.MLP_NTRAIN)).astype(np.float32)
    dp, dm, dv = dev(p), dev(m), dev(v)
    p16 = torch.empty(bamg.MLP_NPARAMS, dtype=torch.int16, device="cuda")
    bamg.mlp_adam(dp, p16, dev(g), dm, dv, 5, lr=1e-3)
    torch.cuda.synchronize()
    po, mo, vo = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    oracle.adam(po, g.astype(np.float64), mo, vo, 5, lr=1e-3)
    np.testing.assert_allclose(dp.cpu().numpy(), po, rtol=0, atol=2e-6)
    np.testing.assert_allclose(dm.cpu().numpy(), mo, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(dv.cpu().numpy(), vo, rtol=1e-6, atol=1e-7)
    np.testing.assert_array_equal(p16.cpu().numpy().view(np.uint16),
                                  dp.cpu().numpy().astype(np.float16).view(np.uint16))


def learned_params(seed, p_bias):
    """A network whose smoother head varies by node around 0.5 and whose P
    head is the constant p_bias (far from the clip thresholds)."""
    p = random_params(seed, scale=0.3)
    O_W3 = bamg.MLP_NTRAIN - 2 - 2 * 64
    p[O_W3:O_W3 + 64] *= 0.05           # head 0: small node-to-node variation around 0.5
    p[O_W3 + 64:O_W3 + 128] = 0.0       # head 1: constant
    p[bamg.MLP_NTRAIN - 2] = 0.45
    p[bamg.MLP_NTRAIN - 1] = p_bias
    return p


@pytest.mark.parametrize("p_bias,mlp_levels", [(0.15, 0), (-1.0, 0), (0.15, 1)])
def test_learned_setup_matches_oracle(p_bias, mlp_levels):
    s = P.mhd2d(32, 1)
    prm = learned_params(95, p_bias)
    sol = make_solver(s, max_levels=3, max_coarse=0, mlp=prm, mlp_levels=mlp_levels, autotune=0)
    ref = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, mlp=half_rounded(prm), mlp_levels=mlp_levels)
    assert sol.num_levels == ref.num_levels
    for l in range(ref.num_levels - 1):
        gs, gp = sol.omega(l)
        os_, op = ref.omega(l)
        np.testing.assert_allclose(gs, os_, rtol=0, atol=2e-5)
        np.testing.assert_allclose(gp, op, rtol=0, atol=2e-5)
        by_net = mlp_levels == 0 or l < mlp_levels
        assert (sol.prolongator(l) is None) == (p_bias < 0 or not by_net)
        if by_net:
            assert gs.std() > 1e-3  # the weights really vary by node
        else:
            assert (gs == 0.5).all()
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = sol.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=600)
    _, it_o, _, ok = ref.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=600)
    assert st == bamg.BAMG_OK and ok
    assert abs(it - it_o) <= 1, (it, it_o)


def test_smoothed_cycle_with_and_without_programmatic_launch():
    s = P.mhd2d_cells(40, 12)
    ws, wp = weight_arrays(s, 13, 3)
    r = dev(P.uniform_pm1(14, 0, s.n_unknowns))
    zs = []
    for pdl in (1, 0):
        sol = make_solver(s, max_levels=3, max_coarse=0, smooth_p=1, omega_s_arr=ws, omega_p_arr=wp, cycle_prec=32,
                          use_pdl=pdl, autotune=0)
        z = torch.empty_like(r)
        sol.apply(r, z)
        sol.apply(r, z)
        torch.cuda.synchronize()
        zs.append(z)
    assert torch.equal(zs[0], zs[1])
