"""Pins of the oracle's smoothed transfers, per-node damping and learned
damping network against facts that do not come from the oracle: dense
linear algebra, invariances of the definitions, closed forms of special
cases and central finite differences.  CPU only.

Definitions (beyond the paper, whose prolongator is the tentative one and
whose damping is one constant near 0.5, Sec. 4.3.2 and Sec. 5):
  P_f = (I - W_f D_ff^{-1} A_ff) P^_f per field, A_c = P^T A P (Sec. 3),
  x_f += omega_{i,f} x~_f per node (Algorithm 1 with per-node damping),
  features / MLP / mean squared error / Adam as documented in the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import problems as P

FM6 = [0, 0, 0, 1, 1, 1]


def tentative_dense(agg, nc, b):
    n = len(agg)
    Pm = np.zeros((n * b, nc * b))
    for i in range(n):
        for d in range(b):
            Pm[i * b + d, agg[i] * b + d] = 1.0
    return Pm


def p_dense(p_rp, p_ci, p_v, n, nc, b, F):
    """Dense matrix of a field-block-diagonal P (F sub-blocks per stored block)."""
    fb = b // F
    Pm = np.zeros((n * b, nc * b))
    for i in range(n):
        for q in range(p_rp[i], p_rp[i + 1]):
            J = p_ci[q]
            for f in range(F):
                Pm[i * b + f * fb:i * b + (f + 1) * fb, J * b + f * fb:J * b + (f + 1) * fb] = p_v[q, f]
    return Pm


def bsr_dense(rp, ci, v, n, b):
    A = np.zeros((n * b, n * b))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i * b:(i + 1) * b, ci[k] * b:(ci[k] + 1) * b] = v[k]
    return A


def rand_system(n_side=5, b=6, fm=FM6, seed=3):
    return P.random_block_system(n_side, b, fm, seed)


def aggregates(s):
    agg, _, nc = oracle.aggregate(s.row_ptr, s.col_idx)
    return agg, nc


# ----------------------------------------------------------------------------
# smoothed prolongator
# ----------------------------------------------------------------------------

def test_prolongator_zero_weight_is_tentative():
    s = rand_system()
    agg, nc = aggregates(s)
    prp, pci, pv = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, 0.0)
    # pattern: the distinct aggregates of the stored neighbours, ascending (brute force)
    for i in range(s.n_nodes):
        want = sorted({int(agg[j]) for j in s.col_idx[s.row_ptr[i]:s.row_ptr[i + 1]]})
        assert list(pci[prp[i]:prp[i + 1]]) == want
    Pm = p_dense(prp, pci, pv, s.n_nodes, nc, s.b, 2)
    np.testing.assert_array_equal(Pm, tentative_dense(agg, nc, s.b))


def test_prolongator_affine_in_the_weight_of_its_aggregate():
    s = rand_system(seed=4)
    agg, nc = aggregates(s)
    w = P.uniform01(11, 0, nc * 2).reshape(nc, 2) * 1.3
    _, _, p0 = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, 0.0)
    _, _, p1 = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, 1.0)
    prp, _, pw = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, w)
    for i in range(s.n_nodes):
        for q in range(prp[i], prp[i + 1]):
            for f in range(2):
                want = p0[q, f] + w[agg[i], f] * (p1[q, f] - p0[q, f])
                np.testing.assert_allclose(pw[q, f], want, rtol=0, atol=1e-13)


def test_prolongator_invariant_under_node_row_scaling():
    """D_ff^{-1} A_ff does not change when the field-f rows of node i are
    multiplied by any nonsingular M: catches D for D^{-1}, transposes, and
    blocks taken from the wrong field."""
    s = rand_system(seed=5)
    agg, nc = aggregates(s)
    w = 0.2 + P.uniform01(12, 0, nc * 2).reshape(nc, 2)
    ref = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, w)[2]
    v2 = s.vals.copy()
    rng = np.random.default_rng(7)
    for i in range(s.n_nodes):
        for f in range(2):
            M = rng.standard_normal((3, 3)) + 3 * np.eye(3)
            for k in range(s.row_ptr[i], s.row_ptr[i + 1]):
                v2[k, 3 * f:3 * f + 3, :] = M @ v2[k, 3 * f:3 * f + 3, :]
    got = oracle.prolongator(s.row_ptr, s.col_idx, v2, s.field_of_dof, agg, nc, w)[2]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_prolongator_ignores_cross_field_blocks():
    s = rand_system(seed=6)
    agg, nc = aggregates(s)
    ref = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, 0.7)[2]
    v2 = s.vals.copy()
    v2[:, 0:3, 3:6] *= -5.0
    v2[:, 3:6, 0:3] += 1.0
    got = oracle.prolongator(s.row_ptr, s.col_idx, v2, s.field_of_dof, agg, nc, 0.7)[2]
    np.testing.assert_array_equal(got, ref)


def test_prolongator_keeps_constants_where_rows_sum_to_zero():
    """Laplacian rows with all neighbours interior sum to zero, so the
    smoothed P still interpolates constants exactly there, for any weights."""
    s = P.poisson_block(8, 3)
    agg, nc = aggregates(s)
    w = 0.3 + P.uniform01(13, 0, nc).reshape(nc, 1)
    prp, pci, pv = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, w)
    Pm = p_dense(prp, pci, pv, s.n_nodes, nc, 3, 1)
    ones = Pm @ np.ones(nc * 3)
    A = s.dense()
    row_sums = A @ np.ones(s.n_nodes * 3)
    interior = np.abs(row_sums.reshape(-1, 3)).max(1) < 1e-12
    assert interior.sum() > 10
    np.testing.assert_allclose(ones.reshape(-1, 3)[interior], 1.0, atol=1e-13)
    # and where they do not, P 1 moves away from 1 (the check is not vacuous)
    assert np.abs(ones.reshape(-1, 3)[~interior] - 1.0).max() > 1e-3


# ----------------------------------------------------------------------------
# general Galerkin product
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("b,fm", [(6, FM6), (4, [0, 0, 1, 1]), (3, [0, 0, 0]), (1, [0])])
def test_rap_general_is_the_dense_galerkin_product(b, fm):
    s = rand_system(n_side=5, b=b, fm=fm, seed=8 + b)
    F = max(fm) + 1
    agg, nc = aggregates(s)
    w = P.uniform01(14, 0, nc * F).reshape(nc, F)
    prp, pci, pv = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, fm, agg, nc, w)
    rpc, cic, vc = oracle.rap_general(s.row_ptr, s.col_idx, s.vals, fm, nc, prp, pci, pv)
    Pm = p_dense(prp, pci, pv, s.n_nodes, nc, b, F)
    Ac = Pm.T @ s.dense() @ Pm
    got = bsr_dense(rpc, cic, vc, nc, b)
    np.testing.assert_allclose(got, Ac, rtol=0, atol=1e-12 * np.abs(Ac).max())
    # pattern = structural union of pattern(P)^T pattern(A) pattern(P), ascending
    SA = np.zeros((s.n_nodes, s.n_nodes), bool)
    for i in range(s.n_nodes):
        SA[i, s.col_idx[s.row_ptr[i]:s.row_ptr[i + 1]]] = True
    SP = np.zeros((s.n_nodes, nc), bool)
    for i in range(s.n_nodes):
        SP[i, pci[prp[i]:prp[i + 1]]] = True
    S = (SP.T.astype(int) @ SA.astype(int) @ SP.astype(int)) > 0
    for I in range(nc):
        assert list(cic[rpc[I]:rpc[I + 1]]) == list(np.nonzero(S[I])[0])


def test_rap_general_at_zero_weight_equals_tentative_values():
    s = rand_system(seed=9)
    agg, nc = aggregates(s)
    prp, pci, pv = oracle.prolongator(s.row_ptr, s.col_idx, s.vals, FM6, agg, nc, 0.0)
    rpc, cic, vc = oracle.rap_general(s.row_ptr, s.col_idx, s.vals, FM6, nc, prp, pci, pv)
    trp, tci, tv = oracle.rap_tentative(s.row_ptr, s.col_idx, s.vals, 6, agg, nc)
    np.testing.assert_allclose(bsr_dense(rpc, cic, vc, nc, 6), bsr_dense(trp, tci, tv, nc, 6), rtol=0,
                               atol=1e-12)


# ----------------------------------------------------------------------------
# hierarchy with smoothed transfers and per-node damping
# ----------------------------------------------------------------------------

def _two_level(s, **kw):
    return oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, **kw)


def test_two_grid_correction_is_a_galerkin_projection():
    """With no smoothing, z = P A_c^{-1} P^T r, so P^T (r - A z) = 0: pins the
    explicit restriction, the prolongation and the Galerkin operator."""
    s = rand_system(n_side=6, seed=10)
    agg, nc = aggregates(s)
    w = 0.1 + P.uniform01(15, 0, nc * 2)
    h = _two_level(s, n_pre=0, n_post=0, smooth_p=1, omega_p_arr=w)
    prp, pci, pv = h.prolongator(0)
    Pm = p_dense(prp, pci, pv, s.n_nodes, nc, 6, 2)
    r = P.uniform_pm1(16, 0, s.n_nodes * 6)
    z = h.vcycle(r)
    A = s.dense()
    np.testing.assert_allclose(Pm.T @ (r - A @ z), 0.0, atol=1e-11 * np.abs(Pm.T @ r).max())
    np.testing.assert_allclose(z, Pm @ np.linalg.solve(Pm.T @ A @ Pm, Pm.T @ r), rtol=0,
                               atol=1e-10 * np.abs(z).max())


def test_constant_weight_arrays_reproduce_the_constants():
    s = P.mhd2d(12, 2)
    h0 = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, omega=0.55, smooth_p=1, omega_p=0.2)
    sizes = [h0.level_sizes(l) for l in range(h0.num_levels - 1)]
    ws = np.concatenate([np.full(n * 2, 0.55) for n, _, _, _ in sizes])
    wp = np.concatenate([np.full(na * 2, 0.2) for _, _, _, na in sizes])
    h1 = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, omega=0.9, smooth_p=1, omega_s_arr=ws,
                                      omega_p_arr=wp)
    r = P.uniform_pm1(17, 0, s.n_nodes * 6)
    np.testing.assert_array_equal(h0.vcycle(r), h1.vcycle(r))


def test_weight_arrays_must_match_the_hierarchy():
    s = P.mhd2d(12, 2)
    h0 = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0)
    n_s = sum(h0.level_sizes(l)[0] * 2 for l in range(h0.num_levels - 1))
    for bad in (n_s - 1, n_s + 2):
        with pytest.raises(oracle.OracleError):
            oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, omega_s_arr=np.full(bad, 0.5))


def test_per_node_damping_on_a_block_diagonal_matrix():
    """No neighbour couplings: one sweep of Algorithm 1 is, field by field,
    x_f += omega_{i,f} D_ff,i^{-1} (b_f - sum_g A_fg x_g) at every node."""
    s = rand_system(n_side=6, seed=12)
    v = s.vals.copy()
    for i in range(s.n_nodes):
        for k in range(s.row_ptr[i], s.row_ptr[i + 1]):
            if s.col_idx[k] != i:
                v[k] = 0.0
    h0 = oracle.Hierarchy(s.row_ptr, s.col_idx, v, 6, FM6, max_levels=2, max_coarse=0)
    n0 = h0.level_sizes(0)[0]
    w = 0.2 + P.uniform01(18, 0, n0 * 2).reshape(n0, 2)
    h = oracle.Hierarchy(s.row_ptr, s.col_idx, v, 6, FM6, max_levels=2, max_coarse=0, omega_s_arr=w)
    x0 = P.uniform_pm1(19, 0, n0 * 6)
    rhs = P.uniform_pm1(20, 0, n0 * 6)
    got = h.bgs(0, x0, rhs, 1)
    x = x0.reshape(n0, 6).copy()
    bb = rhs.reshape(n0, 6)
    for i in range(n0):
        Aii = v[[k for k in range(s.row_ptr[i], s.row_ptr[i + 1]) if s.col_idx[k] == i][0]]
        for f in range(2):
            sl = slice(3 * f, 3 * f + 3)
            r = bb[i, sl] - Aii[sl, :] @ x[i]
            x[i, sl] += w[i, f] * np.linalg.solve(Aii[sl, sl], r)
    np.testing.assert_allclose(got, x.ravel(), rtol=0, atol=1e-12 * np.abs(x).max())


# ----------------------------------------------------------------------------
# network and its use in the setup
# ----------------------------------------------------------------------------
NF, NH, NO = oracle.NFEAT, oracle.MLP_H, oracle.MLP_OUT
O_W1, O_B1 = 0, NH * NF
O_W2 = O_B1 + NH
O_B2 = O_W2 + NH * NH
O_W3 = O_B2 + NH
O_B3 = O_W3 + NO * NH
O_XM = O_B3 + NO
O_XS = O_XM + NF


def zero_params():
    p = np.zeros(oracle.MLP_NPARAMS)
    p[O_XS:O_XS + NF] = 1.0
    return p


def random_params(seed, scale=0.3):
    p = (P.uniform01(seed, 0, oracle.MLP_NPARAMS) - 0.5) * 2 * scale
    p[O_XM:O_XM + NF] = P.uniform01(seed + 1, 0, NF) - 0.5
    p[O_XS:O_XS + NF] = 0.5 + P.uniform01(seed + 2, 0, NF)
    return p


def test_mlp_constant_output():
    p = zero_params()
    p[O_B3:O_B3 + 2] = [0.25, -1.5]
    x = P.uniform_pm1(21, 0, 5 * NF) * 10
    np.testing.assert_array_equal(oracle.mlp_forward(p, x), np.tile([0.25, -1.5], (5, 1)))


def test_mlp_second_layer_bias_only():
    p = random_params(22)
    p[O_W2:O_B2] = 0.0
    x = P.uniform_pm1(23, 0, 4 * NF)
    h2 = np.tanh(p[O_B2:O_W3])
    W3 = p[O_W3:O_B3].reshape(NO, NH)
    want = W3 @ h2 + p[O_B3:O_XM]
    np.testing.assert_allclose(oracle.mlp_forward(p, x), np.tile(want, (4, 1)), rtol=1e-14, atol=1e-14)


def test_mlp_single_path_closed_form():
    p = zero_params()
    a, w, v, m0 = 0.7, -1.3, 0.9, 3
    p[O_W1 + 0 * NF + m0] = a
    p[O_W2 + 0 * NH + 0] = w
    p[O_W3 + 0 * NH + 0] = v
    p[O_B3:O_B3 + 2] = [0.1, 0.2]
    p[O_XM + m0] = 0.25
    p[O_XS + m0] = 2.0
    x = P.uniform_pm1(24, 0, 6 * NF).reshape(6, NF)
    y = oracle.mlp_forward(p, x)
    want0 = v * np.tanh(w * np.tanh(a * (x[:, m0] - 0.25) * 2.0)) + 0.1
    np.testing.assert_allclose(y[:, 0], want0, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(y[:, 1], 0.2, rtol=0, atol=0)


def _loss(p, x, t, head):
    y = oracle.mlp_forward(p, x)
    return np.mean((y[np.arange(len(t)), head] - t) ** 2)


def test_mlp_gradient_matches_central_differences():
    p = random_params(25, scale=0.5)
    n = 6
    x = P.uniform_pm1(26, 0, n * NF).reshape(n, NF) * 2
    t = P.uniform_pm1(27, 0, n)
    head = np.array([0, 1, 1, 0, 1, 0], np.int32)
    loss, g = oracle.mlp_grad(p, x, t, head)
    assert loss == pytest.approx(_loss(p, x, t, head), rel=1e-14)
    h = 1e-6
    fd = np.zeros(oracle.MLP_NTRAIN)
    for q in range(oracle.MLP_NTRAIN):
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd[q] = (_loss(pp, x, t, head) - _loss(pm, x, t, head)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6 * np.abs(fd).max())
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)


def test_adam_steps_with_a_constant_gradient():
    """Bias correction makes every step of a constant gradient equal to
    -lr g / (|g| + eps)."""
    p0 = random_params(28)
    g = P.uniform_pm1(29, 0, oracle.MLP_NTRAIN)
    p = p0.copy()
    m = np.zeros(oracle.MLP_NTRAIN)
    v = np.zeros(oracle.MLP_NTRAIN)
    lr, eps = 1e-2, 1e-8
    for t in (1, 2, 3):
        oracle.adam(p, g, m, v, t, lr=lr, eps=eps)
    step = lr * g / (np.abs(g) + eps)
    np.testing.assert_allclose(p[:oracle.MLP_NTRAIN], p0[:oracle.MLP_NTRAIN] - 3 * step, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(p[oracle.MLP_NTRAIN:], p0[oracle.MLP_NTRAIN:])


def test_clip_ranges():
    assert oracle.mlp_clip(0, [-1.0, 0.0, 0.05, 0.7, 2.0, np.nan]).tolist() == [0.05, 0.05, 0.05, 0.7, 1.5, 0.05]
    assert oracle.mlp_clip(1, [-1.0, 0.049, 0.05, 0.7, 2.0, np.nan]).tolist() == [0.0, 0.0, 0.05, 0.7, 1.5, 0.0]


def test_network_setup_with_constant_outputs_matches_constant_weights():
    s = P.mhd2d(12, 3)
    r = P.uniform_pm1(30, 0, s.n_nodes * 6)
    p = zero_params()
    p[O_B3:O_B3 + 2] = [0.6, 0.01]  # P weight below the clip threshold: tentative P everywhere
    h_net = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, mlp=p)
    h_ref = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, omega=0.6)
    np.testing.assert_array_equal(h_net.vcycle(r), h_ref.vcycle(r))
    p[O_B3:O_B3 + 2] = [0.45, 0.3]
    h_net = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, mlp=p)
    h_ref = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, omega=0.45, smooth_p=1, omega_p=0.3)
    np.testing.assert_array_equal(h_net.vcycle(r), h_ref.vcycle(r))


# ----------------------------------------------------------------------------
# features
# ----------------------------------------------------------------------------

def test_features_of_a_laplacian_times_identity():
    """Blocks s_ij I_4 with two fields of two dofs: closed forms in the scalar
    stencil values s_ij."""
    s = P.poisson_block(6, 4, field_of_dof=[0, 0, 1, 1])
    agg, nc = aggregates(s)
    nf, af = oracle.features(s.row_ptr, s.col_idx, s.vals, s.field_of_dof, agg, nc, level=2)
    cnt = np.bincount(agg, minlength=nc)
    for i in range(s.n_nodes):
        ks = range(s.row_ptr[i], s.row_ptr[i + 1])
        sii = [s.vals[k, 0, 0] for k in ks if s.col_idx[k] == i][0]
        off = sum(abs(s.vals[k, 0, 0]) for k in ks if s.col_idx[k] != i)
        for f in range(2):
            want = [np.log(abs(sii) * np.sqrt(2)), off / abs(sii), 0.0, 0.0, np.sign(sii), np.log(cnt[agg[i]]),
                    2.0, float(f)]
            np.testing.assert_allclose(nf[i, f], want, rtol=1e-13, atol=1e-13)
    for I in range(nc):
        np.testing.assert_allclose(af[I], nf[agg == I].mean(axis=0), rtol=1e-13, atol=1e-13)


def test_features_scale_covariance():
    """A -> alpha A shifts log d by log alpha and leaves the other features;
    scaling the rows of field 1 only moves features 0 and 3 of field 1 and
    feature 3 of field 0."""
    s = rand_system(seed=31)
    agg, nc = aggregates(s)
    nf, _ = oracle.features(s.row_ptr, s.col_idx, s.vals, FM6, agg, nc, 0)
    nf2, _ = oracle.features(s.row_ptr, s.col_idx, s.vals * 8.0, FM6, agg, nc, 0)
    d = nf2 - nf
    np.testing.assert_allclose(d[:, :, 0], np.log(8.0), atol=1e-13)
    np.testing.assert_allclose(d[:, :, 1:], 0.0, atol=1e-13)
    v = s.vals.copy()
    v[:, 3:6, :] *= 4.0
    nf3, _ = oracle.features(s.row_ptr, s.col_idx, v, FM6, agg, nc, 0)
    d = nf3 - nf
    np.testing.assert_allclose(d[:, 1, 0], np.log(4.0), atol=1e-13)
    np.testing.assert_allclose(d[:, 1, 3], np.log(4.0) / 2, atol=1e-13)
    np.testing.assert_allclose(d[:, 0, 3], -np.log(4.0) / 2, atol=1e-13)
    np.testing.assert_allclose(d[:, :, [1, 2, 4, 5, 6, 7]], 0.0, atol=1e-13)
    np.testing.assert_allclose(d[:, 0, 0], 0.0, atol=1e-13)


def test_network_limited_to_its_trained_levels():
    """mlp_levels = 1: level 0 takes the network's weights, deeper levels the
    plain damping and the tentative prolongator."""
    s = P.mhd2d(12, 4)
    r = P.uniform_pm1(32, 0, s.n_nodes * 6)
    p = zero_params()
    p[O_B3:O_B3 + 2] = [0.6, 0.3]
    h_net = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, mlp=p, mlp_levels=1, omega=0.5)
    ws0, wp0 = h_net.omega(0)
    ws1, wp1 = h_net.omega(1)
    assert (ws0 == 0.6).all() and (wp0 == 0.3).all()
    assert (ws1 == 0.5).all() and (wp1 == 0.0).all()
    h_net.prolongator(0)
    with pytest.raises(oracle.OracleError):
        h_net.prolongator(1)
    # the same hierarchy with the network's output removed: constant weights on level 0 only
    p[O_B3:O_B3 + 2] = [0.6, 0.01]
    h_a = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, mlp=p, mlp_levels=1)
    n0, n1 = h_a.level_sizes(0)[0], h_a.level_sizes(1)[0]
    ws = np.concatenate([np.full(n0 * 2, 0.6), np.full(n1 * 2, 0.5)])
    h_b = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, omega_s_arr=ws)
    np.testing.assert_array_equal(h_a.vcycle(r), h_b.vcycle(r))
