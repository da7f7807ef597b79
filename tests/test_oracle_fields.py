"""Pins of the oracle's fields on disjoint node sets (fields that are not
co-located: separate aggregation per field block, Sec. 4.3.1; the mixed
Q2/Q1 example of Sec. 5).  CPU only.

Facts used, none of them from the oracle's node-field code:
* brute force: the roots of each field's aggregates are the
  lexicographically first maximal distance-2 independent set of the graph of
  that field's diagonal block (the aggregation rule, applied per field);
* dense linear algebra: Galerkin products P^T A P with the block-diagonal
  piecewise-constant P, Algorithm 1 as block forward substitutions per field,
  the V-cycle of Fig. 1 in matrix form;
* a reduction: with the coupling blocks set to zero the hierarchy must be the
  two co-located hierarchies of the diagonal blocks side by side (bit for
  bit), and those are pinned in test_oracle_pins.py;
* the paper's observation that the system cannot be handled as one
  non-blocked operator (Sec. 5, mixed elements).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

import oracle
from paper_2103_07537_gb300 import problems as P
from test_oracle_pins import brute_force_lex_first_mis2, bsr_dense, check_first_fit, csr_from_edges, tentative_P


def two_field_system(n0, n1, b, seed, p_in=0.3, p_cross=0.25):
    """Random structurally symmetric block system on two node sets: field 0 =
    nodes 0..n0-1, field 1 = nodes n0..n0+n1-1, random edges inside each set
    and across them, block-diagonally dominant values."""
    rng = np.random.default_rng(seed)
    n = n0 + n1
    fld = np.array([0] * n0 + [1] * n1)
    edges = []
    for a in range(n):
        for c in range(a + 1, n):
            if rng.random() < (p_in if fld[a] == fld[c] else p_cross):
                edges.append((a, c))
    rp, ci = csr_from_edges(n, edges)
    vals = rng.uniform(-1.0, 1.0, (len(ci), b, b))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            if ci[k] == i:
                vals[k] += np.eye(b) * (2.0 * b * (rp[i + 1] - rp[i]))
    return rp, ci, vals, [0, n0, n]


def subgraph(rp, ci, lo, hi):
    """CSR graph of the nodes lo..hi-1 (renumbered from 0), edges inside."""
    n = len(rp) - 1
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))[lo:hi, lo:hi].tocsr()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32)


def node_field_bgs_matrix_form(A, x, rhs, b, foff, colour, omega):
    """One sweep of Algorithm 1 with the field blocks on node sets, dense.

    Field g (nodes foff[g]..foff[g+1]-1, all dofs): r_g = rhs_g - A[g, :] x;
    the multicolour node-block Gauss-Seidel sweep from zero on A_gg is a block
    forward substitution with the part of A_gg that is block lower triangular
    in (colour, index) order; x_g += omega x~_g.
    """
    x = x.copy()
    for g in range(len(foff) - 1):
        nodes = list(range(foff[g], foff[g + 1]))
        order = sorted(nodes, key=lambda i: (colour[i], i))
        rank = {i: t for t, i in enumerate(order)}
        rows = np.array([i * b + r for i in nodes for r in range(b)])
        r_g = rhs[rows] - A[rows, :] @ x
        Agg = A[np.ix_(rows, rows)]
        T = np.zeros_like(Agg)
        m = len(nodes)
        for p in range(m):
            for q in range(m):
                if rank[nodes[q]] <= rank[nodes[p]]:
                    T[p * b:(p + 1) * b, q * b:(q + 1) * b] = Agg[p * b:(p + 1) * b, q * b:(q + 1) * b]
        x[rows] += omega * np.linalg.solve(T, r_g)
    return x


def hier(rp, ci, vals, foff, **kw):
    return oracle.Hierarchy(rp, ci, vals, vals.shape[1], [0] * vals.shape[1], node_field_off=foff, **kw)


# ----------------------------------------------------------------------------
# the Q2/Q1 input
# ----------------------------------------------------------------------------


def test_q2q1_system_structure():
    N = 5
    s = P.mhd2d_q2q1(N, 3)
    n2, n1 = (2 * N + 1) ** 2, (N + 1) ** 2
    assert s.node_field_off == [0, n2, n2 + n1] and s.n_nodes == n2 + n1 and s.b == 3
    rp, ci = s.row_ptr, s.col_idx
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(s.n_nodes, s.n_nodes))
    assert (A != A.T).nnz == 0  # structurally symmetric
    for i in range(s.n_nodes):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and i in row
    # a Q1 vertex shares a cell with at most 25 Q2 nodes and 9 Q1 vertices;
    # a Q2 cell-centre node only with its own cell's 9 Q2 nodes and 4 vertices
    deg = np.diff(rp)
    assert deg[n2:].max() == 25 + 9
    centre = (2 * 1 + 1) + (2 * N + 1) * (2 * 1 + 1)
    assert deg[centre] == 9 + 4
    # Dirichlet: identity rows for B and psi on boundary vertices
    v0 = n2  # vertex (0, 0)
    k = rp[v0] + int(np.nonzero(ci[rp[v0]:rp[v0 + 1]] == v0)[0][0])
    assert np.array_equal(s.vals[k], np.eye(3))
    assert np.count_nonzero(s.vals[rp[v0]:rp[v0 + 1]]) == 3


def test_q2_element_closed_form():
    # biquadratic element on [0, h]^2 with 3 x 3 Gauss points: K = Kx (x) My + Mx (x) Ky
    # with the 1D quadratic stiffness (1/(3h)) [[7,-8,1],[-8,16,-8],[1,-8,7]] and mass
    # (h/30) [[4,2,-1],[2,16,2],[-1,2,4]] (local node l = lx + 3 ly)
    h = 0.25
    g = np.sqrt(3.0 / 5.0)
    x1 = np.array([-g, 0.0, g])
    w1 = np.array([5.0, 8.0, 5.0]) / 9.0
    xi, et = np.tile(x1, 3), np.repeat(x1, 3)
    wq = np.tile(w1, 3) * np.repeat(w1, 3)
    phi, dphi = P._tensor_basis_2d(2, xi, et)
    grad = dphi * (2.0 / h)
    jac = (h / 2.0) ** 2
    K = np.einsum("q,qla,qma->lm", wq, grad, grad) * jac
    M = np.einsum("q,ql,qm->lm", wq, phi, phi) * jac
    K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3.0 * h)
    M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * (h / 30.0)
    assert np.allclose(K, np.kron(K1, M1) + np.kron(M1, K1), rtol=1e-13, atol=1e-15)
    assert np.allclose(M, np.kron(M1, M1), rtol=1e-13, atol=1e-16)
    # partition of unity and the nodal property of the basis
    assert np.allclose(phi.sum(axis=1), 1.0) and np.allclose(dphi.sum(axis=1), 0.0)
    nodes = np.array([-1.0, 0.0, 1.0])
    pv, _ = P._tensor_basis_2d(2, np.tile(nodes, 3), np.repeat(nodes, 3))
    assert np.allclose(pv, np.eye(9))


def test_q2q1_velocity_rows_annihilate_constants():
    # away from the boundary, the u-u part of a Q2 node's row is nu K2 (rows sum
    # to zero), and the B-B part of a Q1 vertex's row is eta K1
    N = 6
    s = P.mhd2d_q2q1(N, 2)
    m2 = 2 * N + 1
    rp, ci, v = s.row_ptr, s.col_idx, s.vals
    n2 = s.node_field_off[1]
    for X, Y in ((6, 6), (5, 7), (4, 5)):
        i = X + m2 * Y
        q2 = ci[rp[i]:rp[i + 1]] < n2
        blocks = v[rp[i]:rp[i + 1]][q2]
        for a in range(2):
            assert abs(blocks[:, a, a].sum()) < 1e-12 * np.abs(blocks[:, a, a]).max()
            assert np.all(blocks[:, a, 1 - a] == 0.0)
    j = n2 + 3 + (N + 1) * 3
    q1 = ci[rp[j]:rp[j + 1]] >= n2
    bl = v[rp[j]:rp[j + 1]][q1]
    for a in range(2):
        assert abs(bl[:, a, a].sum()) < 1e-12 * np.abs(bl[:, a, a]).max()
    assert abs(bl[:, 2, 2].sum()) < 1e-12 * np.abs(bl[:, 2, 2]).max()


def test_q2q1_bench_workload_sizes():
    # the sizes the benchmark's description states
    import bench

    wl = bench.WORKLOADS["mhd2d_q2q1_128"]
    s = wl["make"](1)
    assert (s.node_field_off, s.n_unknowns, s.nnzb) == ([0, 66049, 82690], 248070, 2020612)
    for text in ("66,049 Q2 nodes", "16,641 Q1 vertices", "248,070 unknowns", "omega=0.6"):
        assert text in wl["desc"]
    assert wl["omega"] == 0.6 and wl["levels"] == 4


# ----------------------------------------------------------------------------
# separate aggregation and colouring per field block
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("seed", range(5))
def test_roots_per_field_are_lex_first_distance2_mis(seed):
    rp, ci, vals, foff = two_field_system(9, 8, 2, seed)
    h = hier(rp, ci, vals, foff, max_levels=2, max_coarse=0)
    L = h.level(0)
    agg = L["agg"]
    coarse_off = h.fields(1)[0]
    for g in range(2):
        lo, hi = foff[g], foff[g + 1]
        srp, sci = subgraph(rp, ci, lo, hi)
        roots = brute_force_lex_first_mis2(srp, sci)
        # the roots are the nodes that carry a new aggregate id first, in order
        ids = agg[lo:hi]
        assert ids.min() == coarse_off[g] and ids.max() == coarse_off[g + 1] - 1
        root_of = {}
        for t, r in enumerate(roots):
            root_of[coarse_off[g] + t] = r
        for I, r in root_of.items():
            assert agg[lo + r] == I
            # the root's neighbourhood in A_gg is in its aggregate (rule step 1)
            assert np.all(agg[lo + sci[srp[r]:srp[r + 1]]] == I)


@pytest.mark.parametrize("make", [lambda: two_field_system(40, 30, 2, 11, 0.08, 0.05),
                                  lambda: (lambda s: (s.row_ptr, s.col_idx, s.vals, s.node_field_off))(
                                      P.mhd2d_q2q1(6, 1))])
def test_aggregates_and_colours_stay_in_their_field(make):
    rp, ci, vals, foff = make()
    h = hier(rp, ci, vals, foff, max_levels=3, max_coarse=0)
    assert h.num_levels == 3
    for l in range(2):
        L = h.level(l)
        no, co = h.fields(l)
        nc_off = h.fields(l + 1)[0]
        lrp, lci = L["row_ptr"], L["col_idx"]
        assert no[0] == 0 and no[-1] == L["n"] and nc_off[-1] == L["n_agg"]
        for g in range(2):
            lo, hi = no[g], no[g + 1]
            srp, sci = subgraph(lrp, lci, lo, hi)
            a = L["agg"][lo:hi] - nc_off[g]
            nag = nc_off[g + 1] - nc_off[g]
            assert a.min() == 0 and a.max() == nag - 1
            # a disjoint cover of the field's nodes by aggregates that are
            # connected in the graph of A_gg
            assert len(np.unique(a)) == nag
            G = sp.csr_matrix((np.ones(len(sci)), sci, srp), shape=(hi - lo, hi - lo))
            for I in range(nag):
                mem = np.nonzero(a == I)[0]
                assert csgraph.connected_components(G[mem][:, mem], directed=False)[0] == 1
            # colours of field g: first fit on the graph of A_gg, after field g-1's
            c = L["colour"][lo:hi]
            assert c.min() == co[g] and c.max() == co[g + 1] - 1
            check_first_fit(srp, sci, c - co[g])
        assert co[-1] == L["n_colours"]


# ----------------------------------------------------------------------------
# Galerkin products, smoother and V-cycle in matrix form
# ----------------------------------------------------------------------------


def test_rap_with_block_diagonal_P_equals_dense_galerkin():
    s = P.mhd2d_q2q1(6, 2)
    h = hier(s.row_ptr, s.col_idx, s.vals, s.node_field_off, max_levels=3, max_coarse=0)
    A = s.dense()
    for l in range(2):
        L = h.level(l)
        Pm = tentative_P(L["agg"], L["n_agg"], 3)
        no, nc_off = h.fields(l)[0], h.fields(l + 1)[0]
        # P = diag(P_0, P_1): no entry couples a fine node of one field with a
        # coarse node of the other
        assert not Pm[no[0] * 3:no[1] * 3, nc_off[1] * 3:].any()
        assert not Pm[no[1] * 3:, :nc_off[1] * 3].any()
        Ac = Pm.T @ A @ Pm
        C = h.level(l + 1)
        assert np.allclose(bsr_dense(C["row_ptr"], C["col_idx"], C["vals"]), Ac, rtol=1e-12,
                           atol=1e-12 * np.abs(Ac).max())
        # the coupling blocks survive on the coarse level
        assert np.abs(Ac[nc_off[1] * 3:, :nc_off[1] * 3]).max() > 0
        A = Ac


@pytest.mark.parametrize("omega", [0.6, 1.0])
@pytest.mark.parametrize("kind", ["q2q1", "random"])
def test_bgs_node_fields_equals_matrix_form(kind, omega):
    if kind == "q2q1":
        s = P.mhd2d_q2q1(3, 4)
        rp, ci, vals, foff, rhs = s.row_ptr, s.col_idx, s.vals, s.node_field_off, s.rhs
    else:
        rp, ci, vals, foff = two_field_system(12, 9, 3, 5)
        rhs = P.uniform_pm1(9, 0, 21 * 3)
    b = vals.shape[1]
    h = hier(rp, ci, vals, foff, max_levels=2, max_coarse=0, omega=omega)
    A = bsr_dense(rp, ci, vals)
    colour = h.level(0)["colour"]
    x0 = P.uniform_pm1(17, 0, len(rhs))
    ref = node_field_bgs_matrix_form(A, x0, rhs, b, foff, colour, omega)
    assert np.allclose(h.bgs(0, x0, rhs, sweeps=1), ref, rtol=1e-10, atol=1e-12)
    ref2 = node_field_bgs_matrix_form(A, ref, rhs, b, foff, colour, omega)
    assert np.allclose(h.bgs(0, x0, rhs, sweeps=2), ref2, rtol=1e-10, atol=1e-12)


def test_vcycle_two_level_no_smoothing_is_coarse_correction():
    s = P.mhd2d_q2q1(4, 5)
    h = hier(s.row_ptr, s.col_idx, s.vals, s.node_field_off, max_levels=2, max_coarse=0, n_pre=0, n_post=0)
    L = h.level(0)
    Pm = tentative_P(L["agg"], L["n_agg"], 3)
    A = s.dense()
    ref = Pm @ np.linalg.solve(Pm.T @ A @ Pm, Pm.T @ s.rhs)
    assert np.allclose(h.vcycle(s.rhs), ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())


def test_vcycle_three_levels_matches_matrix_form():
    s = P.mhd2d_q2q1(6, 7)
    om = 0.6
    h = hier(s.row_ptr, s.col_idx, s.vals, s.node_field_off, max_levels=3, max_coarse=0, omega=om)
    L0, L1 = h.level(0), h.level(1)
    f0, f1 = h.fields(0)[0], h.fields(1)[0]
    P0 = tentative_P(L0["agg"], L0["n_agg"], 3)
    P1 = tentative_P(L1["agg"], L1["n_agg"], 3)
    A0 = s.dense()
    A1 = P0.T @ A0 @ P0
    A2 = P1.T @ A1 @ P1

    def mgv(A, r, colour, foff, Pl, below):
        u = node_field_bgs_matrix_form(A, np.zeros_like(r), r, 3, foff, colour, om)
        u = u + Pl @ below(Pl.T @ (r - A @ u))
        return node_field_bgs_matrix_form(A, u, r, 3, foff, colour, om)

    ref = mgv(A0, s.rhs, L0["colour"], f0, P0,
              lambda rc: mgv(A1, rc, L1["colour"], f1, P1, lambda rcc: np.linalg.solve(A2, rcc)))
    z = h.vcycle(s.rhs)
    assert np.allclose(z, ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("sub", [{}, dict(sub_ilu=1), dict(sub_ilu=2), dict(sub_schwarz=2), dict(sub_schwarz=1)])
def test_decoupled_fields_equal_two_colocated_hierarchies(sub):
    # with A_01 = A_10 = 0 the node-field hierarchy is the co-located
    # hierarchies of A_00 and A_11 side by side: same aggregates, colours,
    # coarse operators and V-cycle, bit for bit, with every sub-solve
    s = P.mhd2d_q2q1(6, 2)
    n2, n = s.node_field_off[1], s.n_nodes
    rp, ci = s.row_ptr, s.col_idx
    v = s.vals.copy()
    r_of = np.repeat(np.arange(n), np.diff(rp))
    v[(r_of < n2) != (ci < n2)] = 0.0

    def part(lo, hi):
        keep = (r_of >= lo) & (r_of < hi) & (ci >= lo) & (ci < hi)
        prp = np.zeros(hi - lo + 1, np.int32)
        prp[1:] = np.cumsum(np.bincount(r_of[keep] - lo, minlength=hi - lo))
        return prp, (ci[keep] - lo).astype(np.int32), v[keep]

    kw = dict(max_levels=3, max_coarse=0, omega=0.6, **sub)
    h = hier(rp, ci, v, s.node_field_off, **kw)
    h0 = oracle.Hierarchy(*part(0, n2), 3, [0, 0, 0], **kw)
    h1 = oracle.Hierarchy(*part(n2, n), 3, [0, 0, 0], **kw)
    assert h.num_levels == h0.num_levels == h1.num_levels == 3
    for l in range(2):
        L, a, c = h.level(l), h0.level(l), h1.level(l)
        no = h.fields(l)[0]
        assert np.array_equal(L["agg"], np.concatenate([a["agg"], c["agg"] + a["n_agg"]]))
        assert np.array_equal(L["colour"], np.concatenate([a["colour"], c["colour"] + a["n_colours"]]))
        assert no.tolist() == [0, a["n"], a["n"] + c["n"]]
    z = h.vcycle(s.rhs)
    z0 = h0.vcycle(s.rhs[:n2 * 3])
    z1 = h1.vcycle(s.rhs[n2 * 3:])
    assert np.array_equal(z, np.concatenate([z0, z1]))


# ----------------------------------------------------------------------------
# the solve, and what the blocked construction buys (Sec. 5, mixed elements)
# ----------------------------------------------------------------------------


def test_fgmres_blocked_converges_nonblocked_does_not():
    # Sec. 5: the mixed system is out of reach of AMG that treats it as one
    # operator; the blocked hierarchy with separate aggregates converges
    s = P.mhd2d_q2q1(16, 1)
    kw = dict(max_levels=4, max_coarse=0, omega=0.6)
    hb = hier(s.row_ptr, s.col_idx, s.vals, s.node_field_off, **kw)
    _, it, rr, ok = hb.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=600)
    assert ok and rr <= 1e-8 and it < 300
    hn = oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, 3, [0, 0, 0], **kw)
    _, itn, rrn, okn = hn.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=600)
    assert not okn and rrn > 1e-6


def test_node_field_validation():
    s = P.mhd2d_q2q1(3, 1)
    args = (s.row_ptr, s.col_idx, s.vals, 3, [0, 0, 0])
    n = s.n_nodes
    for off in ([0, 0, n], [0, 50, n - 1], [1, 50, n], [0, 60, 50, n]):
        with pytest.raises(oracle.OracleError):
            oracle.Hierarchy(*args, max_levels=2, max_coarse=0, node_field_off=off)
    for kw in (dict(smooth_p=1, omega_p=0.5), dict(sub_ilu=1, sub_schwarz=2)):
        with pytest.raises(oracle.OracleError):
            oracle.Hierarchy(*args, max_levels=2, max_coarse=0, node_field_off=s.node_field_off, **kw)
    with pytest.raises(oracle.OracleError):  # dof fields and node fields together
        oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, 3, [0, 0, 1], max_levels=2, max_coarse=0,
                         node_field_off=s.node_field_off)
