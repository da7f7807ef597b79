"""Pins of the FP64 oracle against facts that do not come from the oracle:
published generator values, dense linear algebra (numpy / scipy), brute
force on tiny graphs, closed forms of the tentative transfers, hand-worked
graphs and the matrix form of the smoother.  CPU only.

Paper passages: V-cycle Fig. 1 (Sec. 3); Galerkin product (Sec. 3);
block-diagonal piecewise-constant transfers and cloned aggregates
(Sec. 4.3.1, eq. blocktransfers); aggregates as a disjoint cover
(Sec. 4.3.1); damped block Gauss-Seidel (Sec. 4.3.2, Algorithm 1).
"""
import dataclasses
import os
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

import oracle
from paper_2103_07537_gb300 import problems as P

# ----------------------------------------------------------------------------
# helpers that restate definitions in matrix form (independent of the oracle)
# ----------------------------------------------------------------------------


def graph_of(row_ptr, col_idx):
    n = len(row_ptr) - 1
    A = sp.csr_matrix((np.ones(len(col_idx)), col_idx, row_ptr), shape=(n, n))
    A.setdiag(0)
    A.eliminate_zeros()
    return A


def hop_distances(row_ptr, col_idx):
    return csgraph.shortest_path(graph_of(row_ptr, col_idx), unweighted=True, directed=False)


def csr_from_edges(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    for i in range(n):
        adj[i].add(i)
    rp = [0]
    ci = []
    for i in range(n):
        ci += sorted(adj[i])
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32)


def tentative_P(agg, nc, b):
    """Dense piecewise-constant prolongator, unit entries, every dof."""
    n = len(agg)
    Pm = np.zeros((n * b, nc * b))
    for i in range(n):
        for d in range(b):
            Pm[i * b + d, agg[i] * b + d] = 1.0
    return Pm


def bsr_dense(row_ptr, col_idx, vals):
    b = vals.shape[1]
    n = len(row_ptr) - 1
    return sp.bsr_matrix((vals, col_idx, row_ptr), shape=(n * b, n * b)).toarray()


def bgs_matrix_form(A, x, rhs, b, F, colour, omega, inner=1, fmap=None):
    """One sweep of Algorithm 1 written with dense matrices.

    For field f: r_f = rhs_f - A[f rows, :] x; the multicolour node-block
    Gauss-Seidel sweep from zero is a block forward substitution with the
    part of A_ff that is block lower triangular in (colour, index) order;
    then x_f += omega x~_f.  With inner > 1 the sub-solve iterates
    x~ <- T^-1 (r_f - (A_ff - T) x~) from x~ = 0, inner times (T: that lower part).
    fmap: the field of every dof of a node (fields may differ in size); None:
    F fields of b / F consecutive dofs.
    """
    if fmap is None:
        fmap = [d // (b // F) for d in range(b)]
    n = len(colour)
    order = sorted(range(n), key=lambda i: (colour[i], i))
    rank = np.empty(n, int)
    rank[order] = np.arange(n)
    x = x.copy()
    for f in range(F):
        dofs = [d for d in range(b) if fmap[d] == f]
        fb = len(dofs)
        rows = np.array([i * b + d for i in range(n) for d in dofs])
        r_f = rhs[rows] - A[rows, :] @ x
        Aff = A[np.ix_(rows, rows)]
        T = np.zeros_like(Aff)
        for i in range(n):
            for j in range(n):
                if rank[j] <= rank[i]:
                    T[i * fb:(i + 1) * fb, j * fb:(j + 1) * fb] = Aff[i * fb:(i + 1) * fb, j * fb:(j + 1) * fb]
        xt = np.zeros_like(r_f)
        for _ in range(inner):
            xt = np.linalg.solve(T, r_f - (Aff - T) @ xt)
        x[rows] += omega * xt
    return x


# ----------------------------------------------------------------------------
# input generator
# ----------------------------------------------------------------------------


def test_splitmix64_published_values():
    # first outputs of splitmix64 seeded with 0 (reference C implementation)
    v = P.splitmix64(0, 0, 3)
    assert [int(t) for t in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_q1_stiffness_closed_form():
    # bilinear element on a square: 2/3 diagonal, -1/6 edge, -1/3 diagonal partner
    s = P.poisson_block(1, 1)  # one cell, all four nodes on the boundary -> identity
    assert np.allclose(s.dense(), np.eye(4))
    s = P.poisson_block(2, 1)
    A = s.dense()
    centre = 4  # the only interior node of a 3 x 3 node grid
    row = A[centre].reshape(3, 3)
    assert np.isclose(row[1, 1], 4 * 2.0 / 3.0)
    assert np.isclose(row[0, 1], 0.0) and np.isclose(row[0, 0], 0.0)  # boundary columns eliminated


def test_generated_workload_sizes():
    s = P.stokes2d(32, 1)
    assert (s.n_nodes, s.b, s.n_unknowns, s.nnzb) == (1089, 3, 3267, (3 * 33 - 2) ** 2)
    m = P.mhd2d(16, 1)
    assert m.b == 6 and m.field_of_dof == [0, 0, 0, 1, 1, 1] and m.nnzb == (3 * 17 - 2) ** 2
    lo, hi = 1e-3, 1.0
    assert lo <= m.params["nu"] <= hi and lo <= m.params["eta"] <= hi


# ----------------------------------------------------------------------------
# dense kernels
# ----------------------------------------------------------------------------


def test_lu_matches_numpy_solve():
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 17, 40):
        A = rng.standard_normal((n, n))
        rhs = rng.standard_normal(n)
        lu, piv = oracle.lu_factor(A)
        x = oracle.lu_solve(lu, piv, rhs)
        assert np.allclose(x, np.linalg.solve(A, rhs), rtol=1e-10, atol=1e-12)


def test_lu_pivot_first_maximum():
    A = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [3.0, 0.0, 2.0]])
    lu, piv = oracle.lu_factor(A)
    assert piv[0] == 1  # |-3| and |3| tie: the first wins
    with pytest.raises(oracle.OracleError):
        oracle.lu_factor(np.array([[1.0, 2.0], [2.0, 4.0]]))


def test_block_inverse_matches_numpy():
    rng = np.random.default_rng(4)
    for m in (1, 3, 4, 6):
        for _ in range(5):
            a = rng.standard_normal((m, m)) + m * np.eye(m)
            assert np.allclose(oracle.block_inverse(a), np.linalg.inv(a), rtol=1e-12, atol=1e-12)
    a = np.array([[0.0, 2.0], [3.0, 1.0]])  # needs a row exchange
    assert np.allclose(oracle.block_inverse(a), np.linalg.inv(a))
    with pytest.raises(oracle.OracleError):
        oracle.block_inverse(np.array([[1.0, 1.0], [1.0, 1.0]]))


def test_spmv_matches_scipy():
    s = P.random_block_system(5, 6, [0, 0, 0, 1, 1, 1], seed=7)
    x = np.random.default_rng(0).standard_normal(s.n_unknowns)
    assert np.allclose(oracle.spmv(s.row_ptr, s.col_idx, s.vals, x), s.to_scipy() @ x, rtol=1e-14, atol=1e-13)


# ----------------------------------------------------------------------------
# aggregation
# ----------------------------------------------------------------------------


def brute_force_lex_first_mis2(row_ptr, col_idx):
    """Among all maximal sets with pairwise hop distance >= 3, the one whose
    sorted index tuple is lexicographically smallest (exhaustive search)."""
    n = len(row_ptr) - 1
    D = hop_distances(row_ptr, col_idx)
    best = None
    for mask in range(1, 1 << n):
        S = [i for i in range(n) if mask >> i & 1]
        if any(D[a, b] < 3 for a, b in itertools.combinations(S, 2)):
            continue
        if any(all(D[v, s] >= 3 for s in S) for v in range(n) if v not in S):
            continue  # not maximal
        if best is None or tuple(S) < tuple(best):
            best = S
    return best


@pytest.mark.parametrize("seed", range(6))
def test_aggregation_roots_are_lex_first_distance2_mis(seed):
    rng = np.random.default_rng(seed)
    n = 11
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.22]
    rp, ci = csr_from_edges(n, edges)
    agg, root, nagg = oracle.aggregate(rp, ci)
    assert sorted(np.nonzero(root)[0].tolist()) == brute_force_lex_first_mis2(rp, ci)
    # aggregate ids are the ranks of the roots
    assert agg[np.nonzero(root)[0]].tolist() == list(range(nagg))


def check_aggregate_invariants(rp, ci, agg, root, nagg):
    n = len(rp) - 1
    D = hop_distances(rp, ci)
    roots = np.nonzero(root)[0]
    assert len(roots) == nagg
    assert agg.min() >= 0 and agg.max() == nagg - 1 and len(np.unique(agg)) == nagg  # disjoint cover
    assert all(D[a, b] >= 3 for a, b in itertools.combinations(roots, 2))
    assert all(min(D[v, roots]) <= 2 for v in range(n))  # maximal at distance 2
    for I in range(nagg):
        members = np.nonzero(agg == I)[0]
        assert roots[I] in members
        sub = graph_of(rp, ci)[members][:, members]
        assert csgraph.connected_components(sub, directed=False)[0] == 1
        # the root's whole neighbourhood is in its aggregate
        nbrs = ci[rp[roots[I]]:rp[roots[I] + 1]]
        assert np.all(agg[nbrs] == I)


@pytest.mark.parametrize("seed", range(4))
def test_aggregation_invariants_random_graphs(seed):
    rng = np.random.default_rng(100 + seed)
    n = 60
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.06]
    rp, ci = csr_from_edges(n, edges)
    agg, root, nagg = oracle.aggregate(rp, ci)
    check_aggregate_invariants(rp, ci, agg, root, nagg)


def test_aggregation_hand_worked_attach_tie():
    # edges 0-1, 1-4, 4-3, 3-2: roots 0 {0,1} and 2 {2,3}; node 4 has one
    # neighbour in each, the tie goes to the smaller id
    rp, ci = csr_from_edges(5, [(0, 1), (1, 4), (4, 3), (3, 2)])
    agg, root, nagg = oracle.aggregate(rp, ci)
    assert nagg == 2 and agg.tolist() == [0, 0, 1, 1, 0] and root.tolist() == [1, 0, 1, 0, 0]


def test_aggregation_hand_worked_attach_majority():
    # roots 0 {0,1,2} and 3 {3,4}; node 5 touches 1, 2 (aggregate 0) and 4
    # (aggregate 1): it joins aggregate 0 by majority
    rp, ci = csr_from_edges(6, [(0, 1), (0, 2), (1, 5), (2, 5), (5, 4), (4, 3)])
    agg, root, nagg = oracle.aggregate(rp, ci)
    assert agg.tolist() == [0, 0, 0, 1, 1, 0]


def test_aggregation_path_closed_form():
    # a path of m nodes: {0,1}, {2,3,4}, {5,6,7}, ... and a trailing node joins the last
    for m in (2, 5, 8, 9, 10, 33):
        rp, ci = csr_from_edges(m, [(i, i + 1) for i in range(m - 1)])
        agg, root, nagg = oracle.aggregate(rp, ci)
        expect = [0 if i < 2 else (i - 2) // 3 + 1 for i in range(m)]
        n_roots = len(range(0, m, 3))
        expect = [min(e, n_roots - 1) for e in expect]
        assert agg.tolist() == expect, m


def test_aggregation_structured_grid_3x3():
    # 33 x 33 node grid, 9-point stencil: tensor product of the path rule, 11 x 11 aggregates
    s = P.stokes2d(32, 1)
    agg, root, nagg = oracle.aggregate(s.row_ptr, s.col_idx)
    assert nagg == 121
    one_d = [0 if i < 2 else min((i - 2) // 3 + 1, 10) for i in range(33)]
    expect = np.array([one_d[y] * 11 + one_d[x] for y in range(33) for x in range(33)])
    assert np.array_equal(agg, expect)
    check_aggregate_invariants(s.row_ptr, s.col_idx, agg, root, nagg)


# ----------------------------------------------------------------------------
# colouring
# ----------------------------------------------------------------------------


def check_first_fit(rp, ci, col):
    """A proper colouring in which every node of colour c sees lower-index
    neighbours of every colour below c is exactly first fit in index order."""
    n = len(rp) - 1
    for i in range(n):
        nb = [j for j in ci[rp[i]:rp[i + 1]] if j != i]
        assert all(col[j] != col[i] for j in nb)
        lower = {col[j] for j in nb if j < i}
        assert set(range(col[i])) <= lower


def test_colouring_grid_closed_forms():
    s = P.stokes2d(8, 1)
    col, nc = oracle.colour(s.row_ptr, s.col_idx)
    assert nc == 4
    expect = [(x % 2) + 2 * (y % 2) for y in range(9) for x in range(9)]
    assert col.tolist() == expect
    s3 = P.stokes3d(4, 1)
    col3, nc3 = oracle.colour(s3.row_ptr, s3.col_idx)
    assert nc3 == 8
    expect3 = [(x % 2) + 2 * (y % 2) + 4 * (z % 2) for z in range(5) for y in range(5) for x in range(5)]
    assert col3.tolist() == expect3


@pytest.mark.parametrize("seed", range(4))
def test_colouring_first_fit_random(seed):
    rng = np.random.default_rng(200 + seed)
    n = 80
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.08]
    rp, ci = csr_from_edges(n, edges)
    col, nc = oracle.colour(rp, ci)
    assert nc == col.max() + 1
    check_first_fit(rp, ci, col)


# ----------------------------------------------------------------------------
# Galerkin product with the tentative prolongator
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("kind", ["random6", "stokes", "random4_3d"])
def test_rap_equals_dense_galerkin(kind):
    if kind == "random6":
        s = P.random_block_system(7, 6, [0, 0, 0, 1, 1, 1], seed=11)
    elif kind == "stokes":
        s = P.stokes2d(8, 2)
    else:
        s = P.random_block_system(4, 4, [0, 0, 0, 0], seed=12, d=3)
    agg, root, nc = oracle.aggregate(s.row_ptr, s.col_idx)
    rpc, cic, vc = oracle.rap_tentative(s.row_ptr, s.col_idx, s.vals, s.b, agg, nc)
    Pm = tentative_P(agg, nc, s.b)
    Ac = Pm.T @ s.dense() @ Pm
    assert np.allclose(bsr_dense(rpc, cic, vc), Ac, rtol=1e-13, atol=1e-12)
    # the pattern is the structural product of the patterns, columns ascending
    n = s.n_nodes
    S = sp.csr_matrix((np.ones(s.nnzb), s.col_idx, s.row_ptr), shape=(n, n))
    Pn = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
    Sc = (Pn.T @ S @ Pn).tocsr()
    Sc.sort_indices()
    assert np.array_equal(rpc, Sc.indptr) and np.array_equal(cic, Sc.indices)
    # Galerkin identity on vectors
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(nc * s.b), rng.standard_normal(nc * s.b)
    assert np.isclose(v @ bsr_dense(rpc, cic, vc) @ u, (Pm @ v) @ s.dense() @ (Pm @ u), rtol=1e-11)


def test_rap_block_diagonal_across_fields():
    # with A01 = A10 = 0 the coarse operator keeps them zero (P is block diagonal, eq. blocktransfers)
    s = P.random_block_system(6, 6, [0, 0, 0, 1, 1, 1], seed=13)
    s.vals[:, :3, 3:] = 0.0
    s.vals[:, 3:, :3] = 0.0
    agg, root, nc = oracle.aggregate(s.row_ptr, s.col_idx)
    _, _, vc = oracle.rap_tentative(s.row_ptr, s.col_idx, s.vals, s.b, agg, nc)
    assert np.all(vc[:, :3, 3:] == 0.0) and np.all(vc[:, 3:, :3] == 0.0)


# ----------------------------------------------------------------------------
# hierarchy, smoother, V-cycle
# ----------------------------------------------------------------------------


def test_hierarchy_levels_of_the_named_workloads():
    s = P.stokes2d(32, 1)
    h = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0)
    assert [h.level_sizes(l)[0] for l in range(h.num_levels)] == [1089, 121, 16]
    m = P.mhd2d(128, 1)
    h = oracle.Hierarchy.from_system(m, max_levels=4, max_coarse=0)
    assert [h.level_sizes(l)[0] for l in range(h.num_levels)] == [16641, 1849, 225, 25]
    # the default rule coarsens while n * b > 2500
    h = oracle.Hierarchy.from_system(m, max_levels=10, max_coarse=2500)
    assert [h.level_sizes(l)[0] for l in range(h.num_levels)] == [16641, 1849, 225]


def test_block_diagonal_inverses_in_hierarchy():
    m = P.mhd2d(8, 3)
    h = oracle.Hierarchy.from_system(m, max_levels=2, max_coarse=0)
    L = h.level(0)
    for i in range(L["n"]):
        k = L["row_ptr"][i] + list(L["col_idx"][L["row_ptr"][i]:L["row_ptr"][i + 1]]).index(i)
        for f in range(2):
            D = L["vals"][k][3 * f:3 * f + 3, 3 * f:3 * f + 3]
            assert np.allclose(L["dinv"][i, f] @ D, np.eye(3), atol=1e-10)


@pytest.mark.parametrize("kind,F", [("random6", 2), ("mhd", 2), ("stokes", 1), ("random4", 1)])
@pytest.mark.parametrize("omega", [0.5, 0.8])
def test_bgs_equals_matrix_form(kind, F, omega):
    if kind == "random6":
        s = P.random_block_system(6, 6, [0, 0, 0, 1, 1, 1], seed=21)
    elif kind == "mhd":
        s = P.mhd2d(6, 2)
    elif kind == "stokes":
        s = P.stokes2d(6, 3)
    else:
        s = P.random_block_system(5, 4, [0, 0, 0, 0], seed=22)
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, omega=omega)
    L = h.level(0)
    A = s.dense()
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal(s.n_unknowns)
    x1 = h.bgs(0, x0, s.rhs, 1)
    ref = bgs_matrix_form(A, x0, s.rhs, s.b, F, L["colour"], omega)
    assert np.allclose(x1, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    # two sweeps = the matrix form applied twice
    x2 = h.bgs(0, x0, s.rhs, 2)
    ref2 = bgs_matrix_form(A, ref, s.rhs, s.b, F, L["colour"], omega)
    assert np.allclose(x2, ref2, rtol=1e-10, atol=1e-10 * np.abs(ref2).max())


@pytest.mark.parametrize("kind,F", [("random6", 2), ("mhd", 2), ("random4", 1)])
@pytest.mark.parametrize("inner", [2, 3])
def test_bgs_inner_sweeps_equal_matrix_form(kind, F, inner):
    """inner_sweeps > 1: the Gauss-Seidel sub-solve iterates from its first sweep's
    result, the later colours' values taken from the previous sweep."""
    if kind == "random6":
        s = P.random_block_system(6, 6, [0, 0, 0, 1, 1, 1], seed=21)
    elif kind == "mhd":
        s = P.mhd2d(6, 2)
    else:
        s = P.random_block_system(5, 4, [0, 0, 0, 0], seed=22)
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, omega=0.6, inner_sweeps=inner)
    L = h.level(0)
    x0 = np.random.default_rng(6).standard_normal(s.n_unknowns)
    x1 = h.bgs(0, x0, s.rhs, 1)
    ref = bgs_matrix_form(s.dense(), x0, s.rhs, s.b, F, L["colour"], 0.6, inner)
    assert np.allclose(x1, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    one = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, omega=0.6, inner_sweeps=1)
    assert np.abs(one.bgs(0, x0, s.rhs, 1) - x1).max() > 1e-8  # the extra sweeps change the result


def test_bgs_many_inner_sweeps_solve_the_field_block():
    """Many inner sweeps on a block-diagonally dominant A_ff: the sub-solve
    converges to A_ff^-1 r_f, so the field step is x_f += omega A_ff^-1 r_f."""
    s = P.random_block_system(5, 6, [0, 0, 0, 1, 1, 1], seed=25, diag_shift=8.0)
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, omega=0.7, inner_sweeps=60)
    A, b, n = s.dense(), s.b, s.n_nodes
    x = np.random.default_rng(7).standard_normal(s.n_unknowns)
    got = h.bgs(0, x, s.rhs, 1)
    ref = x.copy()
    for f in range(2):
        rows = np.array([i * b + f * 3 + r for i in range(n) for r in range(3)])
        rf = s.rhs[rows] - A[rows, :] @ ref
        ref[rows] += 0.7 * np.linalg.solve(A[np.ix_(rows, rows)], rf)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_inner_sweeps_validation():
    s = P.random_block_system(4, 6, [0, 0, 0, 1, 1, 1], seed=26)
    for kw in (dict(inner_sweeps=65), dict(inner_sweeps=-1), dict(inner_sweeps=2, sub_ilu=2),
               dict(inner_sweeps=2, sub_schwarz=2)):
        with pytest.raises(oracle.OracleError):
            oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, **kw)


def test_bgs_block_diagonal_exact_with_unit_damping():
    s = P.random_block_system(5, 6, [0, 0, 0, 1, 1, 1], seed=23)
    s.vals[:, 3:, :3] = 0.0  # no A10 coupling
    s.vals[:, :3, 3:] = 0.0
    keep = np.zeros(s.nnzb, bool)
    for i in range(s.n_nodes):
        for k in range(s.row_ptr[i], s.row_ptr[i + 1]):
            keep[k] = s.col_idx[k] == i
    s.vals[~keep] = 0.0
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, omega=1.0)
    x = h.bgs(0, np.zeros(s.n_unknowns), s.rhs, 1)
    assert np.allclose(x, np.linalg.solve(s.dense(), s.rhs), rtol=1e-12, atol=1e-12)


def test_bgs_decoupled_fields_equal_separate_smoothers():
    s = P.random_block_system(6, 6, [0, 0, 0, 1, 1, 1], seed=24)
    s.vals[:, :3, 3:] = 0.0
    s.vals[:, 3:, :3] = 0.0
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0)
    x = h.bgs(0, np.zeros(s.n_unknowns), s.rhs, 1).reshape(-1, 6)
    for f in range(2):
        sub = P.BlockSystem("f", s.n_nodes, 3, s.row_ptr, s.col_idx,
                            np.ascontiguousarray(s.vals[:, 3 * f:3 * f + 3, 3 * f:3 * f + 3]),
                            s.rhs.reshape(-1, 6)[:, 3 * f:3 * f + 3].ravel(), [0, 0, 0], {})
        hf = oracle.Hierarchy.from_system(sub, max_levels=2, max_coarse=0)
        xf = hf.bgs(0, np.zeros(sub.n_unknowns), sub.rhs, 1).reshape(-1, 3)
        assert np.allclose(x[:, 3 * f:3 * f + 3], xf, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["poisson", "stokes"])
def test_smoother_reduces_error_monotonically(kind):
    s = P.poisson_block(16, 3) if kind == "poisson" else P.stokes2d(16, 1)
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0)
    xs = np.linalg.solve(s.dense(), s.rhs)
    x = np.zeros_like(s.rhs)
    errs = [np.linalg.norm(xs)]
    for _ in range(10):
        x = h.bgs(0, x, s.rhs, 1)
        errs.append(np.linalg.norm(x - xs))
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_vcycle_one_level_is_direct_solve():
    s = P.mhd2d(6, 4)
    h = oracle.Hierarchy.from_system(s, max_levels=1)
    assert h.num_levels == 1
    z = h.vcycle(s.rhs)
    assert np.allclose(z, np.linalg.solve(s.dense(), s.rhs), rtol=1e-9, atol=1e-12)


def test_vcycle_two_level_no_smoothing_is_coarse_correction():
    s = P.mhd2d(8, 5)
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, n_pre=0, n_post=0)
    L0 = h.level(0)
    Pm = tentative_P(L0["agg"], L0["n_agg"], s.b)
    A = s.dense()
    ref = Pm @ np.linalg.solve(Pm.T @ A @ Pm, Pm.T @ s.rhs)
    z = h.vcycle(s.rhs)
    assert np.allclose(z, ref, rtol=1e-9, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("kind", ["mhd", "stokes"])
def test_vcycle_matches_matrix_form(kind):
    s = P.mhd2d(8, 6) if kind == "mhd" else P.stokes2d(8, 6)
    F = 2 if kind == "mhd" else 1
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, n_pre=1, n_post=1, omega=0.5)
    L0 = h.level(0)
    Pm = tentative_P(L0["agg"], L0["n_agg"], s.b)
    A = s.dense()
    r = s.rhs
    u = bgs_matrix_form(A, np.zeros_like(r), r, s.b, F, L0["colour"], 0.5)
    uc = np.linalg.solve(Pm.T @ A @ Pm, Pm.T @ (r - A @ u))
    u = u + Pm @ uc
    u = bgs_matrix_form(A, u, r, s.b, F, L0["colour"], 0.5)
    z = h.vcycle(r)
    assert np.allclose(z, u, rtol=1e-9, atol=1e-10 * np.abs(u).max())


def test_vcycle_three_levels_matches_matrix_form():
    s = P.mhd2d(12, 7)
    h = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0)
    assert h.num_levels == 3
    L0, L1 = h.level(0), h.level(1)
    P0 = tentative_P(L0["agg"], L0["n_agg"], s.b)
    P1 = tentative_P(L1["agg"], L1["n_agg"], s.b)
    A0 = s.dense()
    A1 = P0.T @ A0 @ P0
    A2 = P1.T @ A1 @ P1

    def mgv(A, r, colour, Pl, below):
        u = bgs_matrix_form(A, np.zeros_like(r), r, s.b, 2, colour, 0.5)
        rc = Pl.T @ (r - A @ u)
        u = u + Pl @ below(rc)
        return bgs_matrix_form(A, u, r, s.b, 2, colour, 0.5)

    ref = mgv(A0, s.rhs, L0["colour"], P0,
              lambda rc: mgv(A1, rc, L1["colour"], P1, lambda rcc: np.linalg.solve(A2, rcc)))
    z = h.vcycle(s.rhs)
    assert np.allclose(z, ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())


# ----------------------------------------------------------------------------
# FGMRES
# ----------------------------------------------------------------------------


def test_fgmres_identity_is_krylov_minimal_residual():
    s = P.random_block_system(4, 3, [0, 0, 0], seed=31, diag_shift=0.3)
    h = oracle.Hierarchy.from_system(s, max_levels=1)
    A = s.dense()
    b = s.rhs
    for k in (1, 3, 7):
        x, it, rr, conv = h.fgmres(b, tol=1e-30, restart=50, max_iter=k, prec=1)
        assert it == k
        K = np.column_stack([np.linalg.matrix_power(A, p) @ b for p in range(k)])
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        xr = Q @ y
        assert np.allclose(x, xr, rtol=1e-8, atol=1e-10 * np.abs(xr).max())
        assert np.isclose(rr, np.linalg.norm(b - A @ xr) / np.linalg.norm(b), rtol=1e-6)


def test_fgmres_exact_preconditioner_one_iteration():
    s = P.mhd2d(6, 8)
    h = oracle.Hierarchy.from_system(s, max_levels=1)
    x, it, rr, conv = h.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=100)
    assert conv and it == 1 and rr <= 1e-8


def test_fgmres_restarted_dense_solution():
    s = P.stokes2d(8, 9)
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0)
    for restart in (3, 30):
        x, it, rr, conv = h.fgmres(s.rhs, tol=1e-10, restart=restart, max_iter=2000)
        xs = np.linalg.solve(s.dense(), s.rhs)
        assert conv and rr <= 1e-10
        assert np.linalg.norm(s.dense() @ x - s.rhs) / np.linalg.norm(s.rhs) <= 1e-10
        assert np.allclose(x, xs, rtol=1e-4, atol=1e-6 * np.abs(xs).max())


def test_fgmres_zero_rhs_and_initial_guess():
    s = P.stokes2d(4, 1)
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0)
    x, it, rr, conv = h.fgmres(np.zeros(s.n_unknowns))
    assert conv and it == 0 and np.all(x == 0)
    xs = np.linalg.solve(s.dense(), s.rhs)
    x, it, rr, conv = h.fgmres(s.rhs, x0=xs)
    assert conv and it == 0


# ----------------------------------------------------------------------------
# field blocks of unequal size (Algorithm 1 with fields of different widths)
# ----------------------------------------------------------------------------


def with_fields(s, fmap):
    return dataclasses.replace(s, field_of_dof=list(fmap))


UNEQUAL = {
    "random_b3_21": lambda: P.random_block_system(6, 3, [0, 0, 1], seed=31),
    "random_b5_32": lambda: P.random_block_system(5, 5, [0, 0, 0, 1, 1], seed=32),
    "random_b4_121": lambda: P.random_block_system(5, 4, [0, 1, 1, 2], seed=33),
    "stokes2d_u_p": lambda: with_fields(P.stokes2d(6, 3), [0, 0, 1]),
    "mhd2d_u_p_B_r": lambda: with_fields(P.mhd2d(6, 2), [0, 0, 1, 2, 2, 3]),
}


def padded(s):
    """The system with every field filled up to the widest field's size by
    dummy dofs: an identity diagonal entry in the node's diagonal block, no
    coupling, zero right-hand side.  Returns it and the padded index of every
    original unknown."""
    fmap = list(s.field_of_dof)
    F = max(fmap) + 1
    m = max(fmap.count(f) for f in range(F))
    bp = F * m
    pos = np.array([fmap[d] * m + d - fmap.index(fmap[d]) for d in range(s.b)])
    dummy = np.array([q for q in range(bp) if q not in set(pos.tolist())])
    V = np.zeros((s.nnzb, bp, bp))
    V[:, pos[:, None], pos[None, :]] = s.vals
    for i in range(s.n_nodes):
        for k in range(s.row_ptr[i], s.row_ptr[i + 1]):
            if s.col_idx[k] == i:
                V[k, dummy, dummy] = 1.0
    rhs = np.zeros((s.n_nodes, bp))
    rhs[:, pos] = s.rhs.reshape(s.n_nodes, s.b)
    real = (np.arange(s.n_nodes)[:, None] * bp + pos[None, :]).ravel()
    return dataclasses.replace(s, b=bp, vals=V, rhs=rhs.ravel(), field_of_dof=[q // m for q in range(bp)]), real


@pytest.mark.parametrize("name", list(UNEQUAL))
@pytest.mark.parametrize("inner", [1, 2])
def test_bgs_unequal_fields_equal_matrix_form(name, inner):
    s = UNEQUAL[name]()
    F = max(s.field_of_dof) + 1
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, omega=0.6, inner_sweeps=inner)
    L = h.level(0)
    x0 = np.random.default_rng(8).standard_normal(s.n_unknowns)
    got = h.bgs(0, x0, s.rhs, 1)
    ref = bgs_matrix_form(s.dense(), x0, s.rhs, s.b, F, L["colour"], 0.6, inner, fmap=s.field_of_dof)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("name", ["random_b4_121", "mhd2d_u_p_B_r"])
def test_unequal_fields_dinv_are_the_field_block_inverses(name):
    s = UNEQUAL[name]()
    F = max(s.field_of_dof) + 1
    h = oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0)
    dinv = h.level(0)["dinv"]
    assert isinstance(dinv, list) and len(dinv) == F
    V = s.vals
    for i in range(s.n_nodes):
        k = [k for k in range(s.row_ptr[i], s.row_ptr[i + 1]) if s.col_idx[k] == i][0]
        for f in range(F):
            dofs = [d for d in range(s.b) if s.field_of_dof[d] == f]
            want = np.linalg.inv(V[k][np.ix_(dofs, dofs)])
            assert np.allclose(dinv[f][i], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("name", list(UNEQUAL))
def test_unequal_fields_equal_the_padded_system(name):
    """Dummy dofs that are decoupled, with a zero right-hand side, stay zero in
    every step of the method (their residual, sub-solve, restriction and
    coarse solve are zero), so the V-cycle and FGMRES on the padded system with
    equal fields give the unpadded method's values."""
    s = UNEQUAL[name]()
    sp_, real = padded(s)
    kw = dict(max_levels=3, max_coarse=0, omega=0.55)
    h = oracle.Hierarchy.from_system(s, **kw)
    hp = oracle.Hierarchy.from_system(sp_, **kw)
    assert hp.num_levels == h.num_levels
    r = np.random.default_rng(12).standard_normal(s.n_unknowns)
    rp = np.zeros(sp_.n_unknowns)
    rp[real] = r
    z, zp = h.vcycle(r), hp.vcycle(rp)
    assert np.abs(zp[real] - z).max() <= 1e-13 * np.abs(z).max()
    mask = np.ones(sp_.n_unknowns, bool)
    mask[real] = False
    assert np.all(zp[mask] == 0.0)
    x, it, rr, _ = h.fgmres(s.rhs, tol=1e-8, restart=20, max_iter=300)
    xp, itp, rrp, _ = hp.fgmres(sp_.rhs, tol=1e-8, restart=20, max_iter=300)
    assert it == itp and abs(rr - rrp) <= 1e-12 * rr
    assert np.abs(xp[real] - x).max() <= 1e-10 * np.abs(x).max()


def test_unequal_fields_validation():
    s = UNEQUAL["random_b3_21"]()
    for kw in (dict(smooth_p=1), dict(sub_ilu=2), dict(sub_schwarz=2)):
        with pytest.raises(oracle.OracleError):
            oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, **kw)
    with pytest.raises(oracle.OracleError):
        oracle.Hierarchy.from_system(s, max_levels=2, max_coarse=0, mlp=np.zeros(oracle.MLP_NPARAMS))


def test_oracle_params_layout_matches_its_header(tmp_path):
    # the oracle binding's ctypes params against the C compiler's layout of
    # oracle_params: the same offsets and size
    import ctypes
    import subprocess
    fields = [name for name, _ in oracle.Params._fields_]
    src = tmp_path / "layout.c"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "bamg_oracle.h"', 'int main(void) {',
             '    printf("size %zu\\n", sizeof(oracle_params));']
    lines += ['    printf("%s %%zu\\n", offsetof(oracle_params, %s));' % (f, f) for f in fields]
    lines += ['    return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "oracle"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    assert int(got["size"]) == ctypes.sizeof(oracle.Params)
    for f in fields:
        assert int(got[f]) == getattr(oracle.Params, f).offset, f
