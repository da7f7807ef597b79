"""Pins of the oracle's Schwarz sub-solve of Algorithm 1 (Sec. 5: one
additive Schwarz iteration with overlap one approximates each field block's
inverse).  CPU only.

Facts used, none of them from the oracle's Schwarz code: the subdomains are
rebuilt here from the level's aggregates and a scipy graph of the field
block; the sub-solve is then written with dense numpy solves
(x~ = sum_I R_I^T A_I^{-1} R_I r, or the restricted sum); closed forms when
every field is one subdomain; symmetry and definiteness of the additive
operator of a symmetric positive definite matrix.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2103_07537_gb300 import problems as P
from test_oracle_fields import two_field_system
from test_oracle_pins import bsr_dense


def field_blocks(n, b, field_of_dof, node_field_off):
    """[(nodes of the field, first dof, dofs per node)] for every field block."""
    if node_field_off is not None:
        return [(np.arange(node_field_off[g], node_field_off[g + 1]), 0, b)
                for g in range(len(node_field_off) - 1)]
    F = max(field_of_dof) + 1
    fb = b // F
    return [(np.arange(n), f * fb, fb) for f in range(F)]


def schwarz_matrix_form(A, x, rhs, b, agg, rp, ci, blocks, omega, overlap, restricted):
    """One sweep of Algorithm 1 with the Schwarz sub-solve, dense.

    Field (nodes, f0, fb): r = rhs - A x on its rows; subdomain I = the field's
    nodes of aggregate I plus, with overlap, their neighbours of the same
    field; A_I = the field block restricted to the subdomain; x~ = sum over
    subdomains of the local solution (restricted: only on the aggregate's own
    nodes); x += omega x~ on the field's rows.
    """
    x = x.copy()
    n = len(agg)
    G = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n)).tolil()
    for nodes, f0, fb in blocks:
        in_field = np.zeros(n, bool)
        in_field[nodes] = True
        rows = np.array([i * b + f0 + r for i in nodes for r in range(fb)])
        pos = {i: t for t, i in enumerate(nodes)}
        r_f = rhs[rows] - A[rows, :] @ x
        Aff = A[np.ix_(rows, rows)]
        xt = np.zeros_like(r_f)
        for I in sorted(set(agg[nodes].tolist())):
            own = [i for i in nodes if agg[i] == I]
            S = set(own)
            if overlap:
                for i in own:
                    S |= {j for j in G.rows[i] if in_field[j]}
            S = sorted(S)
            idx = np.array([pos[i] * fb + r for i in S for r in range(fb)])
            y = np.linalg.solve(Aff[np.ix_(idx, idx)], r_f[idx])
            for t, i in enumerate(S):
                if restricted and agg[i] != I:
                    continue
                xt[pos[i] * fb:(pos[i] + 1) * fb] += y[t * fb:(t + 1) * fb]
        x[rows] += omega * xt
    return x


CASES = {
    "mhd2d_5": lambda: (lambda s: (s.row_ptr, s.col_idx, s.vals, s.field_of_dof, None, s.rhs))(P.mhd2d(5, 2)),
    "q2q1_3": lambda: (lambda s: (s.row_ptr, s.col_idx, s.vals, [0, 0, 0], s.node_field_off, s.rhs))(
        P.mhd2d_q2q1(3, 4)),
    "random_two_field_b2": lambda: (lambda t: (t[0], t[1], t[2], [0, 0], t[3],
                                               P.uniform_pm1(5, 0, (len(t[0]) - 1) * 2)))(
        two_field_system(14, 11, 2, 3, 0.3, 0.15)),
}


@pytest.mark.parametrize("overlap", [0, 1])
@pytest.mark.parametrize("restricted", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_schwarz_sweep_equals_matrix_form(case, restricted, overlap):
    rp, ci, vals, fmap, foff, rhs = CASES[case]()
    b = vals.shape[1]
    om = 0.6
    h = oracle.Hierarchy(rp, ci, vals, b, fmap, max_levels=2, max_coarse=0, omega=om, node_field_off=foff,
                         sub_schwarz=2 if restricted else 1, schwarz_overlap=overlap)
    agg = h.level(0)["agg"]
    A = bsr_dense(rp, ci, vals)
    x0 = P.uniform_pm1(23, 0, len(rhs))
    blocks = field_blocks(len(rp) - 1, b, fmap, foff)
    ref = schwarz_matrix_form(A, x0, rhs, b, agg, rp, ci, blocks, om, overlap, restricted)
    assert np.allclose(h.bgs(0, x0, rhs, sweeps=1), ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())
    if overlap == 0:  # without overlap both forms are block Jacobi over the aggregates
        h2 = oracle.Hierarchy(rp, ci, vals, b, fmap, max_levels=2, max_coarse=0, omega=om, node_field_off=foff,
                              sub_schwarz=1 if restricted else 2, schwarz_overlap=0)
        assert np.array_equal(h.bgs(0, x0, rhs, sweeps=1), h2.bgs(0, x0, rhs, sweeps=1))


def test_one_subdomain_per_field_is_block_gauss_seidel_with_exact_solves():
    # complete graph inside each field: one aggregate (one subdomain) per
    # field, so with omega = 1 one sweep is x_0 = A00^{-1} b_0,
    # x_1 = A11^{-1} (b_1 - A10 x_0)
    rp, ci, vals, foff = two_field_system(7, 5, 2, 9, p_in=1.0, p_cross=0.4)
    rhs = P.uniform_pm1(3, 0, 24)
    A = bsr_dense(rp, ci, vals)
    for form in (1, 2):
        h = oracle.Hierarchy(rp, ci, vals, 2, [0, 0], max_levels=2, max_coarse=0, omega=1.0, node_field_off=foff,
                             sub_schwarz=form, schwarz_overlap=1)
        assert h.level(0)["n_agg"] == 2
        x = h.bgs(0, np.zeros(24), rhs, sweeps=1)
        x0 = np.linalg.solve(A[:14, :14], rhs[:14])
        x1 = np.linalg.solve(A[14:, 14:], rhs[14:] - A[14:, :14] @ x0)
        assert np.allclose(x, np.concatenate([x0, x1]), rtol=1e-12, atol=1e-13)


def test_additive_operator_is_symmetric_positive_definite():
    # for SPD A the additive Schwarz operator sum_I R_I^T A_I^{-1} R_I is SPD;
    # with omega = 1, one field and x = 0 one sweep applies it to the rhs
    s = P.poisson_block(5, 1)
    n = s.n_nodes
    h = oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, 1, [0], max_levels=2, max_coarse=0, omega=1.0,
                         sub_schwarz=1, schwarz_overlap=1)
    M = np.stack([h.bgs(0, np.zeros(n), np.eye(n)[k], sweeps=1) for k in range(n)], axis=1)
    assert np.allclose(M, M.T, rtol=1e-12, atol=1e-14)
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    # the restricted form is not symmetric on the same subdomains
    hr = oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, 1, [0], max_levels=2, max_coarse=0, omega=1.0,
                          sub_schwarz=2, schwarz_overlap=1)
    Mr = np.stack([hr.bgs(0, np.zeros(n), np.eye(n)[k], sweeps=1) for k in range(n)], axis=1)
    assert not np.allclose(Mr, Mr.T)


def test_restricted_schwarz_is_the_working_reading():
    # measured facts behind the reading of the paper's "additive Schwarz with
    # overlap one" (Sec. 5): the plain sum of overlapping corrections does not
    # converge as a damped sub-solve here, the restricted form converges in
    # fewer iterations than the multicolour sweep
    s = P.mhd2d_q2q1(16, 1)
    its = {}
    for lab, kw in (("sweep", {}), ("ras", dict(sub_schwarz=2)), ("as", dict(sub_schwarz=1))):
        h = oracle.Hierarchy.from_system(s, max_levels=4, max_coarse=0, omega=0.6, **kw)
        _, it, rr, ok = h.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=400)
        its[lab] = it if ok else None
    assert its["as"] is None
    assert its["ras"] is not None and its["sweep"] is not None and its["ras"] * 3 < its["sweep"]


def test_schwarz_validation():
    s = P.mhd2d(4, 1)
    args = (s.row_ptr, s.col_idx, s.vals, s.b, s.field_of_dof)
    for kw in (dict(sub_schwarz=3), dict(sub_schwarz=1, schwarz_overlap=2), dict(sub_schwarz=1, sub_ilu=1),
               dict(sub_schwarz=-1)):
        with pytest.raises(oracle.OracleError):
            oracle.Hierarchy(*args, max_levels=2, max_coarse=0, **kw)
