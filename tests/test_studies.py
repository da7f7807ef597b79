"""Smoother studies (sweeps x damping; field-split against fully coupled
node-block smoothing, Sec. 5): host logic and oracle properties on the CPU,
the study runner and its iteration counts against the oracle on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import problems as P
from paper_2103_07537_gb300 import studies


def test_parse_seeds():
    assert studies.parse_seeds("1-4") == [1, 2, 3, 4]
    assert studies.parse_seeds("3") == [3]
    assert studies.parse_seeds("1,5-6, 9") == [1, 5, 6, 9]
    for bad in ("", "4-2", " , "):
        with pytest.raises(ValueError):
            studies.parse_seeds(bad)


def test_grids():
    g = studies.sweep_grid()
    assert len(g) == len(studies.SWEEPS) * len(studies.OMEGAS)
    assert g[0] == dict(n_pre=1, n_post=1, omega=0.4) and g[-1] == dict(n_pre=3, n_post=3, omega=1.0)
    c = studies.coupling_grid([0, 0, 0, 1, 1, 1])
    assert [r["smoother"] for r in c] == ["field-split", "coupled", "coupled"]
    assert c[0]["field_of_dof"] == [0, 0, 0, 1, 1, 1] and c[1]["field_of_dof"] == [0] * 6
    assert [r["omega"] for r in c] == [0.5, 0.5, 1.0]


def test_summarise():
    recs = [dict(n_pre=1, omega=0.5, iterations=10, converged=True, setup_ms=1.0, solve_ms=4.0, vcycle_ms=0.1),
            dict(n_pre=1, omega=0.5, iterations=12, converged=True, setup_ms=3.0, solve_ms=2.0, vcycle_ms=0.3),
            dict(n_pre=2, omega=0.5, iterations=7, converged=False, setup_ms=2.0, solve_ms=5.0, vcycle_ms=0.2)]
    rows = studies.summarise(recs, ["n_pre", "omega"])
    assert rows[0] == dict(n_pre=1, omega=0.5, seeds=2, converged=True, iterations=11.0, setup_ms=2.0,
                           solve_ms=3.0, vcycle_ms=0.2)
    assert rows[1]["seeds"] == 1 and rows[1]["converged"] is False


def test_coupled_smoother_keeps_the_hierarchy():
    # cloned aggregation and the tentative prolongator ignore the field split
    # (Sec. 4.3.1): the coarse operators of the two smoothers are identical
    s = P.mhd2d(12, 1)
    kw = dict(max_levels=3, max_coarse=0)
    hs = oracle.Hierarchy.from_system(s, **kw)
    hc = oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, s.b, studies.coupled_field_map(s.b), **kw)
    assert hs.num_levels == hc.num_levels == 3
    for l in range(3):
        a, c = hs.level(l), hc.level(l)
        for k in ("row_ptr", "col_idx", "vals"):
            assert np.array_equal(a[k], c[k])
        if l < 2:
            assert np.array_equal(a["agg"], c["agg"]) and np.array_equal(a["colour"], c["colour"])
            # the coupled sub-solve inverts the whole diagonal block
            rp, ci, v = c["row_ptr"], c["col_idx"], c["vals"]
            for i in range(0, c["n"], 7):
                k = rp[i] + int(np.nonzero(ci[rp[i]:rp[i + 1]] == i)[0][0])
                assert np.allclose(c["dinv"][i, 0] @ v[k], np.eye(s.b), atol=1e-10)


def test_more_sweeps_fewer_iterations_oracle():
    # Sec. 5: more block Gauss-Seidel sweeps lower the iteration count
    s = P.mhd2d(16, 1)
    its = []
    for k in (1, 2, 3):
        h = oracle.Hierarchy.from_system(s, max_levels=3, max_coarse=0, n_pre=k, n_post=k, omega=0.5)
        _, it, rr, ok = h.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=600)
        assert ok and rr <= 1e-8
        its.append(it)
    assert its[0] > its[1] >= its[2]


@pytest.mark.gpu
def test_studies_run_and_match_oracle_iterations():
    s = P.mhd2d(16, 1)
    for kind in ("sweeps", "coupling"):
        recs = studies.study(kind, 16, [1], cycle_prec=64, levels=3, max_iter=600, log=lambda *_: None)
        # omega = 1 stalls (one undamped sweep per field from zero): the
        # iteration limit is reached on both sides
        assert all(r["converged"] for r in recs if r["omega"] < 1.0)
        for r in recs:
            if kind == "sweeps" and r["omega"] not in (0.5, 1.0):
                continue
            fm = s.field_of_dof if kind == "sweeps" or r["smoother"] == "field-split" \
                else studies.coupled_field_map(s.b)
            h = oracle.Hierarchy(s.row_ptr, s.col_idx, s.vals, s.b, fm, max_levels=3, max_coarse=0,
                                 n_pre=r.get("n_pre", 1), n_post=r.get("n_post", 1), omega=r["omega"])
            _, it, _, ok = h.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=600)
            assert ok == r["converged"] and abs(it - r["iterations"]) <= 1, (r, it)
        assert all(r["vcycle_ms"] > 0 and r["setup_ms"] > 0 for r in recs)
