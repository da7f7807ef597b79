"""CPU checks behind the batched solver: the oracle run on a concatenated
(block-diagonal) batch gives, system by system, the hierarchy and the V-cycle
of the oracle run on each system alone (the greedy aggregation and colouring
never cross a system, the Galerkin product of a block-diagonal matrix is block
diagonal); and the batch generator's layout."""
import numpy as np

import oracle
from paper_2103_07537_gb300 import problems as P


def test_concatenate_layout():
    systems = [P.mhd2d(N, 7 + q) for q, N in enumerate([5, 9, 6])]
    bt = P.concatenate(systems)
    s = bt.system
    assert list(bt.sys_node_off) == [0, 36, 136, 185]
    assert s.nnzb == sum(m.nnzb for m in systems) and s.row_ptr[-1] == s.nnzb
    k0 = s.row_ptr[36]
    assert np.array_equal(s.col_idx[k0:k0 + systems[1].row_ptr[1]], systems[1].col_idx[:systems[1].row_ptr[1]] + 36)
    assert np.array_equal(s.rhs[36 * 6:136 * 6], systems[1].rhs)


def test_batch_sizes_range_and_determinism():
    a = P.batch_sizes(256, 1)
    assert a == P.batch_sizes(256, 1) and min(a) >= 16 and max(a) <= 160 and len(set(a)) > 50


def test_oracle_on_concatenation_is_per_system():
    systems = [P.mhd2d(N, 60 + q) for q, N in enumerate([16, 22, 17])]
    bt = P.concatenate(systems)
    kw = dict(max_levels=4, max_coarse=0)
    hb = oracle.Hierarchy.from_system(bt.system, **kw)
    hs = [oracle.Hierarchy.from_system(m, **kw) for m in systems]
    assert all(h.num_levels == hb.num_levels for h in hs)
    # level sizes add up; per-system structure is a diagonal block of the batch
    for l in range(hb.num_levels):
        Lb = hb.level(l)
        n0 = 0
        for h in hs:
            Ls = h.level(l)
            k0, k1 = Lb["row_ptr"][n0], Lb["row_ptr"][n0 + Ls["n"]]
            assert np.array_equal(Lb["col_idx"][k0:k1] - n0, Ls["col_idx"])
            assert np.array_equal(Lb["vals"][k0:k1], Ls["vals"])
            if l < hb.num_levels - 1:
                assert np.array_equal(Lb["colour"][n0:n0 + Ls["n"]], Ls["colour"])
            n0 += Ls["n"]
        assert n0 == Lb["n"]
    r = np.random.default_rng(0).standard_normal(bt.system.n_unknowns)
    zb = hb.vcycle(r)
    off = bt.sys_node_off * 6
    for q, h in enumerate(hs):
        zq = h.vcycle(r[off[q]:off[q + 1]])
        assert np.allclose(zb[off[q]:off[q + 1]], zq, rtol=1e-9, atol=1e-9 * np.abs(zq).max())
