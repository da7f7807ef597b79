"""Field blocks of unequal size (velocity | pressure, the four MHD fields
u | p | B | r, random maps) on the GPU against the oracle, which runs
Algorithm 1 with fields of different widths directly.

The library runs such a system padded (every field filled up to the widest
with decoupled dummy dofs); the oracle does not pad.  Bars: the node-level
hierarchy (aggregates, colours) bit for bit; the given dofs' entries of every
level's matrix bit for bit (the tentative Galerkin product sums the same
values in the same order) and the dummy entries off their diagonal zero; the
per-field inverse blocks within 1e-12; the FP64 V-cycle within 1e-12; FGMRES
iterations within +-1 at 1e-8.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def with_fields(s, fmap):
    return dataclasses.replace(s, field_of_dof=list(fmap))


SYSTEMS = {
    "stokes2d_u_p": lambda: (with_fields(P.stokes2d(24, 1), [0, 0, 1]), dict(max_levels=3, max_coarse=0)),
    "mhd2d_u_p_B_r": lambda: (with_fields(P.mhd2d(20, 2), [0, 0, 1, 2, 2, 3]), dict(max_levels=3, max_coarse=0)),
    "stokes3d_u_p": lambda: (with_fields(P.stokes3d(8, 1), [0, 0, 0, 1]), dict(max_levels=3, max_coarse=0)),
    "random_b3_21": lambda: (P.random_block_system(30, 3, [0, 0, 1], seed=31), dict(max_levels=4, max_coarse=0)),
    "random_b5_32": lambda: (P.random_block_system(25, 5, [0, 0, 0, 1, 1], seed=32),
                             dict(max_levels=4, max_coarse=0)),
    "random_b4_121": lambda: (P.random_block_system(25, 4, [0, 1, 1, 2], seed=33), dict(max_levels=4, max_coarse=0)),
    "random_b7_43": lambda: (P.random_block_system(12, 7, [0, 0, 0, 0, 1, 1, 1], seed=34),
                             dict(max_levels=3, max_coarse=0)),
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


def rel_max(a, ref):
    scale = np.abs(ref).max()
    return np.abs(a - ref).max() / (scale if scale > 0 else 1.0)


def padded_places(fmap):
    """Padded dof of every given dof: field f's dofs fill places 0.. of field f's
    fmax-wide slot."""
    F = max(fmap) + 1
    m = max(list(fmap).count(f) for f in range(F))
    return np.array([fmap[d] * m + d - list(fmap).index(fmap[d]) for d in range(len(fmap))]), F * m, m


def apply(g, r):
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    g.apply(dev(r), z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_unequal_hierarchy_matches_oracle(name):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, **kw)
    o = oracle.Hierarchy.from_system(s, **kw)
    pos, bp, m = padded_places(s.field_of_dof)
    st = g.stats()
    assert st["padded"] == 1 and st["b"] == bp and st["b_given"] == s.b
    assert bamg.amg_block_size(g.handle) == bp
    assert g.num_levels == o.num_levels
    dummy = np.array([q for q in range(bp) if q not in set(pos.tolist())])
    F = max(s.field_of_dof) + 1
    for l in range(g.num_levels):
        Lg, Lo = g.level(l), o.level(l)
        assert np.array_equal(Lg["row_ptr"], Lo["row_ptr"]) and np.array_equal(Lg["col_idx"], Lo["col_idx"])
        assert np.array_equal(Lg["vals"][:, pos[:, None], pos[None, :]], Lo["vals"]), l
        off = Lg["vals"][:, dummy[:, None], np.arange(bp)[None, :]].copy()
        for t, q in enumerate(dummy):
            off[:, t, q] = 0.0  # the dummy's own diagonal entry
        assert not off.any() and not Lg["vals"][:, :, dummy][:, pos, :].any()
        if l < g.num_levels - 1:
            assert np.array_equal(Lg["agg"], Lo["agg"]) and np.array_equal(Lg["colour"], Lo["colour"])
            for f in range(F):
                dofs = [d for d in range(s.b) if s.field_of_dof[d] == f]
                places = pos[dofs] - f * m
                got = Lg["dinv"][:, f][:, places[:, None], places[None, :]]
                assert rel_max(got, Lo["dinv"][f]) <= 1e-12, (l, f)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_unequal_vcycle_fp64_matches_oracle(name):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, **kw)
    o = oracle.Hierarchy.from_system(s, **kw)
    r = np.random.default_rng(13).standard_normal(s.n_unknowns)
    assert rel_max(apply(g, r), o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("variant", [dict(n_pre=2, n_post=1, omega=0.7), dict(inner_sweeps=3),
                                     dict(use_graph=0, use_pdl=0), dict(autotune=4)])
def test_unequal_cycle_variants_match_oracle(variant):
    s, kw = SYSTEMS["random_b4_121"]()
    kw = dict(kw, **variant)
    okw = {k: v for k, v in kw.items() if k not in ("use_graph", "use_pdl", "autotune")}
    g = make_solver(s, **kw)
    o = oracle.Hierarchy.from_system(s, **okw)
    assert rel_max(apply(g, s.rhs), o.vcycle(s.rhs)) <= 1e-12


@pytest.mark.parametrize("name", ["stokes2d_u_p", "mhd2d_u_p_B_r", "stokes3d_u_p", "random_b5_32"])
def test_unequal_fgmres_iterations_match_oracle(name):
    s, kw = SYSTEMS[name]()
    g = make_solver(s, **kw)
    o = oracle.Hierarchy.from_system(s, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=600)
    _, it_o, _, _ = o.fgmres(s.rhs, tol=1e-8, restart=30, max_iter=600)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    assert abs(it - it_o) <= 1, (it, it_o)
    res = s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(s.rhs) <= 1e-8


def test_unequal_fp32_cycle_and_host_entry_point():
    s = with_fields(P.mhd2d(48, 3), [0, 0, 1, 2, 2, 3])
    kw = dict(max_levels=4, max_coarse=0, cycle_prec=32)
    g = make_solver(s, **kw)
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, it, rr = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=600)
    assert st == bamg.BAMG_OK and rr <= 1e-8
    res = s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(s.rhs) <= 1e-8
    # the same setup and solve from host buffers (padding inside the library)
    xh = np.zeros(s.n_unknowns)
    st_h, it_h, rr_h = bamg.amg_solve_host(s.row_ptr, s.col_idx, np.ascontiguousarray(s.vals.reshape(-1)),
                                           s.n_nodes, s.nnzb, s.b, s.field_of_dof, s.rhs, xh, tol=1e-8,
                                           restart=30, max_iter=600, params=bamg.amg_default_params(**kw))
    assert st_h == bamg.BAMG_OK and abs(it_h - it) <= 1 and rr_h <= 1e-8
    assert rel_max(xh, x.cpu().numpy()) <= 1e-6


def test_unequal_batch_matches_each_system_alone():
    members = [with_fields(P.stokes2d(N, 1), [0, 0, 1]) for N in (14, 22, 18)]
    bt = P.concatenate(members)
    s = bt.system
    kw = dict(max_levels=3, max_coarse=0)
    g = bamg.BatchSolver(bt.sys_node_off, dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), s.b,
                         s.field_of_dof, **kw)
    r = np.random.default_rng(17).standard_normal(s.n_unknowns)
    zg = apply(g, r)
    off = bt.sys_node_off * s.b
    compared = 0
    for q, m in enumerate(bt.members):
        o = oracle.Hierarchy.from_system(m, **kw)
        if o.num_levels != g.num_levels:
            continue
        assert rel_max(zg[off[q]:off[q + 1]], o.vcycle(r[off[q]:off[q + 1]])) <= 1e-12, q
        compared += 1
    assert compared >= 2
    x = torch.zeros(s.n_unknowns, dtype=torch.float64, device="cuda")
    st, its, rrs = g.solve(dev(s.rhs), x, tol=1e-8, restart=30, max_iter=600)
    assert st == bamg.BAMG_OK and max(rrs) <= 1e-8
    res = s.rhs - oracle.spmv(s.row_ptr, s.col_idx, s.vals, x.cpu().numpy())
    for q in range(len(bt.members)):
        seg = slice(off[q], off[q + 1])
        assert np.linalg.norm(res[seg]) / np.linalg.norm(s.rhs[seg]) <= 1e-8, q


@pytest.mark.parametrize("fmap,kw,status", [
    ([0, 0, 1], dict(smooth_p=1), bamg.BAMG_EUNSUPPORTED),
    ([0, 0, 1], dict(sub_solver=1), bamg.BAMG_EUNSUPPORTED),
    ([0, 0, 1], dict(sub_solver=2), bamg.BAMG_EUNSUPPORTED),
    ([0, 0, 0, 1, 1, 1, 2], {}, bamg.BAMG_EUNSUPPORTED),  # padded to 9 dofs
    ([1, 1, 0], {}, bamg.BAMG_EINVAL),
    ([0, 0, 2], {}, bamg.BAMG_EINVAL),
])
def test_unequal_fields_refused(fmap, kw, status):
    b = len(fmap)
    s = P.random_block_system(6, b, [d * 0 for d in range(b)], seed=40)
    with pytest.raises(bamg.BamgError) as e:
        bamg.Solver(dev(s.row_ptr), dev(s.col_idx), dev(s.vals.reshape(-1)), b, fmap, max_levels=2,
                    max_coarse=0, **kw)
    assert e.value.status == status
