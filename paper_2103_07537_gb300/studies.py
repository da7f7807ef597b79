"""Smoother studies on the GPU solver: sweeps x damping, and field-split
against fully coupled node-block smoothing.

Sec. 5 of the paper varies the number of block Gauss-Seidel sweeps and the
damping omega of Algorithm 1 (iterations against omega for 1, 2 and 3
sweeps; damping near 0.5 works, more sweeps lower the iteration count but
not necessarily the time), and compares the field-split smoother with a
fully coupled one applied to the whole system (found two to three times
slower there).

``sweeps``: every (sweeps, omega) pair on the same systems, sweeps = n_pre =
n_post of the V(n_pre, n_post)-cycle.

``coupling``: on the same hierarchy (the aggregation and the tentative
prolongator do not depend on how the dofs of a node are split into fields),
the field-split smoother (field map of the system, F fields, fb x fb
diagonal sub-blocks inverted) against node-block Gauss-Seidel over the whole
b x b block (field map all zero, F = 1), each at the dampings given.  This is
the fully coupled smoother of the same multicolour kind, not the paper's
FC-AMG with ILU or Schwarz sub-solves.

Each record: FGMRES iterations to tol, setup ms, solve ms and V-cycle ms
(median of 20 graph replays), all CUDA-event times on the launching stream.

Run ``python -m paper_2103_07537_gb300.studies sweeps --N 128 --seeds 1-4`` on
a GPU.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

from . import bamg
from . import problems as P

SWEEPS = (1, 2, 3)
OMEGAS = (0.4, 0.5, 0.6, 1.0)


def parse_seeds(text: str) -> list:
    """"a-b" -> [a..b]; "a,b,c" -> [a, b, c]; "a" -> [a]."""
    out = []
    for part in text.split(","):
        part = part.strip()
        if "-" in part:
            a, b = (int(v) for v in part.split("-"))
            if b < a:
                raise ValueError(f"empty seed range {part!r}")
            out.extend(range(a, b + 1))
        elif part:
            out.append(int(part))
    if not out:
        raise ValueError("no seeds")
    return out


def coupled_field_map(b: int) -> list:
    """Field map of the fully coupled smoother: every dof in field 0."""
    return [0] * b


def sweep_grid(sweeps=SWEEPS, omegas=OMEGAS) -> list:
    """The (n_pre, n_post, omega) settings of the sweeps study, in order."""
    return [dict(n_pre=int(k), n_post=int(k), omega=float(w)) for k in sweeps for w in omegas]


def coupling_grid(split_map, omegas_split=(0.5,), omegas_coupled=(0.5, 1.0)) -> list:
    """The (field map, omega) settings of the coupling study."""
    b = len(split_map)
    rows = [dict(smoother="field-split", field_of_dof=list(split_map), omega=float(w)) for w in omegas_split]
    rows += [dict(smoother="coupled", field_of_dof=coupled_field_map(b), omega=float(w)) for w in omegas_coupled]
    return rows


def run_one(torch, s, field_of_dof, prm, tol, restart, max_iter, replays=20):
    """Setup, solve and V-cycle replays of one system with one setting."""
    dev = torch.device("cuda")
    rp = torch.from_numpy(s.row_ptr).to(dev)
    ci = torch.from_numpy(s.col_idx).to(dev)
    va = torch.from_numpy(np.ascontiguousarray(s.vals.reshape(-1))).to(dev)
    b = torch.from_numpy(s.rhs).to(dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream(dev)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    e0, e1, e2 = ev(), ev(), ev()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    h = bamg.amg_setup(rp, ci, va, s.n_nodes, s.nnzb, s.b, field_of_dof, prm, stream)
    try:
        e1.record(stream)
        st, it, rr = bamg.fgmres_solve(h, b, x, tol, restart, max_iter, stream)
        e2.record(stream)
        e2.synchronize()
        r = b.clone()
        z = torch.empty_like(b)
        for _ in range(3):
            bamg.amg_apply(h, r, z, stream)
        vt = []
        for _ in range(replays):
            a0, a1 = ev(), ev()
            a0.record(stream)
            bamg.amg_apply(h, r, z, stream)
            a1.record(stream)
            a1.synchronize()
            vt.append(a0.elapsed_time(a1))
    finally:
        bamg.amg_destroy(h)
    return dict(iterations=int(it), converged=st == bamg.BAMG_OK, relres=float(rr),
                setup_ms=float(e0.elapsed_time(e1)), solve_ms=float(e1.elapsed_time(e2)),
                vcycle_ms=float(statistics.median(vt)))


def study(kind, N, seeds, cycle_prec=64, levels=4, max_coarse=0, restart=30, max_iter=3000, tol=1e-8,
          log=print):
    """All settings of one study on mhd2d(N, seed) for every seed; one record
    per (setting, seed)."""
    import torch

    out = []
    for q in seeds:
        s = P.mhd2d(N, q)
        grid = sweep_grid() if kind == "sweeps" else coupling_grid(s.field_of_dof)
        for g in grid:
            fm = g.get("field_of_dof", s.field_of_dof)
            prm = bamg.amg_default_params(max_levels=levels, max_coarse=max_coarse, cycle_prec=cycle_prec,
                                          n_pre=g.get("n_pre", 1), n_post=g.get("n_post", 1), omega=g["omega"])
            rec = dict(study=kind, N=int(N), seed=int(q), cycle_prec=int(cycle_prec),
                       **{k: v for k, v in g.items() if k != "field_of_dof"}, F=int(max(fm)) + 1)
            rec.update(run_one(torch, s, fm, prm, tol, restart, max_iter))
            out.append(rec)
            log(json.dumps(rec))
    return out


def summarise(records, keys):
    """Mean iterations and median times per setting over the seeds."""
    groups = {}
    for r in records:
        groups.setdefault(tuple(r[k] for k in keys), []).append(r)
    rows = []
    for k, rs in groups.items():
        rows.append(dict(zip(keys, k), seeds=len(rs), converged=all(r["converged"] for r in rs),
                         iterations=float(np.mean([r["iterations"] for r in rs])),
                         setup_ms=float(statistics.median(r["setup_ms"] for r in rs)),
                         solve_ms=float(statistics.median(r["solve_ms"] for r in rs)),
                         vcycle_ms=float(statistics.median(r["vcycle_ms"] for r in rs))))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("kind", choices=["sweeps", "coupling"])
    ap.add_argument("--N", type=int, default=128, help="cells per side of mhd2d")
    ap.add_argument("--seeds", default="1-4")
    ap.add_argument("--cycle-prec", type=int, default=64, choices=[32, 64])
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--out", default=None, help="write the records and the summary as JSON")
    args = ap.parse_args(argv)
    import torch

    torch.cuda.set_device(0)
    bamg.load()
    recs = study(args.kind, args.N, parse_seeds(args.seeds), cycle_prec=args.cycle_prec, levels=args.levels)
    keys = ["n_pre", "omega"] if args.kind == "sweeps" else ["smoother", "omega"]
    summ = summarise(recs, keys)
    for row in summ:
        print(json.dumps(row))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(dict(records=recs, summary=summ), f, indent=1)


if __name__ == "__main__":
    main()
