"""Writes oracle/solve_counts.json: the inner FGMRES step count and the true
relative residual of one full oracle solve (setup + FGMRES to 1e-8) of every
single-system bench workload, seed 1.

The bench's reference arm times the oracle on a bounded sample (setup plus a
few inner steps) and scales it to one full solve by this count, so that a
3D solve of about two minutes need not run inside the timed arm.  Only the
oracle computes these numbers (the workload generators are the shared input
code); run `python oracle/make_solve_counts.py [workload ...]` after any change
of the oracle's arithmetic or of a workload.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "solve_counts.json")


def main(argv):
    sys.path.insert(0, ROOT)
    import bench

    names = argv or [k for k, wl in bench.WORKLOADS.items() if not wl.get("batched")]
    counts = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        wl = bench.WORKLOADS[name]
        s = wl["make"](1)
        t0 = time.perf_counter()
        full = bench.oracle_full_solve(s, wl)
        counts[name] = {"seed": 1, "iterations": int(full["iters"]), "relres": float(full["relres"]),
                        "converged": bool(full["converged"]), "restart": wl["restart"],
                        "oracle_seconds_here": round(time.perf_counter() - t0, 1)}
        print(name, counts[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(counts, f, indent=1, sort_keys=True)
            f.write("\n")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
