#!/usr/bin/env python
"""Benchmark of the block-AMG-preconditioned FGMRES solve on one GB300.

Workload (default ``stokes3d_64``): the 3D Stokes-type system, Q1-Q1 with
pressure stabilisation on a 64^3 hex grid, 4 dofs per node (u, v, w, p),
274,625 nodes, 1,098,500 unknowns, 7,189,057 stored 4 x 4 blocks (115 M
scalars, far larger than L2); FP32 V(1,1) cycle of damped block Gauss-Seidel
(omega 0.5) with an FP32 LU of the 2048-unknown coarsest level, inside FP64
FGMRES(50) to a relative residual of 1e-8 (FP64 outer SpMV, Arnoldi and
residual test).  The line also carries the FP64 cycle and the FP32 cycle with
a smoothed prolongator whose P and R values are stored in FP32 or in BF16,
each with its own solve rate and true FP64 residual.  Synthetic seeded data
(the paper's MHD systems are not available).  The other workloads (the 2D
systems, the batch of 256, the learned 256^2 system, mixed elements) are
selected with --workload.

One step = one complete solve from the matrix already in HBM: hierarchy setup
(aggregation, colouring, Galerkin products, block inverses, coarse LU),
FGMRES with the V-cycle preconditioner to 1e-8, and release of the
hierarchy.  value = converged solves per second over all ranks: one
independent system per rank (weak scaling), or, for the batch workload, the
systems of the one batch split over the ranks by a longest-processing-time
partition on stored blocks (strong scaling); no collective on the data path,
only the max of the timed regions and the sum of converged systems.  L2 is
flushed between steps (a 256 MiB write, outside the timed step).

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "V-cycle ms & solves/s to 1e-8 rel. residual (FP64 vs mixed/learned); HBM GB/s"
UNIT = "solves/s"
TOL = 1e-8
MAX_ITER = 5000
FLUSH_BYTES = 256 << 20
PR_OMEGA_P = 0.1  # prolongator smoothing weight of the smoothed-P variants
FALLBACK_HBM_GBS = 6800.0
SMS = 152

WORKLOADS = {
    "mhd2d_128": dict(
        make=lambda seed: __import__("paper_2103_07537_gb300.problems", fromlist=["x"]).mhd2d(128, seed),
        levels=4, max_coarse=0, restart=30, prec=64, sub_solver_variants=True,
        desc="2D coupled 4-field Q1 system (u,v,p | Bx,By,psi), 128x128 cells, 6 dofs/node, 99,846 unknowns, "
             "148,225 blocks, nu/eta log-U[1e-3,1], FP64 V(1,1) BGS omega=0.5, 4 levels, FGMRES(30) to 1e-8"),
    "stokes2d_32": dict(
        make=lambda seed: __import__("paper_2103_07537_gb300.problems", fromlist=["x"]).stokes2d(32, seed),
        levels=3, max_coarse=0, restart=30, prec=64,
        desc="2D Stokes Q1-Q1 stabilised, 32x32 cells, 3 dofs/node, 3,267 unknowns, FP64, 3 levels, "
             "FGMRES(30) to 1e-8"),
    "mhd2d_batch256": dict(
        make=lambda seed: __import__("paper_2103_07537_gb300.problems", fromlist=["x"]).mhd2d_batch(256, seed),
        levels=4, max_coarse=0, restart=30, prec=32, batched=True, max_iter=400,
        desc="batch of 256 independent 2D 4-field Q1 systems, cells per side uniform in 16..160 (about 2.0 M "
             "nodes, 12 M unknowns), coefficients as the 2D 4-field workload, one block-diagonal operator "
             "(every V-cycle step one launch over all systems, replayed from a CUDA graph), FP32 V(1,1) "
             "inside per-system FP64 FGMRES(30) to 1e-8, at most 400 inner steps per system"),
    "mhd2d_cells_256": dict(
        make=lambda seed: __import__("paper_2103_07537_gb300.problems", fromlist=["x"]).mhd2d_cells(256, seed),
        levels=10, max_coarse=2500, restart=30, prec=32, coarse_prec=32, learned=True, cpu_sample_iters=5,
        desc="2D coupled 4-field Q1 system, 256x256 cells, 66,049 nodes, 396,294 unknowns, resistivity drawn per "
             "cell log-U[1e-4,1] (viscosity log-U[1e-3,1]); learned damping: network 8-64-64-2 (FP16 weights, "
             "FP32 arithmetic, trained on 2000 instances of 64^2..128^2 cells) gives the smoother damping per node "
             "and field and the prolongator smoothing per aggregate and field; FP32 V(1,1) (FP32 coarsest LU) "
             "inside FP64 FGMRES(30) to 1e-8; variants: the plain hierarchy (omega 0.5, tentative P) in FP64 and "
             "FP32"),
    "mhd2d_q2q1_128": dict(
        make=lambda seed: __import__("paper_2103_07537_gb300.problems", fromlist=["x"]).mhd2d_q2q1(128, seed),
        levels=4, max_coarse=0, restart=30, prec=64, omega=0.6, cpu_sample_iters=5, sub_solver_variants=True,
        desc="2D coupled system on mixed elements: (u,v,p) on 66,049 Q2 nodes, (Bx,By,psi) on 16,641 Q1 vertices "
             "(128x128 cells, 248,070 unknowns), 3 dofs/node, separate aggregation per field block, FP64 V(1,1) "
             "BGS omega=0.6 with the node fields as field blocks, 4 levels, FGMRES(30) to 1e-8"),
    "stokes3d_64": dict(
        make=lambda seed: __import__("paper_2103_07537_gb300.problems", fromlist=["x"]).stokes3d(64, seed),
        levels=10, max_coarse=2500, restart=50, prec=32, coarse_prec=32, cpu_sample_iters=5, pr_variants=True,
        desc="3D Stokes Q1-Q1 stabilised, 64^3 hex cells, 4 dofs/node, 1,098,500 unknowns, 7,189,057 blocks "
             "(115 M scalars), FP32 V(1,1) BGS omega=0.5 (FP32 LU of the 2048-unknown coarsest level) inside FP64 "
             "FGMRES(50) to 1e-8, 3 levels"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stokes3d_64", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--weights", default=None, help="damping network parameters (default: the committed file)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="row mappings: 1 = timed at setup (default); 0 / 2 / 3 / 4 = warp per row, thread per "
                         "row, thread per row in half-size CTAs, four lanes per row everywhere (for profiler runs "
                         "that must use the mappings a timed run chose)")
    ap.add_argument("--tail-dofs", type=int, default=None,
                    help="levels of at most this many unknowns run as one recorded launch (amg_params.tail_dofs)")
    ap.add_argument("--tail-grid", type=int, default=None, choices=[0, 1],
                    help="1: that launch is cooperative over every SM with grid barriers (amg_params.tail_grid)")
    ap.add_argument("--pdl", type=int, default=1, choices=[0, 1],
                    help="1 (default): programmatic dependent launches of the V-cycle kernels (amg_params.use_pdl)")
    ap.add_argument("--coarse-prec", type=int, default=None, choices=[32, 64],
                    help="precision of the coarsest direct solve of FP32 cycles (default: the workload's)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other-precision and plain-hierarchy comparisons (for profiler launch lists)")
    ap.add_argument("--ref-iters", type=int, default=5,
                    help="reference arm: inner FGMRES steps timed per step (the sample)")
    return ap.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_systems(weights, world):
    """Longest-processing-time partition of independent systems over ranks:
    systems by decreasing weight (stored blocks; ties by index), each to the
    least-loaded rank (ties: lowest rank). Returns each rank's system indices,
    ascending. Deterministic, so every rank computes the same partition."""
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += weights[i]
    return [sorted(p) for p in parts]


def reduce_timing(dist, ms, solved, device):
    """The job's timed region and output over ranks: (max of the ranks' times,
    sum of their converged systems). No data of the solve is exchanged."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(solved)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))


# the sources that define the kernels of each kind (the shared header and the
# public header are part of every kernel)
KIND_SOURCES = {
    "smooth": ["k_solve.cu", "bgs_body.cuh"], "residual": ["k_solve.cu"], "cast": ["k_solve.cu"], "coarse": ["k_solve.cu"],
    "tail": ["k_solve.cu", "bgs_body.cuh"], "spmv": ["k_solve.cu"], "restrict": ["k_solve.cu", "k_transfer.cu"],
    "prolong": ["k_solve.cu", "k_transfer.cu"], "krylov": ["k_krylov.cu"],
}


def source_digest(kind):
    """Digest of the sources of one kernel kind: a committed ncu traffic figure
    is used only while these files are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_07537_gb300", "csrc")
    for f in sorted(KIND_SOURCES.get(kind, sorted(os.listdir(csrc)))) + ["common.cuh"]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "bamg.h"), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu_index), "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        try:
            for line in open(self.file.name):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_median": statistics.median(float(r[3]) for r in rows
                                                                          if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def physical_gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local < len(ids) and ids[local].isdigit():
            return int(ids[local])
    return local


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_mlp(wl):
    """The learned workloads' network as the oracle reads it (FP16-rounded)."""
    if not wl.get("learned"):
        return None
    from paper_2103_07537_gb300 import learn

    return learn.load_weights(wl.get("weights") or learn.WEIGHTS_PATH).astype(np.float16).astype(np.float64)


def oracle_mlp_levels(wl):
    if not wl.get("learned"):
        return 0
    from paper_2103_07537_gb300 import learn

    return learn.trained_levels(wl.get("weights") or learn.WEIGHTS_PATH)


def oracle_full_solve(sys_, wl):
    import oracle

    t0 = time.perf_counter()
    h = oracle.Hierarchy.from_system(sys_, max_levels=wl["levels"], max_coarse=wl["max_coarse"], mlp=oracle_mlp(wl),
                                     mlp_levels=oracle_mlp_levels(wl), omega=wl.get("omega", 0.5))
    t1 = time.perf_counter()
    _, it, rr, conv = h.fgmres(sys_.rhs, tol=TOL, restart=wl["restart"], max_iter=wl.get("max_iter", MAX_ITER))
    t2 = time.perf_counter()
    return dict(setup_s=t1 - t0, solve_s=t2 - t1, iters=it, relres=rr, converged=conv)


def oracle_sample(sys_, wl, iters):
    """setup + `iters` inner FGMRES steps of the oracle (a bounded sample)."""
    import oracle

    t0 = time.perf_counter()
    h = oracle.Hierarchy.from_system(sys_, max_levels=wl["levels"], max_coarse=wl["max_coarse"], mlp=oracle_mlp(wl),
                                     mlp_levels=oracle_mlp_levels(wl), omega=wl.get("omega", 0.5))
    t1 = time.perf_counter()
    _, it, _, _ = h.fgmres(sys_.rhs, tol=1e-300, restart=wl["restart"], max_iter=iters)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(it, 1)


SOLVE_COUNTS = os.path.join(ROOT, "oracle", "solve_counts.json")


def oracle_solve_count(name, s, wl):
    """Inner steps of one full oracle solve of workload `name`, seed 1: the
    committed count (written by oracle/make_solve_counts.py, which runs the
    oracle only), else an untimed full oracle solve here."""
    try:
        c = json.load(open(SOLVE_COUNTS))[name]
        if c.get("seed") == 1 and c.get("restart") == wl["restart"]:
            return int(c["iterations"]), float(c["relres"]), "oracle/solve_counts.json"
    except Exception:
        pass
    full = oracle_full_solve(s, wl)
    return int(full["iters"]), float(full["relres"]), "an untimed full oracle solve"


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    s = wl["make"](1)
    full_iters, full_rr, src = oracle_solve_count(args.workload, s, wl)
    for _ in range(max(0, args.warmup)):
        oracle_sample(s, wl, 1)
    step_s, rates = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        t_setup, t_iter = oracle_sample(s, wl, args.ref_iters)
        step_s.append(time.perf_counter() - t0)
        rates.append(1.0 / (t_setup + t_iter * full_iters))  # one full solve, scaled from the sample
    value = statistics.mean(rates)
    sample = (f"per step: oracle setup + {args.ref_iters} inner FGMRES({wl['restart']}) steps of {args.workload} "
              f"seed 1 (timed: ms_per_step); value scales each step to one full solve of {full_iters} inner steps "
              f"(relres {full_rr:.2e}, from {src})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(step_s),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "name": args.workload, "seed": 1},
            "full_solve_scaling": {"inner_steps_sampled": args.ref_iters, "inner_steps_full_solve": full_iters,
                                   "source": src},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": 1, "sample": sample,
                             "host_cores_available": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2103_07537_gb300 import bamg

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    bamg.load()
    wl = dict(WORKLOADS[args.workload])
    if args.weights:
        wl["weights"] = args.weights
    learned = bool(wl.get("learned"))
    weights, mlp_levels = None, 0
    if learned:
        from paper_2103_07537_gb300 import learn

        weights = learn.load_weights(wl.get("weights") or learn.WEIGHTS_PATH)
        mlp_levels = learn.trained_levels(wl.get("weights") or learn.WEIGHTS_PATH)
    seed = 1 + rank
    batched = bool(wl.get("batched"))
    sharded = batched and world > 1
    if sharded:  # one batch; its systems split over the ranks (no exchange in the solve)
        from paper_2103_07537_gb300 import problems

        full = wl["make"](1)
        part = shard_systems([m.nnzb for m in full.members], world)[rank]
        made = problems.concatenate([full.members[i] for i in part])
        del full
    else:  # independent replicas
        made = wl["make"](seed)
    bt = made if batched else None
    s = made.system if batched else made
    max_iter = wl.get("max_iter", MAX_ITER)
    rp = torch.from_numpy(s.row_ptr).to(dev)
    ci = torch.from_numpy(s.col_idx).to(dev)
    va = torch.from_numpy(np.ascontiguousarray(s.vals.reshape(-1))).to(dev)
    b = torch.from_numpy(s.rhs).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    restart = wl["restart"]
    main_prec = wl["prec"]
    other_prec = 32 if main_prec == 64 else 64
    coarse_prec = (args.coarse_prec or wl.get("coarse_prec", 64)) if main_prec == 32 else 64
    node_fields = getattr(s, "node_field_off", None)
    params64 = bamg.amg_default_params(max_levels=wl["levels"], max_coarse=wl["max_coarse"], cycle_prec=main_prec,
                                       omega=wl.get("omega", 0.5),
                                       mlp=weights, mlp_levels=mlp_levels, autotune=args.autotune,
                                       coarse_prec=coarse_prec, use_pdl=args.pdl,
                                       tail_dofs=args.tail_dofs if args.tail_dofs is not None else wl.get("tail_dofs", 0),
                                       tail_grid=args.tail_grid if args.tail_grid is not None else wl.get("tail_grid", 0))

    def setup(params):
        if batched:
            return bamg.amg_setup_batched(bt.sys_node_off, rp, ci, va, s.n_nodes, s.nnzb, s.b, s.field_of_dof, params,
                                          stream)
        if node_fields is not None:
            return bamg.amg_setup_fields(node_fields, rp, ci, va, s.n_nodes, s.nnzb, s.b, params, stream)
        return bamg.amg_setup(rp, ci, va, s.n_nodes, s.nnzb, s.b, s.field_of_dof, params, stream)

    solved = [0]  # converged systems of the last step

    def step(params, profile=False):
        h = setup(params)
        try:
            if profile:
                bamg.amg_profile(h, True)
            x.zero_()
            if batched:
                st, its, rrs = bamg.fgmres_solve_batched(h, b, x, TOL, restart, max_iter, stream)
                solved[0] = int((rrs <= TOL).sum())
                it, rr = int(its.max()), float(rrs[rrs <= TOL].max()) if solved[0] else float("nan")
            else:
                st, it, rr = bamg.fgmres_solve(h, b, x, TOL, restart, max_iter, stream)
                solved[0] = 1 if st == 0 else 0
            prof = None
            if profile:  # per kernel kind and hierarchy level (-1: the outer FGMRES kernels)
                nl = bamg.amg_num_levels(h)
                prof = {(k, l): bamg.amg_profile_read_level(h, k, l) for k in bamg.KERNEL_KINDS
                        for l in range(-1, nl)}
        finally:
            bamg.amg_destroy(h)
        return st, it, rr, prof

    def timed(params, k_steps):
        tot = 0.0
        last = None
        nsolved = 0
        for _ in range(k_steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = step(params)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
            nsolved += solved[0]
        timed.solved = nsolved
        return tot, last

    for _ in range(max(args.warmup, 0)):
        step(params64)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    launches0 = bamg.amg_launch_count()
    with ClockSampler(physical_gpu_index(local)) as clk:
        total_ms, (st, iters, relres, _) = timed(params64, args.steps)
    launches = bamg.amg_launch_count() - launches0
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    t_max, job_solved = total_ms, timed.solved
    if pg:
        t_max, job_solved = reduce_timing(pg, total_ms, timed.solved, dev)
    solves_per_step = job_solved / args.steps  # converged systems per step over all ranks
    value = job_solved / (t_max / 1e3)
    clocks = clk.summary()

    # --- V-cycle and setup timings (the metric's "V-cycle ms") -------------------
    h = setup(params64)
    r = b.clone()
    z = torch.empty_like(b)
    for _ in range(5):
        bamg.amg_apply(h, r, z, stream)
    vt = []
    for _ in range(20):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bamg.amg_apply(h, r, z, stream)
        e1.record(stream)
        e1.synchronize()
        vt.append(e0.elapsed_time(e1))
    stats = bamg.amg_stats(h)
    bamg.amg_destroy(h)
    st_times = []
    for _ in range(3):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hh = setup(params64)
        e1.record(stream)
        e1.synchronize()
        bamg.amg_destroy(hh)
        st_times.append(e0.elapsed_time(e1))

    # --- the other cycle precision (FP32 cycle inside FP64 FGMRES, or FP64 cycle) --
    params_o = bamg.amg_default_params(max_levels=wl["levels"], max_coarse=wl["max_coarse"], cycle_prec=other_prec,
                                       mlp=weights, mlp_levels=mlp_levels, omega=wl.get("omega", 0.5))
    k_o = max(1, min(args.steps, 5))
    variant = None
    if not args.no_variants:
        step(params_o)
        ms_o, (st_o, it_o, rr_o, _) = timed(params_o, k_o)
        variant = {"cycle": (f"fp{other_prec} V-cycle inside fp64 FGMRES (fp64 outer SpMV, Arnoldi, coarse solve)"),
                   "value": timed.solved / (ms_o / 1e3), "unit": UNIT, "iterations": it_o, "relres": rr_o,
                   "converged": st_o == 0}
        # one V-cycle of each precision on the rhs: relative 2-norm distance
        # of the two outputs, the FP64 cycle's output as the reference
        try:
            outs = {}
            for prec_, pp_ in ((main_prec, params64), (other_prec, params_o)):
                hh_ = setup(pp_)
                try:
                    outs[prec_] = torch.empty_like(b)
                    bamg.amg_apply(hh_, b, outs[prec_], stream)
                    torch.cuda.synchronize(dev)
                finally:
                    bamg.amg_destroy(hh_)
            variant["vcycle_rel_diff_vs_fp64"] = float((outs[32] - outs[64]).norm() / outs[64].norm())
        except Exception:
            variant["vcycle_rel_diff_vs_fp64"] = None
    if learned and variant:
        variant["cycle"] = f"learned damping, {variant['cycle']}"
    # --- the paper's sub-solvers of Algorithm 1 against the multicolour sweep -------
    sub_solvers = None
    if wl.get("sub_solver_variants") and not args.no_variants:
        sub_solvers = {"multicolour_sweep": {"value": value, "unit": UNIT, "iterations": iters, "relres": relres,
                                             "vcycle_ms": statistics.median(vt), "cycle_prec": main_prec}}
        for key, sub in (("ilu0_colour_order", 1), ("restricted_schwarz_overlap1", 2)):
            for prec in (main_prec, other_prec):
                pp = bamg.amg_default_params(max_levels=wl["levels"], max_coarse=wl["max_coarse"], cycle_prec=prec,
                                             omega=wl.get("omega", 0.5), sub_solver=sub, use_pdl=args.pdl)
                name = key if prec == main_prec else f"{key}_fp{prec}"
                try:
                    step(pp)
                    ms_v, (st_v, it_v, rr_v, _) = timed(pp, k_o)
                    hh_ = setup(pp)
                    try:
                        zz = torch.empty_like(b)
                        for _ in range(3):
                            bamg.amg_apply(hh_, b, zz, stream)
                        ts_ = []
                        for _ in range(10):
                            e0 = torch.cuda.Event(enable_timing=True)
                            e1 = torch.cuda.Event(enable_timing=True)
                            e0.record(stream)
                            bamg.amg_apply(hh_, b, zz, stream)
                            e1.record(stream)
                            e1.synchronize()
                            ts_.append(e0.elapsed_time(e1))
                    finally:
                        bamg.amg_destroy(hh_)
                    sub_solvers[name] = {"value": timed.solved / (ms_v / 1e3), "unit": UNIT, "iterations": it_v,
                                         "relres": rr_v, "converged": st_v == 0,
                                         "vcycle_ms": statistics.median(ts_), "cycle_prec": prec}
                except Exception as exc:  # reported, not fatal
                    sub_solvers[name] = {"error": str(exc)[:200]}
    # --- FP32 cycle with a smoothed prolongator, P / R values in FP32 or BF16 ------
    pr_variants = None
    if wl.get("pr_variants") and not args.no_variants and main_prec == 32:
        pr_variants = {}
        z_ref = None
        for storage in (32, 16):
            pp = bamg.amg_default_params(max_levels=wl["levels"], max_coarse=wl["max_coarse"], cycle_prec=32,
                                         coarse_prec=coarse_prec, omega=wl.get("omega", 0.5), smooth_p=1,
                                         omega_p=PR_OMEGA_P, pr_storage=storage, use_pdl=args.pdl)
            key = f"smoothed_p_{'bf16' if storage == 16 else 'fp32'}"
            try:
                step(pp)
                ms_v, (st_v, it_v, rr_v, _) = timed(pp, k_o)
                hh_ = setup(pp)
                try:
                    zz = torch.empty_like(b)
                    bamg.amg_apply(hh_, b, zz, stream)
                    torch.cuda.synchronize(dev)
                finally:
                    bamg.amg_destroy(hh_)
                if z_ref is None:
                    z_ref = zz
                pr_variants[key] = {
                    "cycle": f"fp32 V-cycle, smoothed prolongator (omega_P {PR_OMEGA_P}) with P and R values "
                             f"stored in {'bf16' if storage == 16 else 'fp32'}, inside fp64 FGMRES",
                    "value": timed.solved / (ms_v / 1e3), "unit": UNIT, "iterations": it_v, "relres": rr_v,
                    "converged": st_v == 0,
                    "vcycle_rel_diff_vs_fp32_storage": float((zz - z_ref).norm() / z_ref.norm())}
            except Exception as exc:  # reported, not fatal: the main line stands
                pr_variants[key] = {"error": str(exc)[:200]}
    # --- learned workloads: the plain hierarchy, and the fallback rule --------
    plain = None
    if learned and not args.no_variants:
        plain = {}
        for prec in (64, 32):
            pp = bamg.amg_default_params(max_levels=wl["levels"], max_coarse=wl["max_coarse"], cycle_prec=prec)
            step(pp)
            ms_p, (st_p, it_p, rr_p, _) = timed(pp, k_o)
            plain[f"fp{prec}"] = {"value": timed.solved / (ms_p / 1e3), "unit": UNIT, "iterations": it_p,
                                  "relres": rr_p, "converged": st_p == 0,
                                  "cycle": f"plain hierarchy (omega 0.5, tentative P), fp{prec} V-cycle"}
        hl = setup(params64)
        hp = setup(bamg.amg_default_params(max_levels=wl["levels"], max_coarse=wl["max_coarse"], cycle_prec=main_prec))
        ch, il, ip = bamg.amg_select(hl, hp, b, TOL, restart, max_iter, stream)
        lstats = bamg.amg_stats(hl)
        bamg.amg_destroy(hl)
        bamg.amg_destroy(hp)
        plain["fallback"] = {"rule": "amg_select: the plain hierarchy is kept unless the learned one converges in "
                                     "no more iterations", "choice": "learned" if ch == 0 else "plain",
                             "iterations_learned": il, "iterations_plain": ip,
                             "smoothed_p_levels": [lv.get("smoothed_p", 0) for lv in lstats["levels"]]}
        plain["learned_vs_plain_fp64"] = value / plain["fp64"]["value"] if plain["fp64"]["value"] else None

    # --- per-kernel profile pass (events around every launch) --------------------
    kernels = {}     # per kind
    kernels_kl = {}  # per (kind, level)
    prof_iters_tot = 0
    for _ in range(max(1, args.profile_steps)):
        flush.zero_()
        _, it_p_, _, prof = step(params64, profile=True)
        prof_iters_tot += it_p_
        for (k, l), v in prof.items():
            for key, dst in ((k, kernels), ((k, l), kernels_kl)):
                acc = dst.setdefault(key, dict(ms=0.0, launches=0, bytes=0.0, flops=0.0))
                for f in acc:
                    acc[f] += v[f]
    peak_gbs, peak_src = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or 1920.0
    # The dominant kernel of the V-cycle (the metric's "V-cycle ms") and its
    # time per launch in the unprofiled cycle: the graph-replayed V-cycle time
    # times the kernel's share of the cycle's kernel time in the profiled pass
    # (events around every launch, which also cost each launch its gap), over
    # its launches per cycle.
    cycle_kinds = {"smooth", "residual", "restrict", "prolong", "tail", "cast", "coarse"}
    prof_iters = max(1, prof_iters_tot // max(1, args.profile_steps))  # V-cycles per profiled solve
    # the dominant kernel of the cycle: one kind on one level (one kernel
    # instance and row mapping, e.g. the finest level's smoother)
    cyc = {kl: v for kl, v in kernels_kl.items() if kl[0] in cycle_kinds and kl[1] >= 0 and v["launches"]}
    cyc_ms = sum(v["ms"] for v in cyc.values())
    dom_kl = max(cyc, key=lambda kl: cyc[kl]["ms"])
    dom = dom_kl[0]
    d = cyc[dom_kl]
    share = d["ms"] / cyc_ms if cyc_ms > 0 else 0.0
    vcycle_med = statistics.median(vt)
    launches_per_cycle = d["launches"] / (max(1, args.profile_steps) * prof_iters)
    us_per_launch = 1e3 * vcycle_med * share / max(launches_per_cycle, 1e-9)
    bytes_per_launch = d["bytes"] / max(1, d["launches"])
    flops_per_launch = d["flops"] / max(1, d["launches"])
    kernel_prec = main_prec if dom != "coarse" else (coarse_prec if main_prec == 32 else 64)
    fma_per_clk = 2 if kernel_prec == 64 else 128  # per SM on GB300 (FP64: measured 2.08 / clk / SM)
    alu_peak_tflops = SMS * fma_per_clk * 2 * sm_mhz * 1e6 / 1e12
    gbs = bytes_per_launch / (us_per_launch * 1e-6) / 1e9 if us_per_launch > 0 else 0.0
    tfl = flops_per_launch / (us_per_launch * 1e-6) / 1e12 if us_per_launch > 0 else 0.0
    t_mem = bytes_per_launch / (peak_gbs * 1e9)
    t_alu = flops_per_launch / (alu_peak_tflops * 1e12)
    # DRAM bytes per launch of the dominant kernel from a committed ncu capture,
    # only when the kernel sources are unchanged since that capture
    traffic = None
    pdir = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not f.endswith("_traffic.json"):
            continue
        try:
            tj = json.load(open(os.path.join(pdir, f)))
        except Exception:
            continue
        # the capture's kernel: the same sources, kind and workload, and (when
        # it names them) the same level and that level's smoother mapping
        mapping = tj.get("smoother_mapping")
        lv = tj.get("level")
        same_mapping = mapping is None or (
            mapping == [x.get("smoother_mapping") for x in stats["levels"][:-1]] if isinstance(mapping, list)
            else mapping == stats["levels"][dom_kl[1]].get("smoother_mapping"))
        if tj.get("source_digest") == source_digest(dom) and tj.get("kind") == dom and \
                tj.get("workload") == args.workload and (lv is None or lv == dom_kl[1]) and same_mapping:
            traffic = tj.get("dram_bytes_per_launch")
    if t_alu > t_mem:
        roofline = {"bound": "alu", "achieved": tfl, "peak": alu_peak_tflops, "unit": "TFLOP/s",
                    "frac": tfl / alu_peak_tflops, "traffic": traffic,
                    "peak_source": f"derived FP{kernel_prec} FMA peak: {SMS} SMs x {fma_per_clk} FMA/clk x 2 flop "
                                   f"x {sm_mhz:.0f} MHz",
                    "hbm_gbs": gbs, "hbm_frac": gbs / peak_gbs}
    else:
        roofline = {"bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs,
                    "traffic": traffic, "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "alu_tflops": tfl, "alu_frac": tfl / alu_peak_tflops}
    roofline.update({"kernel": dom, "level": dom_kl[1],
                     "mapping": (stats["levels"][dom_kl[1]].get("smoother_mapping") if dom == "smooth" else
                                 stats["levels"][dom_kl[1]].get("residual_mapping") if dom == "residual" else None),
                     "kernel_prec": f"fp{kernel_prec}",
                     "launches_per_cycle": launches_per_cycle, "us_per_launch": us_per_launch,
                     "bytes_per_launch": bytes_per_launch, "flops_per_launch": flops_per_launch,
                     "share_of_cycle": share, "vcycle_ms": vcycle_med,
                     "how": "us_per_launch = vcycle_ms x share_of_cycle / launches_per_cycle (share: the "
                            "kernel's part, on its level, of the cycle's kernel time in a profiled solve); achieved "
                            "= bytes_per_launch (algorithmic) / us_per_launch"})
    by_level = {f"{k}@{l}": {"ms_per_solve": v["ms"] / max(1, args.profile_steps),
                             "launches": v["launches"] // max(1, args.profile_steps),
                             "share_of_cycle": v["ms"] / cyc_ms if cyc_ms > 0 else None,
                             "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0}
                for (k, l), v in sorted(kernels_kl.items(), key=lambda kv: -kv[1]["ms"]) if v["launches"]}
    ksum = {k: {"ms_per_solve": v["ms"] / max(1, args.profile_steps), "launches": v["launches"] // max(1, args.profile_steps),
                "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0,
                "TFLOPs": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] > 0 else 0.0}
            for k, v in kernels.items() if v["launches"]}

    # --- end to end through the host-buffer entry point ---------------------------
    e2e = None
    if not args.no_e2e and (node_fields is not None or batched):
        # through the public API with host buffers: the host entry point copies
        # A and b to the device, sets up, solves and copies x back
        hp = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
              for a in (s.row_ptr, s.col_idx, s.vals.reshape(-1), s.rhs)]
        x_h = torch.zeros(s.n_unknowns, dtype=torch.float64).pin_memory().numpy()
        k_e = max(1, min(args.steps, 3))

        def host_solve():
            x_h[:] = 0.0
            if batched:
                _, _, rrs = bamg.amg_solve_batched_host(bt.sys_node_off, hp[0], hp[1], hp[2], s.n_nodes, s.nnzb, s.b,
                                                        s.field_of_dof, hp[3], x_h, TOL, restart, max_iter, params64,
                                                        stream)
                return int((rrs <= TOL).sum())
            st_e, _, _ = bamg.amg_solve_fields_host(node_fields, hp[0], hp[1], hp[2], s.n_nodes, s.nnzb, s.b, hp[3],
                                                    x_h, TOL, restart, MAX_ITER, params64, stream)
            return 1 if st_e == 0 else 0

        host_solve()
        tot = 0.0
        nsol = 0
        for _ in range(k_e):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nsol += host_solve()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        h2d = sum(a.nbytes for a in hp) + x_h.nbytes
        if pg:
            tot, nsol = reduce_timing(pg, tot, nsol, dev)
        e2e = {"value": nsol / (tot / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(x_h.nbytes),
               "api": ("amg_solve_batched_host" if batched else "amg_solve_fields_host") + " (pinned host buffers)"}
    elif not args.no_e2e:
        rp_h = torch.from_numpy(s.row_ptr).pin_memory().numpy()
        ci_h = torch.from_numpy(s.col_idx).pin_memory().numpy()
        va_h = torch.from_numpy(np.ascontiguousarray(s.vals.reshape(-1))).pin_memory().numpy()
        b_h = torch.from_numpy(s.rhs).pin_memory().numpy()
        x_h = torch.zeros(s.n_unknowns, dtype=torch.float64).pin_memory().numpy()
        k_e = max(1, min(args.steps, 5))
        bamg.amg_solve_host(rp_h, ci_h, va_h, s.n_nodes, s.nnzb, s.b, s.field_of_dof, b_h, x_h, TOL, restart,
                            MAX_ITER, params64, stream)
        tot = 0.0
        per_call = []
        for _ in range(k_e):
            x_h[:] = 0.0
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bamg.amg_solve_host(rp_h, ci_h, va_h, s.n_nodes, s.nnzb, s.b, s.field_of_dof, b_h, x_h, TOL,
                                restart, MAX_ITER, params64, stream)
            e1.record(stream)
            e1.synchronize()
            per_call.append(e0.elapsed_time(e1))
            tot += per_call[-1]
        h2d = rp_h.nbytes + ci_h.nbytes + va_h.nbytes + b_h.nbytes + x_h.nbytes
        nsol = k_e
        if pg:
            tot, nsol = reduce_timing(pg, tot, nsol, dev)
        e2e = {"value": nsol / (tot / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(x_h.nbytes), "api": "amg_solve_host (pinned host buffers)",
               "ms_per_call": [round(t, 3) for t in per_call]}

    # --- CPU baseline: the oracle on this host ------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if batched:
            # bounded sample: full oracle solves of the batch's systems in order
            # until about 15 s are spent, scaled by unknowns to the whole batch
            t_s = 0.0
            n_s = 0
            q = 0
            while t_s < 15.0 and q < len(bt.members):
                m = bt.members[q]
                full = oracle_full_solve(m, dict(wl, restart=restart))
                t_s += full["setup_s"] + full["solve_s"]
                n_s += m.n_unknowns
                q += 1
            t_all = t_s * s.n_unknowns / n_s
            cpu = {"kind": "oracle", "value": len(bt.members) / t_all, "unit": UNIT, "cores": 1,
                   "sample": f"full oracle solves (FGMRES({restart}) to 1e-8) of the first {q} of "
                             f"{len(bt.members)} systems ({t_s:.1f} s), scaled by unknowns to the batch",
                   "host_cores_available": os.cpu_count()}
        elif wl.get("cpu_sample_iters"):
            # bounded sample: oracle setup + a few inner steps, scaled to the
            # inner-step count of this solve (the oracle's count agrees within
            # one iteration, see the parity tests)
            k = wl["cpu_sample_iters"]
            n_full, src = iters, "this solve's count (the oracle's agrees within one step)"
            try:
                c = json.load(open(SOLVE_COUNTS))[args.workload]
                if c.get("seed") == seed and c.get("restart") == restart:
                    n_full, src = int(c["iterations"]), "oracle/solve_counts.json"
            except Exception:
                pass
            t_setup, t_iter = oracle_sample(s, wl, k)
            t = t_setup + t_iter * n_full
            cpu = {"kind": "oracle", "value": 1.0 / t, "unit": UNIT, "cores": 1,
                   "sample": f"oracle setup + {k} inner FGMRES({restart}) steps of {args.workload} seed {seed}, "
                             f"scaled to {n_full} inner steps (from {src}); single-threaded C oracle",
                   "host_cores_available": os.cpu_count()}
        else:
            full = oracle_full_solve(s, wl)
            t = full["setup_s"] + full["solve_s"]
            cpu = {"kind": "oracle", "value": 1.0 / t, "unit": UNIT, "cores": 1,
                   "sample": f"one full solve (setup + FGMRES({restart}) to 1e-8, {full['iters']} inner steps) of "
                             f"{args.workload} seed {seed}, single-threaded C oracle",
                   "host_cores_available": os.cpu_count(), "iterations": full["iters"]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "strong" if sharded else "weak", "vs_baseline": None,
                "dtype": "f64" if main_prec == 64 else "f32+f64",
                "data": "synthetic",
                "config": {"workload": wl["desc"], "name": args.workload, "seed": seed,
                           "l2": "flushed between steps (256 MiB write outside the timed step)",
                           "parallelism": ("systems of one batch sharded over ranks (LPT on stored blocks)"
                                           if sharded else "replicas" if world > 1 else "single GPU"),
                           "step": "amg_setup + fgmres_solve to 1e-8 + amg_destroy, inputs resident in HBM"},
                "iterations": iters, "relres": relres, "converged": st == 0,
                "solves_per_step": solves_per_step,
                "vcycle_ms": statistics.median(vt), "setup_ms": statistics.median(st_times),
                "levels": [lv["n"] for lv in stats["levels"]],
                "field_nodes": ([lv.get("field_nodes") for lv in stats["levels"]]
                                if stats.get("node_fields", 1) > 1 else None),
                "colours": [lv["colours"] for lv in stats["levels"]],
                "mappings": {"smoother": [lv.get("smoother_mapping") for lv in stats["levels"][:-1]],
                             "residual": [lv.get("residual_mapping") for lv in stats["levels"][:-1]],
                             "tune_us": [lv.get("tune_us") for lv in stats["levels"][:-1]],
                             "tune_step_us": [lv.get("tune_step_us") for lv in stats["levels"][:-1]],
                             "field_major": [lv.get("field_major") for lv in stats["levels"][:-1]],
                             "outer_spmv": stats.get("outer_mapping"), "outer_us": stats.get("outer_us")},
                "setup_phase_ms": stats.get("setup_phase_ms"),
                "cycle_prec": main_prec, "coarse_prec": coarse_prec,
                "use_pdl": args.pdl,
                "tail": {"level": stats.get("tail_level"), "grid_ctas": stats.get("tail_grid"),
                         "cluster": stats.get("tail_cluster")}, "variant": variant, "pr_variants": pr_variants, "sub_solvers": sub_solvers,
                "plain": plain,
                "kernels": ksum, "kernels_by_level": by_level, "roofline": roofline,
                "clocks": clocks,
                "gpu_launches": int(launches), "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
