"""Training and use of the damping network (beyond the paper).

The paper fixes one damping of its block Gauss-Seidel smoother near 0.5 and
shows (Sec. 5, iterations against the BGS damping) that the best value
depends on the problem.  Here a network 8 -> 64 -> 64 -> 2 maps features of
a level's matrix to the damping of every node and field (head 0) and to the
prolongator-smoothing weight of every aggregate and field (head 1).

Targets come from the convergence histories of the plain method itself: for
every training instance a coordinate search over the damping of (fine level,
field) and (coarser levels, field), started from the paper's 0.5, keeps the
values with the fewest FGMRES iterations to 1e-8; it runs once on the
tentative hierarchy and once on a hierarchy whose prolongator is smoothed
with weight P_WEIGHT, and the instance keeps the better of the two (its
P-smoothing target is then P_WEIGHT or 0).  All instances of a group are
searched together by the batched GPU solver (per-node dampings set with
amg_set_omega).  Each node row is labelled with its instance's damping for
its level and field and each aggregate row with the instance's P-smoothing
weight; the network is trained with the library's gradient and Adam kernels
(FP16 parameters, FP32 arithmetic).  The plain hierarchy stays the fallback
(amg_select).

Run ``python -m paper_2103_07537_gb300.learn --out <file.npz>`` on a GPU.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

from . import bamg
from . import problems as P

FINE = (0.55, 0.6, 0.65)                  # candidate dampings of the finest level
COARSE = (0.6, 0.7, 0.8, 0.9)             # candidate dampings of the coarser levels
P_WEIGHT = 0.1                            # candidate P-smoothing weight (0 = tentative P)
PLAIN = 0.5                               # the paper's damping
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "damping_mlp.npz")

# parameter offsets (include/bamg.h)
NF, NH, NO = bamg.NFEAT, bamg.MLP_H, bamg.MLP_OUT
O_W1, O_B1 = 0, NH * NF
O_W2 = O_B1 + NH
O_B2 = O_W2 + NH * NH
O_W3 = O_B2 + NH
O_B3 = O_W3 + NO * NH
O_XM = O_B3 + NO
O_XS = O_XM + NF


def instance_size(seed: int, lo: int, hi: int) -> int:
    """Cells per side of training instance `seed`, uniform in [lo, hi] (a
    stream position of its own, far from the instance's draws)."""
    u = P.uniform01(seed, 1 << 40, 1)[0]
    return min(hi, lo + int(u * (hi - lo + 1)))


def _make(args):
    N, seed = args
    return P.mhd2d_cells(N, seed)


def make_instances(seeds, lo=64, hi=128, pool=None):
    """The per-cell-resistivity systems of the given seeds, generated by
    `pool` (a spawn pool: safe after the parent has touched the GPU) or here."""
    jobs = [(instance_size(q, lo, hi), q) for q in seeds]
    if pool is None:
        return [_make(j) for j in jobs]
    return pool.map(_make, jobs, chunksize=2)


def _dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


class BatchSearch:
    """One batched hierarchy of a group of instances and the damping search on it."""

    def __init__(self, systems, levels=3, restart=30, max_iter=600, tol=1e-8, cycle_prec=32):
        import torch

        self.torch = torch
        self.systems = systems
        self.bt = P.concatenate(systems)
        s = self.bt.system
        self.F = max(s.field_of_dof) + 1
        self.rp, self.ci, self.va = _dev(torch, s.row_ptr), _dev(torch, s.col_idx), _dev(torch, s.vals.reshape(-1))
        self.rhs = _dev(torch, s.rhs)
        self.x = torch.zeros_like(self.rhs)
        self.kw = dict(max_levels=levels, max_coarse=0, cycle_prec=cycle_prec, autotune=0)
        self.restart, self.max_iter, self.tol = restart, max_iter, tol
        self.solver = bamg.BatchSolver(self.bt.sys_node_off, self.rp, self.ci, self.va, s.b, s.field_of_dof,
                                       **self.kw)
        self.nlev = self.solver.num_levels

    def _apply(self, solver, cfg):
        """cfg[nsys, 2, F]: damping of group 0 (finest level) and 1 (the others)."""
        for l in range(solver.num_levels - 1):
            counts = np.diff(solver.level_systems(l))
            arr = np.repeat(cfg[:, 0 if l == 0 else 1, :], counts, axis=0)
            solver.set_omega(l, _dev(self.torch, arr.reshape(-1)))

    def iterations(self, cfg, solver=None):
        solver = solver or self.solver
        self._apply(solver, cfg)
        self.x.zero_()
        _, its, rr = solver.solve(self.rhs, self.x, self.tol, self.restart, self.max_iter)
        its = its.astype(np.int64)
        its[~(rr <= self.tol)] = self.max_iter + 100  # not converged: worse than any count
        return its

    def _coordinate_search(self, solver):
        """Coordinate descent over (group, field) from the paper's damping;
        returns (cfg, iterations at the start, best iterations)."""
        cfg = np.full((len(self.systems), 2, self.F), PLAIN)
        start = self.iterations(cfg, solver)
        best = start.copy()
        for g, cands in ((0, FINE), (1, COARSE)):
            for f in range(self.F):
                for v in cands:
                    trial = cfg.copy()
                    trial[:, g, f] = v
                    it = self.iterations(trial, solver)
                    better = it < best
                    cfg[better, g, f] = v
                    best[better] = it[better]
        return cfg, start, best

    def search(self):
        """Searches the dampings on the tentative and on the smoothed (weight
        P_WEIGHT) hierarchy; each instance keeps the better of the two."""
        s = self.bt.system
        sp = bamg.BatchSolver(self.bt.sys_node_off, self.rp, self.ci, self.va, s.b, s.field_of_dof, smooth_p=1,
                              omega_p=P_WEIGHT, **self.kw)
        cfg0, plain, best0 = self._coordinate_search(self.solver)
        cfg1, start1, best1 = self._coordinate_search(sp)
        del sp
        use_p = best1 < best0
        cfg = np.where(use_p[:, None, None], cfg1, cfg0)
        return dict(cfg=cfg, plain=plain, best=np.minimum(best0, best1), wp=np.where(use_p, P_WEIGHT, 0.0),
                    smoothed_plain_damping=start1, best_tentative=best0)

    def rows(self, result, rng, node_rows=256, agg_rows=128):
        """Features (FP32, computed by amg_features on every level of the
        plain hierarchy) and targets of sampled node and aggregate rows."""
        torch = self.torch
        F = self.F
        lib = bamg.load()
        s = self.bt.system
        X, T, H = [], [], []
        for l in range(self.nlev - 1):
            info = bamg.amg_level_info(self.solver.handle, l)
            n, nnzb, nagg = info[0], info[1], info[3]
            rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
            ci = torch.empty(nnzb, dtype=torch.int32, device="cuda")
            va = torch.empty(nnzb * s.b * s.b, dtype=torch.float64, device="cuda")
            agg = torch.empty(n, dtype=torch.int32, device="cuda")
            st = lib.amg_level_copy(self.solver.handle, l, rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                                    agg.data_ptr(), None, None)
            if st != bamg.BAMG_OK:
                raise bamg.BamgError(st, "amg_level_copy")
            nf = torch.empty((n, F, NF), dtype=torch.float32, device="cuda")
            af = torch.empty((nagg, F, NF), dtype=torch.float32, device="cuda")
            bamg.amg_features(rp, ci, va, n, s.b, s.field_of_dof, agg, nagg, l, nf, af)
            nf, af = nf.cpu().numpy(), af.cpu().numpy()
            off = self.solver.level_systems(l)
            offc = self.solver.level_systems(l + 1)
            g = 0 if l == 0 else 1
            for q in range(len(self.systems)):
                nodes = np.arange(off[q], off[q + 1])
                pick = rng.choice(nodes.size * F, size=min(node_rows, nodes.size * F), replace=False)
                rows = nf[nodes].reshape(-1, NF)[pick]
                X.append(rows)
                T.append(result["cfg"][q, g, pick % F])
                H.append(np.zeros(pick.size, np.int32))
                aggs = np.arange(offc[q], offc[q + 1])
                pick = rng.choice(aggs.size * F, size=min(agg_rows, aggs.size * F), replace=False)
                X.append(af[aggs].reshape(-1, NF)[pick])
                T.append(np.full(pick.size, result["wp"][q]))
                H.append(np.ones(pick.size, np.int32))
            del rp, ci, va, agg
        return (np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32),
                np.concatenate(H).astype(np.int32))


def init_params(seed: int, X: np.ndarray, T: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Uniform fan-in scaled weights from the seeded generator; the input
    normalisation from the training rows; output biases at the mean targets."""
    p = np.zeros(bamg.MLP_NPARAMS, np.float32)
    u = P.uniform01(seed, 0, bamg.MLP_NTRAIN) * 2.0 - 1.0
    p[O_W1:O_B1] = u[O_W1:O_B1] * np.sqrt(3.0 / NF)
    p[O_W2:O_B2] = u[O_W2:O_B2] * np.sqrt(3.0 / NH)
    p[O_W3:O_B3] = u[O_W3:O_B3] * np.sqrt(3.0 / NH) * 0.1
    p[O_B3] = T[H == 0].mean() if (H == 0).any() else PLAIN
    p[O_B3 + 1] = T[H == 1].mean() if (H == 1).any() else 0.0
    p[O_XM:O_XS] = X.mean(axis=0)
    sd = X.std(axis=0)
    p[O_XS:] = np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 1.0)
    return p


def train(X, T, H, epochs=20, batch=4096, lr=2e-3, seed=7, Xv=None, Tv=None, Hv=None, log=print):
    """Adam on the mean squared error with the library's kernels; returns
    (params, history)."""
    import torch

    p = init_params(seed, X, T, H)
    dp = torch.from_numpy(p).cuda()
    p16 = torch.empty(bamg.MLP_NPARAMS, dtype=torch.int16, device="cuda")
    bamg.mlp_pack(dp, p16)
    m = torch.zeros(bamg.MLP_NTRAIN, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    g = torch.empty_like(m)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dX, dT, dH = (torch.from_numpy(a).cuda() for a in (X, T, H))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    step = 0
    hist = []
    n = X.shape[0]
    for ep in range(epochs):
        lr_ep = lr * (0.5 * (1.0 + np.cos(np.pi * ep / epochs)))  # cosine decay
        perm = torch.randperm(n, device="cuda", generator=gen)
        tot, cnt = 0.0, 0
        for s0 in range(0, n - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            xb, tb, hb = dX[idx].contiguous(), dT[idx].contiguous(), dH[idx].contiguous()
            bamg.mlp_grad(p16, xb, tb, hb, batch, g, loss)
            step += 1
            bamg.mlp_adam(dp, p16, g, m, v, step, lr=lr_ep)
            if s0 % (batch * 64) == 0:
                tot += float(loss.item())
                cnt += 1
        rec = dict(epoch=ep, train_loss=tot / max(cnt, 1))
        if Xv is not None:
            rec["val_loss"] = evaluate_loss(p16, Xv, Tv, Hv)
        hist.append(rec)
        log(json.dumps(rec))
    return dp.cpu().numpy(), hist


def evaluate_loss(p16, X, T, H):
    import torch

    n = X.shape[0]
    y = torch.empty((n, NO), dtype=torch.float32, device="cuda")
    bamg.mlp_forward(p16, torch.from_numpy(X).cuda(), n, y)
    y = y.cpu().numpy()
    return float(np.mean((y[np.arange(n), H] - T) ** 2))


def load_weights(path: str = WEIGHTS_PATH) -> np.ndarray:
    with np.load(path) as z:
        return z["params"].astype(np.float32)


def trained_levels(path: str = WEIGHTS_PATH) -> int:
    """Levels (from the finest) the network was trained on: its weights are
    used there (amg_params.mlp_levels); deeper levels keep the plain method."""
    with np.load(path) as z:
        return int(json.loads(str(z["meta"])).get("levels_trained", 0))


def evaluate(seeds, N, weights, cycle_prec=64, levels=10, max_coarse=2500, restart=30, max_iter=3000, tol=1e-8,
             log=print, mlp_levels=None):
    """Plain against learned hierarchy on held-out instances: iterations to
    tol, setup + solve time (CUDA events), and the fallback choice of
    amg_select (the plain hierarchy judges the learned one)."""
    import torch

    if mlp_levels is None:
        mlp_levels = trained_levels()
    out = []
    for q in seeds:
        s = P.mhd2d_cells(N, q)
        rp, ci, va = _dev(torch, s.row_ptr), _dev(torch, s.col_idx), _dev(torch, s.vals.reshape(-1))
        b = _dev(torch, s.rhs)
        rec = dict(seed=int(q), N=int(N))
        hs = {}
        for name, extra in (("plain", {}), ("learned", dict(mlp=weights, mlp_levels=mlp_levels))):
            prm = bamg.amg_default_params(max_levels=levels, max_coarse=max_coarse, cycle_prec=cycle_prec, **extra)
            x = torch.zeros_like(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            h = bamg.amg_setup(rp, ci, va, s.n_nodes, s.nnzb, s.b, s.field_of_dof, prm)
            st, it, rr = bamg.fgmres_solve(h, b, x, tol, restart, max_iter)
            e1.record()
            e1.synchronize()
            stats = bamg.amg_stats(h)
            rec[name] = dict(iterations=int(it), converged=st == bamg.BAMG_OK, relres=float(rr),
                             ms=float(e0.elapsed_time(e1)),
                             smoothed_levels=[lv.get("smoothed_p", 0) for lv in stats["levels"]])
            hs[name] = h
        ch, il, ip = bamg.amg_select(hs["learned"], hs["plain"], b, tol, restart, max_iter)
        rec["choice"] = "learned" if ch == 0 else "plain"
        for h in hs.values():
            bamg.amg_destroy(h)
        out.append(rec)
        log(json.dumps(rec))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--instances", type=int, default=2000)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--lo", type=int, default=64)
    ap.add_argument("--hi", type=int, default=128)
    ap.add_argument("--group", type=int, default=250, help="instances per batched search")
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    ap.add_argument("--log", default=None)
    ap.add_argument("--search-out", default=None, help="per-instance search results (JSON)")
    ap.add_argument("--evaluate", default=None, metavar="SEEDS",
                    help="instead of training: compare plain and learned on seeds a-b of the given --N")
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--cycle-prec", type=int, default=64)
    ap.add_argument("--weights", default=WEIGHTS_PATH)
    args = ap.parse_args(argv)
    if args.evaluate:
        import torch

        a, b = (int(v) for v in args.evaluate.split("-"))
        torch.cuda.set_device(0)
        res = evaluate(range(a, b + 1), args.N, load_weights(args.weights), cycle_prec=args.cycle_prec,
                       mlp_levels=trained_levels(args.weights))
        pl = [r["plain"]["iterations"] for r in res]
        le = [r["learned"]["iterations"] for r in res]
        ch = [min(r["plain"]["iterations"], r["learned"]["iterations"]) if r["choice"] == "learned"
              else r["plain"]["iterations"] for r in res]
        summ = dict(seeds=[a, b], N=args.N, cycle_prec=args.cycle_prec, plain_mean=float(np.mean(pl)),
                    learned_mean=float(np.mean(le)), with_fallback_mean=float(np.mean(ch)),
                    learned_better=int(sum(l < p for l, p in zip(le, pl))),
                    plain_ms_mean=float(np.mean([r["plain"]["ms"] for r in res])),
                    learned_ms_mean=float(np.mean([r["learned"]["ms"] for r in res])))
        print(json.dumps(dict(summary=summ)))
        if args.out and args.out != WEIGHTS_PATH:
            with open(args.out, "w") as f:
                json.dump(dict(summary=summ, instances=res), f)
        return
    logf = open(args.log, "w") if args.log else None

    def log(msg):
        print(msg, flush=True)
        if logf:
            logf.write(msg + "\n")
            logf.flush()

    seeds = list(range(args.seed0, args.seed0 + args.instances))
    t0 = time.time()
    # instance generation in worker processes, one group at a time (the pool is
    # started before the first GPU call)
    pool = mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1)))
    import torch

    torch.cuda.set_device(0)
    bamg.load()
    rng = np.random.default_rng(args.seed0)
    Xs, Ts, Hs, summary = [], [], [], []
    levels_trained = 0
    for g0 in range(0, len(seeds), args.group):
        t1 = time.time()
        group = make_instances(seeds[g0:g0 + args.group], args.lo, args.hi, pool)
        t_gen = time.time() - t1
        bs = BatchSearch(group)
        res = bs.search()
        X, T, H = bs.rows(res, rng)
        levels_trained = max(levels_trained, bs.nlev - 1)
        Xs.append(X)
        Ts.append(T)
        Hs.append(H)
        summary.append(dict(plain=res["plain"].tolist(), best=res["best"].tolist(),
                            best_tentative=res["best_tentative"].tolist(),
                            smoothed_plain_damping=res["smoothed_plain_damping"].tolist(),
                            cfg=res["cfg"].reshape(len(bs.systems), -1).tolist(), wp=res["wp"].tolist()))
        log(json.dumps(dict(stage="search", first=g0, plain_mean=float(res["plain"].mean()),
                            best_mean=float(res["best"].mean()), p_smoothed=int((res["wp"] > 0).sum()),
                            rows=int(X.shape[0]), generate_s=round(t_gen, 1), s=round(time.time() - t1, 1))))
        del bs, group
        torch.cuda.empty_cache()
    pool.close()
    ngrp = len(Xs)
    nval = max(1, ngrp // 10)  # the last groups hold out instances for the validation loss
    X, T, H = (np.concatenate(a[:ngrp - nval]) for a in (Xs, Ts, Hs))
    Xv, Tv, Hv = (np.concatenate(a[ngrp - nval:]) for a in (Xs, Ts, Hs))
    params, hist = train(X, T, H, epochs=args.epochs, Xv=Xv, Tv=Tv, Hv=Hv, log=log)
    meta = dict(instances=len(seeds), seeds=[seeds[0], seeds[-1]], sizes=[args.lo, args.hi], levels_trained=levels_trained,
                workload="mhd2d_cells (per-cell resistivity log-uniform in [1e-4, 1])", fine=FINE, coarse=COARSE,
                p_weight=P_WEIGHT, rows_train=int(X.shape[0]), rows_val=int(Xv.shape[0]), history=hist,
                search=dict(plain_mean=float(np.mean([np.mean(s["plain"]) for s in summary])),
                            best_mean=float(np.mean([np.mean(s["best"]) for s in summary]))),
                seconds=round(time.time() - t0, 1))
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, params=params, meta=json.dumps(meta))
    if args.search_out:
        with open(args.search_out, "w") as f:
            json.dump(dict(meta=meta, groups=summary), f)
    log(json.dumps(dict(stage="done", out=args.out, s=meta["seconds"])))


if __name__ == "__main__":
    main()
