"""The benchmark's multi-rank path on the CPU (gloo, two ranks): the
partition of a batch's independent systems over ranks and the reduction of
the timed region and converged counts.  The systems are solved by the oracle
here, so no GPU is involved; the GPU path uses the same two helpers."""
import os
import socket

import numpy as np
import pytest

import bench
import oracle
from paper_2103_07537_gb300 import problems as P

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def test_shard_systems_lpt():
    w = [5, 3, 3, 2, 2, 2, 9, 1]
    parts = bench.shard_systems(w, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(w)))                 # every system exactly once
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(w)           # LPT bound
    assert parts == bench.shard_systems(w, 3)          # deterministic
    assert bench.shard_systems([4, 4], 1) == [[0, 1]]
    assert bench.shard_systems([1, 1], 4) == [[0], [1], [], []]
    # greedy by decreasing weight: the heaviest systems go to distinct ranks
    assert [6 in p for p in parts].count(True) == 1 and not any(6 in p and 0 in p for p in parts)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        full = P.mhd2d_batch(6, 3, nmin=8, nmax=14)
        part = bench.shard_systems([m.nnzb for m in full.members], world)[rank]
        mine = P.concatenate([full.members[i] for i in part])
        solved = 0
        for m in mine.members:  # each rank's systems, independently (oracle on the CPU)
            h = oracle.Hierarchy.from_system(m, max_levels=3, max_coarse=0)
            _, _, rr, ok = h.fgmres(m.rhs, tol=1e-8, restart=30, max_iter=400)
            solved += int(ok and rr <= 1e-8)
        ms = 10.0 * (rank + 1)
        t, n = bench.reduce_timing(dist, ms, solved, "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, part)
        q.put((rank, t, n, solved, gathered))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_batch_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    full = P.mhd2d_batch(6, 3, nmin=8, nmax=14)
    total = 0
    for m in full.members:
        h = oracle.Hierarchy.from_system(m, max_levels=3, max_coarse=0)
        _, _, rr, ok = h.fgmres(m.rhs, tol=1e-8, restart=30, max_iter=400)
        total += int(ok and rr <= 1e-8)
    for rank, t, n, solved, gathered in out:
        assert t == 20.0                                     # max of the ranks' timed regions
        assert n == total == sum(o[3] for o in out)          # converged systems summed over ranks
        flat = sorted(i for p in gathered for i in p)
        assert flat == list(range(len(full.members)))        # the shards cover the batch once
        assert all(set(a).isdisjoint(b) for a in gathered for b in gathered if a is not b)
