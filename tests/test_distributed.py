"""Sharded Multi-start SPVAR on CPU: world size 2 over gloo.

Each rank runs its block of global starts (here with the oracle, which has no
GPU needs); combining the shards must reproduce the single-process run
exactly: the same per-start best energies, the same global minimum and the
same success rate.
"""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import distributed as D
from paper_1706_07826_gb300 import instances as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    inst = I.cubic3d(3, 77)
    p = O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h)
    thr = O.thresholds(O.beta_geometric(40, 0.1, 3.0), O.dmax(p), 1)
    return p, thr


STARTS = 7


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, thr = _problem()
        first, count = D.shard_starts(STARTS, rank, world)
        r = O.solve(p, thr, seed=9, num_starts=count, fixing_sample_size=16, solving_sample_size=8,
                    elite_threshold=0.25, start0=first)
        gmin, allb = D.combine_best(r.best_e, device=None)
        q.put((rank, gmin, allb.tolist()))
    finally:
        dist.destroy_process_group()


def test_shard_starts_partitions_exactly():
    for n in (0, 1, 7, 10, 64):
        for w in (1, 2, 3, 8):
            blocks = [D.shard_starts(n, r, w) for r in range(w)]
            covered = [s for f, c in blocks for s in range(f, f + c)]
            assert covered == list(range(n))
            assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1


def test_two_gloo_ranks_reproduce_single_process():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, thr = _problem()
    ref = O.solve(p, thr, seed=9, num_starts=STARTS, fixing_sample_size=16, solving_sample_size=8,
                  elite_threshold=0.25)
    for rank, gmin, allb in out:
        assert allb == ref.best_e.tolist()
        assert gmin == ref.best_e.min()
    assert D.success_rate(ref.best_e, ref.best_e.min()) == pytest.approx((ref.best_e == ref.best_e.min()).mean())
