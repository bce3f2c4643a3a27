"""The multi-rank path on CPU: two gloo ranks take the shot ranges that
bench.py gives them, decode with the oracle, judge, and sum their failure
counters; the result equals one process decoding the union of the shots,
and the ranges of all (step, rank, p) are disjoint and cover the job."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2605_14170_gb300 import shard
from paper_2605_14170_gb300.inputs import named_code

P_LIST = (0.04, 0.08)
S, STEPS, R, ITERS = 12, 2, 4, 30


def failures(first, p, H, Ho, sets):
    ex, _ = oracle.sample(7, first, S, H.shape[1], p, "depolarizing")
    s = oracle.syndrome(H, ex)
    llr = np.full(H.shape[1], np.log((1 - 2 * p / 3) / (2 * p / 3)))
    out = oracle.mbbp_decode(H, sets, s, llr, ITERS, 0.625)
    return int((oracle.judge(H, Ho, ex, out["ehat"]) != 0).sum())


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = named_code("bb72")
    sets = oracle.collect_subtrees(c.HZ, R, 3)
    counts = torch.zeros(len(P_LIST), dtype=torch.int64)
    firsts = []
    for k in range(STEPS):
        for ip, p in enumerate(P_LIST):
            first = shard.first_shot(k, rank, world, ip, len(P_LIST), S)
            firsts.append(first)
            counts[ip] += failures(first, p, c.HZ, c.HX, sets)
    shard.reduce_counters(dist, counts)
    t = shard.max_over_ranks(dist, float(rank + 1), "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, firsts)
    if rank == 0:
        q.put((counts.tolist(), t, gathered))
    dist.destroy_process_group()


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_match_one_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    counts, tmax, firsts = q.get(timeout=600)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == float(world)  # max over ranks
    starts = sorted(f for fs in firsts for f in fs)
    assert starts == [i * S for i in range(STEPS * world * len(P_LIST))]  # disjoint, covering
    # one process over the same shots
    c = named_code("bb72")
    sets = oracle.collect_subtrees(c.HZ, R, 3)
    want = [0] * len(P_LIST)
    for k in range(STEPS):
        for r in range(world):
            for ip, p in enumerate(P_LIST):
                want[ip] += failures(shard.first_shot(k, r, world, ip, len(P_LIST), S), p, c.HZ, c.HX, sets)
    assert counts == want
    assert sum(want) > 0
