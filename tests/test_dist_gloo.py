"""The multi-process (one rank per GPU) host logic on CPU with gloo, world
size 2: shards cover the elements once, timings reduce by max over ranks,
and -- with the oracle as the computation -- the ranks' ciphertexts, each
drawn at its global index, concatenate to the single-process encryption."""
import multiprocessing as mp
import os
import socket

import numpy as np

from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W
from paper_2601_14980_b300.dist import max_over_ranks, shard

TOTAL, SEED, STREAM = 13, 31, 5


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, count = shard(TOTAL, rank, world)
        parts = [None] * world
        dist.all_gather_object(parts, (start, count))
        mx = max_over_ranks([rank + 0.5, 10.0 - rank])
        p, q = W.primes(256, 3)
        key = P.derive_key(p, q)
        m = W.plaintexts_u64(TOTAL, seed=2)[start:start + count]
        cts = P.encrypt(key, [int(x) for x in m], [P.r_of(key, SEED, STREAM, start + i) for i in range(count)])
        allc = [None] * world
        dist.all_gather_object(allc, cts)
        out.put((rank, parts, mx, allc))
    finally:
        dist.destroy_process_group()


def test_shards_and_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [out.get(timeout=120) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    res.sort()
    parts = res[0][1]
    assert parts == res[1][1]
    covered = [i for (s, c) in parts for i in range(s, s + c)]
    assert covered == list(range(TOTAL))
    assert res[0][2] == res[1][2] == [1.5, 10.0]
    p, q = W.primes(256, 3)
    key = P.derive_key(p, q)
    m = W.plaintexts_u64(TOTAL, seed=2)
    whole = P.encrypt(key, [int(x) for x in m], [P.r_of(key, SEED, STREAM, i) for i in range(TOTAL)])
    assert res[0][3][0] + res[0][3][1] == whole


def test_shard_bounds():
    for total in (0, 1, 7, 100):
        for world in (1, 2, 3, 8):
            spans = [shard(total, r, world) for r in range(world)]
            assert sum(c for _, c in spans) == total
            assert all(spans[r][0] + spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


# ------------------------------------------------------------------ failure detection (host side)
def _edge(rank, port, drop_round, ready):
    import torch.distributed as dist

    from paper_2601_14980_b300.dist import post_segment

    store = dist.TCPStore("127.0.0.1", port, 3, False, timeout=__import__("datetime").timedelta(seconds=60))
    for rnd in (1, 2):
        if rnd == drop_round:
            ready.wait(60)  # a delayed node: its segment arrives only after the master gave up waiting
        post_segment(store, rnd, rank - 1)


def test_missing_edge_segment_detected_then_recovered():
    """Three processes (a master and two edge nodes) share a TCP store on
    127.0.0.1.  Round 1: both segments arrive.  Round 2: node 1 is late; the
    master's bounded wait names it as missing; once it arrives, a second
    wait finds nothing missing."""
    import datetime

    import torch.distributed as dist

    from paper_2601_14980_b300.dist import missing_segments

    ctx = mp.get_context("spawn")
    port = _free_port()
    store = dist.TCPStore("127.0.0.1", port, 3, True, timeout=datetime.timedelta(seconds=60), wait_for_workers=False)
    ready = ctx.Event()
    procs = [ctx.Process(target=_edge, args=(r, port, 2 if r == 2 else 0, ready)) for r in (1, 2)]
    for pr in procs:
        pr.start()
    try:
        assert missing_segments(store, 1, [0, 1], timeout_s=30.0) == []
        assert missing_segments(store, 2, [0, 1], timeout_s=0.5) == [1]
        ready.set()
        assert missing_segments(store, 2, [0, 1], timeout_s=30.0) == []
    finally:
        ready.set()
        for pr in procs:
            pr.join(timeout=60)
    assert all(pr.exitcode == 0 for pr in procs)
