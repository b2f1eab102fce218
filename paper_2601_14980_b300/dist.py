"""Host-side helpers for running the path on several GPUs, one process each.

The path shards without a data-path exchange: every element's encryption,
aggregation and decryption is independent, so each rank takes its own
elements.  A rank's element i is the global element ``start + i``; the
Philox counter of its randomness is that global index (the ``e0`` of
pc2_encrypt), so the union of the ranks' ciphertexts is exactly the
single-process encryption of the whole vector.  The only collective is the
max over ranks of the measured time.

Failure detection (host side): in every round of Algorithm 1 the master
needs each edge node's segment.  Edge processes announce a segment with
post_segment; the master's missing_segments waits a bounded time and names
the nodes whose segment has not arrived, which it then marks absent in the
library (pc2_admm_set_node_present) so that the round is refused instead of
computed on stale data."""
from __future__ import annotations

import os
import time


def rank_world() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced share of `total` elements: (first global index, count)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def max_over_ranks(values, device=None):
    """Element-wise max of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def _seg_key(round_: int, node: int) -> str:
    return "pc2/segment/%d/%d" % (round_, node)


def post_segment(store, round_: int, node: int) -> None:
    """Edge node `node` announces its segment of round `round_` (a key in a
    torch.distributed Store shared with the master)."""
    store.set(_seg_key(round_, node), b"1")


def missing_segments(store, round_: int, nodes, timeout_s: float, poll_s: float = 0.01) -> list:
    """Master side: waits at most `timeout_s` seconds for every node in
    `nodes` to announce its segment of round `round_`; returns the nodes whose
    segment is still missing (empty when all arrived)."""
    deadline = time.monotonic() + timeout_s
    pending = set(int(k) for k in nodes)
    while pending:
        pending = {k for k in pending if not store.check([_seg_key(round_, k)])}
        if not pending or time.monotonic() >= deadline:
            break
        time.sleep(poll_s)
    return sorted(pending)
