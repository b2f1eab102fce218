"""Host-side helpers for running the path on several GPUs, one process each.

The path shards without a data-path exchange: every element's encryption,
aggregation and decryption is independent, so each rank takes its own
elements.  A rank's element i is the global element ``start + i``; the
Philox counter of its randomness is that global index (the ``e0`` of
pc2_encrypt), so the union of the ranks' ciphertexts is exactly the
single-process encryption of the whole vector.  The only collective is the
max over ranks of the measured time."""
from __future__ import annotations

import os


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
