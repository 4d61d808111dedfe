"""The exchange step of a database sharded over several GPUs.

One process per GPU (torch.distributed; NCCL on GPUs, gloo on CPU).  Every
rank holds one shard of the database (sw_shard_plan, the same partition on
every rank) and searches the full query batch against it, keeping its own
top-k.  The shards then exchange only those lists: an all-gather of
n_q x top_k (score, shard-local index) per rank, a few KB per query, after
which sw_hits_merge gives the unsharded top-k (the paper leaves multi-GPU
execution to future work, Section 5).  Nothing else crosses between GPUs:
each rank reads only its own HBM.
"""
from __future__ import annotations

import numpy as np

from . import binding


def hits_to_tensor(hits, device=None):
    """HIT_DTYPE [n_q, top_k] (host) -> int64 tensor [n_q, top_k, 2] (score, index)."""
    import torch
    t = torch.empty((hits.shape[0], hits.shape[1], 2), dtype=torch.int64)
    t[:, :, 0] = torch.from_numpy(hits["score"].astype(np.int64))
    t[:, :, 1] = torch.from_numpy(hits["db_index"].astype(np.int64))
    return t.to(device) if device is not None else t


def tensor_to_hits(t) -> np.ndarray:
    """int64 [..., top_k, 2] tensor in the sw_hit memory layout (sw_search's
    device output viewed as int64 pairs, or hits_to_tensor's) -> HIT_DTYPE."""
    a = t.cpu().numpy()
    out = np.empty(a.shape[:-1], dtype=binding.HIT_DTYPE)
    out["score"] = (a[..., 0] & 0xffffffff).astype(np.uint32).astype(np.int32)
    out["reserved"] = 0
    out["db_index"] = a[..., 1]
    return out


def exchange_hits(dist, local_hits, members, member_offsets, top_k: int, dst: int | None = None):
    """All-gather every rank's shard-local top-k (int64 tensor [n_q, top_k, 2]
    in the sw_hit layout: the device output of sw_search, or hits_to_tensor's)
    and merge them into the unsharded top-k with sw_hits_merge.

    dist is torch.distributed with an initialised process group whose world
    size equals the number of shards; rank r holds shard r.  Returns the
    merged HIT_DTYPE [n_q, top_k] on every rank (dst=None), or on rank dst
    only (None elsewhere)."""
    world = dist.get_world_size()
    if len(member_offsets) != world + 1:
        raise ValueError("one shard per rank: member_offsets must have world_size + 1 entries")
    gathered = [local_hits.new_empty(local_hits.shape) for _ in range(world)]
    dist.all_gather(gathered, local_hits.contiguous())
    if dst is not None and dist.get_rank() != dst:
        return None
    import torch
    shard_hits = tensor_to_hits(torch.stack([g.cpu() for g in gathered]))
    return binding.sw_hits_merge(shard_hits, members, member_offsets, top_k)
