"""Alg. 2's reverse sorting across ranks: the sort of one array held in shards
by several processes (one per GPU), the multi-GPU form of the method.

Sec. 4 (Alg. 2) has every processing element sort its share by the most
significant digit first, exchange bucket sizes, and then sort a contiguous
range of MSD buckets on its own with the LSD passes.  Here every rank holds
one shard of the global array of (uint32 key, uint32 value) pairs, in global
order (rank r's shard follows rank r-1's):

1. every rank partitions its shard stably by the top byte of the key (one
   counting-sort pass, rs_msd_partition_ex) and so learns its 256 bucket
   sizes;
2. the bucket sizes of all ranks are gathered (one all_gather);
3. the 256 buckets are cut into `world` contiguous ranges balanced by item
   count (assign_ranges; the same computation on every rank);
4. the items of range d are sent to rank d (one all_to_all with per-rank
   counts).  After step 1 they are one contiguous slice of the partitioned
   shard.  Rank d receives the slices of ranks 0, 1, ... in that order, each
   in its local input order, so equal keys keep their global input order;
5. every rank sorts what it received (stable, all four digits);
6. the ranks' results, concatenated in rank order, are the stable ascending
   sort of the global array.

A bucket is never split across ranks (its items are not yet ordered by the
lower digits), so keys concentrated in few top-byte values leave the ranks
unevenly loaded, as Sec. 4 notes for skewed inputs.

The local steps are an object with three methods (see GpuOps): msd_partition,
sort, and empty (a receive buffer).  The exchange uses torch.distributed: NCCL
between GPUs, or gloo for tests on the CPU.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

RADIX = 256


def assign_ranges(counts: Sequence[int], world: int) -> np.ndarray:
    """Cut the buckets 0..255 into `world` contiguous ranges balanced by
    count: bounds[r] .. bounds[r+1] is rank r's range (possibly empty).
    Each cut is placed at the bucket boundary nearest to the ideal share
    r * total / world, never before the previous cut."""
    counts = np.asarray(counts, dtype=np.int64)
    if counts.shape != (RADIX,):
        raise ValueError("counts must hold 256 bucket sizes")
    if world < 1:
        raise ValueError("world must be at least 1")
    cum = np.concatenate([[0], np.cumsum(counts)])
    total = int(cum[-1])
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        b = int(np.searchsorted(cum, target, side="left"))  # first boundary at or past target
        if b > 0 and target - cum[b - 1] <= cum[b] - target:
            b -= 1
        bounds.append(min(max(b, bounds[-1]), RADIX))
    bounds.append(RADIX)
    return np.asarray(bounds, dtype=np.int64)


def exchange_counts(hists: np.ndarray, bounds: np.ndarray, rank: int) -> Tuple[List[int], List[int]]:
    """Items rank `rank` sends to every rank, and receives from every rank,
    given every rank's bucket sizes hists[world][256] and the ranges."""
    world = hists.shape[0]
    send = [int(hists[rank, bounds[d]:bounds[d + 1]].sum()) for d in range(world)]
    recv = [int(hists[s, bounds[rank]:bounds[rank + 1]].sum()) for s in range(world)]
    return send, recv


def partition_sort_pairs(keys, vals, ops, group=None):
    """Sort the global array whose shard this rank holds (keys, vals: 1-D
    tensors of 32-bit words on the device `ops` works on).  Returns this
    rank's part of the sorted array (keys, values) and the bucket ranges."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    kp, vp, offsets = ops.msd_partition(keys, vals)
    local = np.diff(np.asarray(offsets, dtype=np.int64))
    if world == 1:
        hists = local[None, :]
    else:
        mine = torch.as_tensor(local, dtype=torch.int64, device=kp.device)
        everyone = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(everyone, mine, group=group)
        hists = np.stack([t.cpu().numpy() for t in everyone])
    bounds = assign_ranges(hists.sum(axis=0), world)
    send, recv = exchange_counts(hists, bounds, rank)
    if world == 1:
        rk, rv = kp, vp
    else:
        rk = ops.empty(sum(recv), like=kp)
        rv = ops.empty(sum(recv), like=vp)
        dist.all_to_all_single(rk, kp, recv, send, group=group)
        dist.all_to_all_single(rv, vp, recv, send, group=group)
    ops.sort(rk, rv)
    return rk, rv, bounds


class GpuOps:
    """The local steps on this rank's GPU through librs.so."""

    def __init__(self, device=None):
        import torch

        from paper_1008_2849_gb300 import rs
        self.torch, self.rs = torch, rs
        self.device = torch.device("cuda") if device is None else torch.device(device)

    def empty(self, n: int, like):
        return self.torch.empty(n, dtype=like.dtype, device=like.device)

    def msd_partition(self, keys, vals):
        torch, rs = self.torch, self.rs
        out_k, out_v = torch.empty_like(keys), torch.empty_like(vals)
        offsets = torch.empty(RADIX + 1, dtype=torch.int32, device=keys.device)
        ws = rs.alloc_workspace(keys.numel(), True, device=keys.device)
        rs.msd_partition_ex(keys, vals, out_k, out_v, offsets, ws)
        rs.check_stream()
        return out_k, out_v, offsets.cpu().numpy().view(np.uint32).astype(np.int64)

    def sort(self, keys, vals):
        if keys.numel():
            ws = self.rs.alloc_workspace(keys.numel(), True, device=keys.device)
            self.rs.sort_pairs_ex(keys, vals, ws)
