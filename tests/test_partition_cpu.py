"""The multi-rank sort of Alg. 2 (partition.py) on CPU: gloo ranks, the CPU
oracle as every rank's local step (its one-pass counting sort by the top
byte, and its full sort), and torch.distributed for the gather of bucket
sizes and the exchange of the items.

The ranks' results, concatenated in rank order, must equal the oracle's
stable sort of the whole array bit for bit (keys, and values = input index,
so stability shows), at world sizes 2 and 3, with shards of unequal length
and key distributions that put everything in one bucket or skew the buckets.
The range assignment is also checked on its own.
"""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1008_2849_gb300 import inputs
from paper_1008_2849_gb300.partition import assign_ranges, exchange_counts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleOps:
    """Local steps by the CPU oracle on CPU tensors of 32-bit words."""

    @staticmethod
    def empty(n, like):
        return torch.empty(n, dtype=like.dtype)

    @staticmethod
    def msd_partition(keys, vals):
        k = keys.numpy().view(np.uint32)
        v = vals.numpy().view(np.uint32)
        ko, vo = oracle.counting_pass(k, v, 3)
        g = oracle.exclusive_prefix(oracle.digit_histograms(k))[3].astype(np.int64)
        offsets = np.concatenate([g, [k.size]])
        return (torch.from_numpy(ko.view(np.int32).copy()), torch.from_numpy(vo.view(np.int32).copy()),
                offsets)

    @staticmethod
    def sort(keys, vals):
        ko, vo = oracle.sort_pairs(keys.numpy().view(np.uint32), vals.numpy().view(np.uint32))
        keys.copy_(torch.from_numpy(ko.view(np.int32)))
        vals.copy_(torch.from_numpy(vo.view(np.int32)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _global_input(dist_name: str, n: int, seed: int):
    return inputs.keys(dist_name, n, seed=seed), inputs.index_values(n)


def _shard_bounds(n: int, world: int):
    # Unequal shards: rank r holds a share proportional to r + 1.
    w = np.arange(1, world + 1, dtype=np.float64)
    cuts = np.floor(np.cumsum(w) / w.sum() * n).astype(np.int64)
    return np.concatenate([[0], cuts])


def _rank_main(rank, world, port, out_dir, dist_name, n, seed):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_1008_2849_gb300.partition import partition_sort_pairs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        k, v = _global_input(dist_name, n, seed)
        sb = _shard_bounds(n, world)
        ks = torch.from_numpy(k[sb[rank]:sb[rank + 1]].view(np.int32).copy())
        vs = torch.from_numpy(v[sb[rank]:sb[rank + 1]].view(np.int32).copy())
        rk, rv, bounds = partition_sort_pairs(ks, vs, OracleOps())
        np.save(os.path.join(out_dir, "k%d.npy" % rank), rk.numpy().view(np.uint32))
        np.save(os.path.join(out_dir, "v%d.npy" % rank), rv.numpy().view(np.uint32))
        np.save(os.path.join(out_dir, "b%d.npy" % rank), bounds)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dist_name,n", [(2, "uniform", 50_001), (3, "uniform", 70_003),
                                              (2, "and4", 40_000), (3, "and4", 33_333),
                                              (3, "equal", 9_000), (2, "low16", 20_000),
                                              (3, "distinct256", 30_000)])
def test_partition_sort_equals_oracle_gloo(tmp_path, world, dist_name, n):
    seed = 900 + n % 97
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), dist_name, n, seed),
                       nprocs=world, start_method="spawn", join=True)
    k, v = _global_input(dist_name, n, seed)
    ko, vo = oracle.sort_pairs(k, v)
    got_k = np.concatenate([np.load(tmp_path / ("k%d.npy" % r)) for r in range(world)])
    got_v = np.concatenate([np.load(tmp_path / ("v%d.npy" % r)) for r in range(world)])
    assert np.array_equal(got_k, ko)
    assert np.array_equal(got_v, vo)
    # Every rank computed the same ranges, and rank r holds exactly the keys
    # whose top byte lies in its range.
    b0 = np.load(tmp_path / "b0.npy")
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / ("b%d.npy" % r)), b0)
        top = np.load(tmp_path / ("k%d.npy" % r)) >> np.uint32(24)
        assert np.all((top >= b0[r]) & (top < b0[r + 1]))


def test_assign_ranges_properties():
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 5, 8, 17, 256, 300):
        for trial in range(20):
            kind = trial % 4
            if kind == 0:
                counts = rng.integers(0, 1000, 256)
            elif kind == 1:
                counts = np.zeros(256, dtype=np.int64)
                counts[rng.integers(0, 256)] = 12345  # one bucket holds everything
            elif kind == 2:
                counts = np.zeros(256, dtype=np.int64)  # nothing at all
            else:
                counts = (rng.pareto(1.0, 256) * 100).astype(np.int64)  # skewed
            b = assign_ranges(counts, world)
            assert b.shape == (world + 1,) and b[0] == 0 and b[-1] == 256
            assert np.all(np.diff(b) >= 0)  # contiguous, in order, possibly empty
            # Every cut is within one bucket's size of its ideal share.
            cum = np.concatenate([[0], np.cumsum(counts)])
            total = cum[-1]
            for r in range(1, world):
                ideal = total * r / world
                lo = cum[b[r]]
                step = counts.max() if counts.size else 0
                assert abs(lo - ideal) <= step + 1e-9 or b[r] == b[r - 1]
    # Uniform buckets split evenly.
    assert list(assign_ranges(np.ones(256, dtype=np.int64), 4)) == [0, 64, 128, 192, 256]


def test_exchange_counts_balance():
    rng = np.random.default_rng(6)
    for world in (2, 3, 4):
        hists = rng.integers(0, 50, (world, 256))
        b = assign_ranges(hists.sum(0), world)
        sends = [exchange_counts(hists, b, r)[0] for r in range(world)]
        recvs = [exchange_counts(hists, b, r)[1] for r in range(world)]
        # What s sends to d is what d receives from s; nothing is lost.
        for s in range(world):
            for d in range(world):
                assert sends[s][d] == recvs[d][s]
            assert sum(sends[s]) == hists[s].sum()
        assert sum(map(sum, recvs)) == hists.sum()
