"""GPU parity tests of Alg. 2's local MSD pass (rs_msd_partition_ex) and of
the multi-rank sort's local steps (partition.py, GpuOps) against the CPU
oracle, bit for bit.

rs_msd_partition_ex must equal the oracle's one counting-sort pass by byte 3
(keys and values), and its bucket offsets the oracle's exclusive prefix of
the byte-3 histogram.  The multi-rank sort is run at one rank through
partition_sort_pairs, and at two and three ranks on this one GPU with the
exchange done by host-side slicing in place of the all-to-all (the ranks'
GPU work is exactly that of a real run; only the transport differs).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs
from tests.gpu_util import oracle_sort, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


def _oracle_msd(k, v):
    ko, vo = oracle.counting_pass(k, v, 3)
    g = oracle.exclusive_prefix(oracle.digit_histograms(k))[3].astype(np.int64)
    return ko, vo, np.concatenate([g, [k.size]])


@pytest.mark.parametrize("n", [1, 33, 4097, 70_001, 1_000_003, (1 << 24) + 3])
@pytest.mark.parametrize("dist_name", ["uniform", "and4", "equal", "low16"])
def test_msd_partition_matches_oracle(rs, n, dist_name):
    import torch
    k = inputs.keys(dist_name, n, seed=400 + n % 89)
    v = inputs.splitmix32(401, n, 2)
    kd, vd = to_dev(k), to_dev(v)
    ok, ov = torch.empty_like(kd), torch.empty_like(vd)
    off = torch.empty(257, dtype=torch.int32, device="cuda")
    ws = rs.alloc_workspace(n, True)
    rs.msd_partition_ex(kd, vd, ok, ov, off, ws)
    rs.check_stream()
    ko, vo, go = _oracle_msd(k, v)
    assert np.array_equal(to_host(ok), ko)
    assert np.array_equal(to_host(ov), vo)
    assert np.array_equal(to_host(off).astype(np.int64), go)
    # The inputs are untouched.
    assert np.array_equal(to_host(kd), k) and np.array_equal(to_host(vd), v)


@pytest.mark.parametrize("off_elems", [1, 3])
def test_msd_partition_keys_only_unaligned(rs, off_elems):
    import torch
    n = 123_457
    k = inputs.keys("and2", n, seed=410)
    kd = to_dev(k, off_elems)
    out = to_dev(np.zeros(n, dtype=np.uint32), off_elems)
    off = torch.empty(257, dtype=torch.int32, device="cuda")
    ws = rs.alloc_workspace(n, False)
    rs.msd_partition_ex(kd, None, out, None, off, ws)
    rs.check_stream()
    ko, _, go = _oracle_msd(k, None)
    assert np.array_equal(to_host(out), ko)
    assert np.array_equal(to_host(off).astype(np.int64), go)


def test_msd_partition_argument_errors(rs):
    import torch
    n = 1000
    kd = to_dev(np.zeros(n, dtype=np.uint32))
    off = torch.empty(257, dtype=torch.int32, device="cuda")
    ws = rs.alloc_workspace(n, True)
    with pytest.raises(rs.RsError):  # output overlapping the input
        rs.msd_partition_ex(kd, None, kd, None, off, ws)
    with pytest.raises(ValueError):  # offsets of the wrong length
        rs.msd_partition_ex(kd, None, torch.empty_like(kd), None, off[:256], ws)


def test_partition_sort_one_rank(rs):
    from paper_1008_2849_gb300.partition import GpuOps, partition_sort_pairs
    n = 3_000_001
    k = inputs.keys("uniform", n, seed=420)
    v = inputs.index_values(n)
    rk, rv, bounds = partition_sort_pairs(to_dev(k), to_dev(v), GpuOps())
    ko, vo = oracle_sort(k, v)
    assert list(bounds) == [0, 256]
    assert np.array_equal(to_host(rk), ko) and np.array_equal(to_host(rv), vo)


@pytest.mark.parametrize("world,dist_name", [(2, "uniform"), (3, "and4"), (3, "low16")])
def test_partition_sort_ranks_on_one_gpu(rs, world, dist_name):
    """The GPU steps of a world-rank run (MSD pass per shard, ranges, exchange
    by slices, local sorts), their concatenation against the oracle."""
    import torch

    from paper_1008_2849_gb300.partition import GpuOps, assign_ranges, exchange_counts
    n = 2_000_003
    k = inputs.keys(dist_name, n, seed=430 + world)
    v = inputs.index_values(n)
    cuts = np.linspace(0, n, world + 1).astype(np.int64)
    ops = GpuOps()
    parts = [ops.msd_partition(to_dev(k[cuts[r]:cuts[r + 1]]), to_dev(v[cuts[r]:cuts[r + 1]]))
             for r in range(world)]
    hists = np.stack([np.diff(p[2]) for p in parts])
    bounds = assign_ranges(hists.sum(0), world)
    out_k, out_v = [], []
    for d in range(world):
        pieces_k, pieces_v = [], []
        for s in range(world):
            send = exchange_counts(hists, bounds, s)[0]
            start = int(sum(send[:d]))
            pieces_k.append(parts[s][0][start:start + send[d]])
            pieces_v.append(parts[s][1][start:start + send[d]])
        rk, rv = torch.cat(pieces_k), torch.cat(pieces_v)
        ops.sort(rk, rv)
        out_k.append(to_host(rk))
        out_v.append(to_host(rv))
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(np.concatenate(out_k), ko)
    assert np.array_equal(np.concatenate(out_v), vo)
