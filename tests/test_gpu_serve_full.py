"""The serving workload at full size (20 000 requests, 70 % keys only and 30 %
key-value, sizes floor(10^U) with U uniform on [3, 8], uniform or AND-of-2
keys, seed 11), all present at time 0, under the 60 GB budget, checked as it
is served:

* every request: invariants on the device -- keys nondecreasing; with values,
  the values a permutation of 0..n-1, each key the input key at its value,
  equal keys in input order; keys only, the same multiset as the input
  (compared with torch's own sort of the input);
* every request of at most 10^6 items, and a seeded 5 % sample of the larger
  ones: bit for bit against the CPU oracle.

It takes a minute or two; it is part of the GPU suite (RS_SKIP_FULL_CHECKS=1
leaves it out of a quick run)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs
from paper_1008_2849_gb300.serve import SortServer, host_keys, make_requests, pool_window

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("RS_SKIP_FULL_CHECKS") == "1",
                                 reason="full-size checks skipped: RS_SKIP_FULL_CHECKS=1")]


def _sampled(rid: int) -> bool:
    return int(inputs.splitmix32(12, 1, 0, start=rid)[0]) % 20 == 0


def test_serving_workload_full():
    import torch
    from paper_1008_2849_gb300.serve import GpuExecutor
    ex = GpuExecutor(streams=4)
    reqs = make_requests(20000, 11)
    stats = {"requests": 0, "items": 0, "oracle_checked": 0, "oracle_items": 0,
             "invariants_checked": 0}
    mask = 0xFFFFFFFF

    def check(d):
        r = d.request
        k = d.keys.to(torch.int64) & mask
        assert bool((k[1:] >= k[:-1]).all()), r.id
        o = pool_window(r, ex.pool_n)
        src = ex.pool[r.dist][o:o + r.n].to(torch.int64) & mask
        if r.with_values:
            v = d.vals.to(torch.int64)
            assert bool(((v >= 0) & (v < r.n)).all()), r.id   # before any indexing by v
            seen = torch.zeros(r.n, dtype=torch.bool, device=v.device)
            seen[v] = True
            assert bool(seen.all()), r.id
            assert bool((src[v] == k).all()), r.id
            same = k[1:] == k[:-1]
            assert bool((v[1:][same] > v[:-1][same]).all()), r.id
        else:
            assert bool((torch.sort(src).values == k).all()), r.id
        stats["invariants_checked"] += 1
        if r.n <= 10**6 or _sampled(r.id):
            hk = host_keys(r, ex.pool_n)
            hv = inputs.index_values(r.n) if r.with_values else None
            if r.n > (1 << 22):
                ko, vo = oracle.sort_pairs_threaded(hk, hv, os.cpu_count() or 4)
            else:
                ko, vo = oracle.sort_pairs(hk, hv)
            assert np.array_equal(d.keys.cpu().numpy().view(np.uint32), ko), r.id
            if r.with_values:
                assert np.array_equal(d.vals.cpu().numpy().view(np.uint32), vo), r.id
            stats["oracle_checked"] += 1
            stats["oracle_items"] += r.n
        stats["requests"] += 1
        stats["items"] += r.n

    srv = SortServer(ex, budget_bytes=60 * 10**9, max_inflight=8, keep_results=True,
                     on_done=check)
    res = srv.run(reqs, realtime=False)
    assert stats["requests"] == len(reqs) and len(res["done"]) == len(reqs)
    assert res["peak_bytes"] <= 60 * 10**9
    print("serving workload verified:", stats, "peak_bytes", res["peak_bytes"])
