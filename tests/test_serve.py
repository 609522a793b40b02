"""Tests of the serving loop.

CPU part: a fake executor sorts with the CPU oracle and completes work after
a fixed number of polls, so admission, batching and the memory budget can be
checked without a GPU.  GPU part (marked gpu): the real executor; every
request's result must equal the oracle's sort of that request alone, however
requests were batched.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs
from paper_1008_2849_gb300.serve import (Request, SerialServer, SortServer, host_keys,
                                         make_requests)

POOL_N = 1 << 20


class FakeExecutor:
    """Sorts on the host with the oracle; a launch completes after `delay`
    polls.  Records the bytes it was asked to hold."""

    def __init__(self, delay=3):
        self.delay = delay
        self.launched = []

    def bytes_for(self, sizes, with_values, segmented):
        n = sum(sizes)
        return n * (8 if with_values else 4) * 2 + 1024

    def launch(self, reqs, segmented):
        self.launched.append([r.id for r in reqs])
        out = []
        for r in reqs:
            k = host_keys(r, POOL_N)
            v = inputs.index_values(r.n) if r.with_values else None
            if segmented:
                off = np.array([0, r.n], dtype=np.uint32)
                ko, vo = oracle.sort_pairs_segmented(k, v, off)
            else:
                ko, vo = oracle.sort_pairs(k, v)
            out.append((ko, vo))
        return {"left": self.delay, "out": out}

    def poll(self, h):
        h["left"] -= 1
        return h["left"] <= 0

    def take(self, h, keep):
        return h["out"] if keep else [(None, None)] * len(h["out"])

    def check(self):
        pass


def _reqs(num, seed, lo=2.0, hi=4.5):
    return make_requests(num, seed, lo, hi)


def test_every_result_is_its_own_sort_cpu():
    reqs = _reqs(60, 3)
    ex = FakeExecutor()
    srv = SortServer(ex, budget_bytes=10**9, max_inflight=4, small_max=2000, batch_items=5000,
                     keep_results=True)
    res = srv.run(reqs, realtime=False)
    assert len(res["done"]) == len(reqs)
    for d in res["done"]:
        r = d.request
        k = host_keys(r, POOL_N)
        v = inputs.index_values(r.n) if r.with_values else None
        ko, vo = oracle.sort_pairs(k, v)
        assert np.array_equal(d.keys, ko)
        if r.with_values:
            assert np.array_equal(d.vals, vo)
    # Small requests were coalesced; batches never mix keys-only with pairs.
    by_id = {r.id: r for r in reqs}
    assert any(len(b) > 1 for b in ex.launched)
    for b in ex.launched:
        assert len({by_id[i].with_values for i in b}) == 1


def test_completion_callback_sees_every_result_cpu():
    """on_done receives every request once, with its result; the returned
    list then keeps requests and latencies only (results are not retained)."""
    reqs = _reqs(40, 5)
    seen = {}

    def on_done(d):
        r = d.request
        assert r.id not in seen
        k = host_keys(r, POOL_N)
        v = inputs.index_values(r.n) if r.with_values else None
        ko, vo = oracle.sort_pairs(k, v)
        assert np.array_equal(d.keys, ko)
        if r.with_values:
            assert np.array_equal(d.vals, vo)
        seen[r.id] = d.batch

    srv = SortServer(FakeExecutor(), budget_bytes=10**9, max_inflight=4, small_max=2000,
                     batch_items=5000, keep_results=True, on_done=on_done)
    res = srv.run(reqs, realtime=False)
    assert sorted(seen) == sorted(r.id for r in reqs)
    assert all(d.keys is None and d.vals is None for d in res["done"])
    assert {d.request.id: d.batch for d in res["done"]} == seen


def test_budget_is_never_exceeded_cpu():
    reqs = _reqs(80, 4, 2.0, 4.0)
    ex = FakeExecutor(delay=5)
    budget = 200_000
    srv = SortServer(ex, budget_bytes=budget, max_inflight=8, small_max=3000, batch_items=8000)
    res = srv.run(reqs, realtime=False)
    assert res["peak_bytes"] <= budget
    assert len(res["done"]) == len(reqs)


def test_oversized_request_is_refused_cpu():
    reqs = [Request(0, 10_000, True, "uniform", 1)]
    srv = SortServer(FakeExecutor(), budget_bytes=1000, small_max=100)
    with pytest.raises(MemoryError):
        srv.run(reqs, realtime=False)


def test_oversized_small_request_is_refused_cpu():
    """A small request that alone needs more than the budget, with nothing in
    flight, raises instead of waiting forever."""
    reqs = [Request(0, 50, True, "uniform", 1)]
    srv = SortServer(FakeExecutor(), budget_bytes=1000, small_max=100)
    with pytest.raises(MemoryError):
        srv.run(reqs, realtime=False)


def test_small_batch_shrinks_to_fit_budget_cpu():
    """When a whole batch of small requests does not fit the budget, its
    longest prefix that fits is launched, and the rest follow later."""
    reqs = [Request(i, 1000, False, "uniform", i + 1) for i in range(6)]
    ex = FakeExecutor(delay=2)
    one = ex.bytes_for([1000], False, True)
    budget = ex.bytes_for([1000, 1000], False, True) + one // 2  # two at once, not three
    srv = SortServer(ex, budget_bytes=budget, max_inflight=8, small_max=2000,
                     batch_items=10_000, keep_results=True)
    res = srv.run(reqs, realtime=False)
    assert len(res["done"]) == len(reqs)
    assert res["peak_bytes"] <= budget
    assert [len(b) for b in ex.launched][0] == 2
    assert sorted(i for b in ex.launched for i in b) == list(range(6))
    for d in res["done"]:
        ko, _ = oracle.sort_pairs(host_keys(d.request, POOL_N), None)
        assert np.array_equal(d.keys, ko)


def test_admission_order_cpu():
    """Requests are admitted in arrival order (a large request at the head
    is not overtaken by later ones)."""
    reqs = [Request(0, 50_000, False, "uniform", 1), Request(1, 10, False, "uniform", 2),
            Request(2, 60_000, True, "and2", 3)]
    ex = FakeExecutor()
    SortServer(ex, budget_bytes=10**9, small_max=100).run(reqs, realtime=False)
    assert [b[0] for b in ex.launched] == [0, 1, 2]


@pytest.mark.gpu
def test_gpu_results_alone_and_in_the_mix():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300.serve import GpuExecutor
    reqs = make_requests(120, 5, 2.0, 5.5)
    srv = SortServer(GpuExecutor(streams=3, pool_n=POOL_N), budget_bytes=2 * 10**9,
                     max_inflight=6, small_max=1 << 14, batch_items=1 << 16, keep_results=True)
    res = srv.run(reqs, realtime=False)
    assert len(res["done"]) == len(reqs)
    assert any(d.batch > 1 for d in res["done"])
    for d in res["done"]:
        r = d.request
        k = host_keys(r, POOL_N)
        v = inputs.index_values(r.n) if r.with_values else None
        ko, vo = oracle.sort_pairs(k, v)
        assert np.array_equal(d.keys.cpu().numpy().view(np.uint32), ko), r.id
        if r.with_values:
            assert np.array_equal(d.vals.cpu().numpy().view(np.uint32), vo), r.id
    # The serial baseline sorts the same requests one by one.
    ser = SerialServer(GpuExecutor(streams=1, pool_n=POOL_N)).run(reqs[:20], realtime=False)
    assert ser["items_per_s"] > 0


def _host_results_and_peak(srv, reqs, realtime):
    """Run `srv`, copying every result to the host as it completes (so no
    device result outlives its launch); returns (results by id, run stats,
    the allocator's peak bytes above its level at the start)."""
    import torch
    got = {}

    def on_done(d):
        k = d.keys.cpu().numpy().view(np.uint32).copy()
        v = None if d.vals is None else d.vals.cpu().numpy().view(np.uint32).copy()
        got[d.request.id] = (k, v)

    srv.on_done = on_done
    srv.keep = True
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    res = srv.run(reqs, realtime=realtime)
    peak = torch.cuda.max_memory_allocated() - base
    return got, res, peak


def _check_against_oracle(reqs, got):
    from tests.gpu_util import oracle_sort
    for r in reqs:
        k = host_keys(r, POOL_N)
        v = inputs.index_values(r.n) if r.with_values else None
        ko, vo = oracle_sort(k, v)
        gk, gv = got[r.id]
        assert np.array_equal(gk, ko), r.id
        if r.with_values:
            assert np.array_equal(gv, vo), r.id


@pytest.mark.gpu
def test_gpu_allocator_peak_within_budget():
    """The device memory the allocator actually hands out while serving stays
    within the server's budget, and the budget is what limits admission."""
    from paper_1008_2849_gb300.serve import GpuExecutor
    reqs = make_requests(150, 6, 3.0, 6.0)
    ex = GpuExecutor(streams=3, pool_n=POOL_N)
    largest = max(ex.bytes_for([r.n], r.with_values, False) for r in reqs)
    budget = 3 * largest
    srv = SortServer(ex, budget_bytes=budget, max_inflight=16, small_max=1 << 14,
                     batch_items=1 << 17)
    got, res, peak = _host_results_and_peak(srv, reqs, realtime=False)
    assert len(res["done"]) == len(reqs)
    assert res["peak_bytes"] <= budget
    assert peak <= budget, (peak, budget)
    _check_against_oracle(reqs, got)
    # Key-value requests of nearly equal size (each launched alone) under a
    # budget of three of them: the budget, not the 16 slots, bounds the
    # launches in flight, and the allocator stays within it.
    sizes = 900_000 + (inputs.splitmix32(8, 40, 0) % np.uint32(100_000)).astype(np.int64)
    reqs = [Request(i, int(m), True, "uniform", 100 + i) for i, m in enumerate(sizes)]
    largest = max(ex.bytes_for([r.n], r.with_values, False) for r in reqs)
    budget = 3 * largest
    srv = SortServer(ex, budget_bytes=budget, max_inflight=16, small_max=1 << 14)
    got, res, peak = _host_results_and_peak(srv, reqs, realtime=False)
    log = res["launch_log"]
    inflight = max(sum(1 for a, b, _ in log if a <= t < b) for t, _, _ in log)
    assert 2 <= inflight <= 3, inflight
    assert peak <= budget, (peak, budget)
    _check_against_oracle(reqs, got)


@pytest.mark.gpu
def test_gpu_realtime_arrivals_overlap():
    """Poisson arrivals in real time: requests are admitted while earlier
    ones are still on the GPU (a launch starts before an earlier launch is
    seen complete), and every result equals the oracle's sort of that
    request alone."""
    from paper_1008_2849_gb300.serve import GpuExecutor
    reqs = make_requests(200, 7, 3.5, 6.0, rate_per_s=4000.0)
    ex = GpuExecutor(streams=4, pool_n=POOL_N)
    srv = SortServer(ex, budget_bytes=4 * 10**9, max_inflight=8, small_max=1 << 14,
                     batch_items=1 << 17)
    got, res, peak = _host_results_and_peak(srv, reqs, realtime=True)
    assert len(res["done"]) == len(reqs)
    log = res["launch_log"]
    assert all(b is not None for _, b, _ in log)
    overlapped = sum(1 for j in range(1, len(log)) if any(log[i][1] > log[j][0] for i in range(j)))
    assert overlapped > 0, log[:10]
    assert peak <= srv.budget
    _check_against_oracle(reqs, got)
