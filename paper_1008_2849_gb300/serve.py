"""Continuous-batching sort server on one GPU.

Requests (sort n uint32 keys, optionally with uint32 values) arrive over time.
The server admits them in arrival order as long as the device-memory budget
and the number of work items in flight allow, keeps their buffers resident on
the device, and runs them on a pool of CUDA streams so that admitted work
overlaps on the GPU:

* a request of at most ``small_max`` items joins a batch of its kind (keys
  only, or key-value); a batch is launched as ONE segmented sort
  (rs_sort_*_segmented_ex) once it holds ``batch_items`` items, or as soon as
  no further small request of its kind is waiting;
* a larger request is launched alone (rs_sort_*_ex).

A request's latency runs from its arrival to the moment the server sees its
sort complete on the device (its CUDA event has fired).  The sort of a
request never depends on which other requests share its batch: every segment
is sorted on its own (tests check each result alone and in the mix).

The work itself is done by an executor: ``GpuExecutor`` (the library's CUDA
kernels through the C ABI; PyTorch only supplies memory, streams and events),
or any object with the same methods (the CPU tests use a fake one).
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    id: int
    n: int
    with_values: bool
    dist: str
    key_seed: int
    arrival: float = 0.0  # seconds after the start of the run


@dataclasses.dataclass
class Done:
    request: Request
    latency: float
    batch: int                      # requests that shared the launch
    keys: object = None             # sorted keys (kept only with keep_results)
    vals: object = None


POOL_SEED = 2011


def pool_window(r: Request, pool_n: int) -> int:
    """First pool index of request r's keys (a seeded, deterministic window)."""
    return (r.key_seed * 2654435761) % (pool_n - r.n + 1)


def host_keys(r: Request, pool_n: int) -> np.ndarray:
    """Request r's keys, drawn on the host (for checks against the oracle)."""
    from paper_1008_2849_gb300 import inputs
    o = pool_window(r, pool_n)
    k = inputs.splitmix32(POOL_SEED, r.n, 0, start=o)
    if r.dist == "and2":
        k &= inputs.splitmix32(POOL_SEED, r.n, 1, start=o)
    return k


class GpuExecutor:
    """Runs admitted work through librs.so on a pool of CUDA streams.

    A request's keys are a seeded window of a key pool drawn once on the
    device (uniform words, and their AND with a second stream for ``and2``);
    copying the window into the request's own buffer stands in for the
    payload upload.  Values are the index inside the request."""

    def __init__(self, streams: int = 4, device: int = 0, pool_n: int = 1 << 27):
        import torch

        from paper_1008_2849_gb300 import build, inputs, rs
        build.build_library()
        self.torch, self.inputs, self.rs = torch, inputs, rs
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.next_stream = 0
        self.pool_n = pool_n
        u = inputs.splitmix32_torch(POOL_SEED, pool_n, 0, device=self.device)
        a = inputs.splitmix32_torch(POOL_SEED, pool_n, 1, device=self.device).bitwise_and_(u)
        self.pool = {"uniform": u, "and2": a}
        torch.cuda.synchronize(self.device)

    # -- sizes ---------------------------------------------------------------
    def bytes_for(self, sizes: List[int], with_values: bool, segmented: bool) -> int:
        """Device bytes that launch() allocates for this work: keys, values,
        the segment table and the workspace, each rounded up to the 512-byte
        blocks of PyTorch's caching allocator."""
        def block(b):
            return (int(b) + 511) // 512 * 512
        n = int(sum(sizes))
        ws = int(self.rs.workspace_bytes(n, with_values, len(sizes) if segmented else 0))
        return (block(4 * n) + (block(4 * n) if with_values else 0)
                + (block(4 * (len(sizes) + 1)) if segmented else 0) + block(max(ws, 1) + 256))

    # -- launches ------------------------------------------------------------
    def launch(self, reqs: List[Request], segmented: bool):
        """Draw the inputs of `reqs` into one device buffer and enqueue their
        sort; returns a handle for poll() / take()."""
        torch, rs = self.torch, self.rs
        s = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        pairs = reqs[0].with_values
        sizes = [r.n for r in reqs]
        n = int(sum(sizes))
        with torch.cuda.stream(s):
            keys = torch.empty(n, dtype=torch.int32, device=self.device)
            vals = torch.empty(n, dtype=torch.int32, device=self.device) if pairs else None
            off = 0
            for r in reqs:
                o = pool_window(r, self.pool_n)
                keys[off:off + r.n].copy_(self.pool[r.dist][o:o + r.n])
                if pairs:
                    torch.arange(r.n, dtype=torch.int32, device=self.device, out=vals[off:off + r.n])
                off += r.n
            ws = rs.alloc_workspace(n, pairs, len(reqs) if segmented else 0, device=self.device)
            table = None
            if segmented:
                host = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
                table = torch.from_numpy(host.view(np.int32)).to(self.device)
                if pairs:
                    rs.sort_pairs_segmented_ex(keys, vals, table, ws, stream=s)
                else:
                    rs.sort_keys_segmented_ex(keys, table, ws, stream=s)
            else:
                if pairs:
                    rs.sort_pairs_ex(keys, vals, ws, stream=s)
                else:
                    rs.sort_keys_ex(keys, ws, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        return {"event": ev, "keys": keys, "vals": vals, "ws": ws, "table": table,
                "sizes": sizes, "stream": s}

    def poll(self, handle) -> bool:
        return handle["event"].query()

    def take(self, handle, keep: bool):
        """Per request (keys, vals) views of a completed launch, or Nones."""
        handle["ws"] = None  # the workspace may be reused now
        out, off = [], 0
        for m in handle["sizes"]:
            if keep:
                v = handle["vals"]
                out.append((handle["keys"][off:off + m], None if v is None else v[off:off + m]))
            else:
                out.append((None, None))
            off += m
        return out

    def check(self):
        self.torch.cuda.synchronize(self.device)
        self.rs.check_stream()


class SortServer:
    def __init__(self, executor, budget_bytes: int = 60 * 10**9, max_inflight: int = 8,
                 small_max: int = 1 << 16, batch_items: int = 1 << 22, keep_results=False,
                 on_done: Optional[Callable[[Done], None]] = None):
        """on_done, if given, receives every completed request as it is taken
        (with its result views when keep_results); the returned list then
        holds the requests and latencies only, so results are not retained."""
        self.ex = executor
        self.budget = int(budget_bytes)
        self.max_inflight = max_inflight
        self.small_max = small_max
        self.batch_items = batch_items
        self.keep = keep_results
        self.on_done = on_done
        self.peak_bytes = 0
        self.launch_log: List[list] = []

    def _fitting_prefix(self, batch: List[Request], with_values: bool, used: int):
        """The longest prefix of `batch` whose segmented launch fits the
        budget next to `used` bytes, and its bytes ([], 0 if none does)."""
        def need(k):
            return self.ex.bytes_for([r.n for r in batch[:k]], with_values, True)
        lo, hi = 0, len(batch)  # prefix lengths: lo fits (or is empty), hi is the candidate
        if used + need(hi) <= self.budget:
            return batch, need(hi)
        hi -= 1
        while lo < hi:  # the bytes grow with the prefix: largest k that fits
            mid = (lo + hi + 1) // 2
            if used + need(mid) <= self.budget:
                lo = mid
            else:
                hi = mid - 1
        return (batch[:lo], need(lo)) if lo else ([], 0)

    def _collect(self, inflight, done: List[Done], now, realtime: bool):
        """Take every completed launch of `inflight`: its requests go to
        `done` (and to on_done).  Returns the launches still running and the
        bytes the completed ones held.  The completed handles are dropped
        before this returns, so their device buffers are free by then."""
        still, freed = [], 0
        for entry in inflight:
            h, rs_, b, li = entry
            if not self.ex.poll(h):
                still.append(entry)
                continue
            tdone = now()
            self.launch_log[li][1] = tdone
            for r, (k, v) in zip(rs_, self.ex.take(h, self.keep)):
                d = Done(r, tdone - r.arrival if realtime else tdone, len(rs_), k, v)
                if self.on_done is not None:
                    self.on_done(d)
                    d = Done(d.request, d.latency, d.batch)
                done.append(d)
            freed += b
        return still, freed

    def run(self, requests: List[Request], realtime: bool = True) -> dict:
        """Serve `requests` (sorted by arrival).  With realtime, a request is
        visible only once the wall clock passes its arrival time.

        The budget bounds the device bytes of the work in flight (its input
        buffers, segment tables and workspaces) as the executor counts them.
        Results handed out after completion (keep_results, on_done) are no
        longer charged, and the executor's resident key pool is outside it."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        waiting = collections.deque()
        inflight = []          # (handle, [requests], bytes, index in launch_log)
        # Per launch: [time launched, time seen complete, requests]; seconds
        # after the start of the run.
        self.launch_log = []
        done: List[Done] = []
        used = 0
        nxt = 0
        t0 = time.perf_counter()
        launches = 0

        def now():
            return time.perf_counter() - t0

        while len(done) < len(reqs):
            t = now()
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= t):
                waiting.append(reqs[nxt])
                nxt += 1
            # Completions free memory and a slot.
            inflight, freed = self._collect(inflight, done, now, realtime)
            used -= freed
            # Admission, in arrival order.
            while waiting and len(inflight) < self.max_inflight:
                head = waiting[0]
                if head.n <= self.small_max:
                    group = [r for r in waiting
                             if r.n <= self.small_max and r.with_values == head.with_values]
                    batch, total = [], 0
                    for r in group:
                        if batch and total + r.n > self.batch_items:
                            break
                        batch.append(r)
                        total += r.n
                    batch, need = self._fitting_prefix(batch, head.with_values, used)
                    if not batch:
                        if not inflight:
                            raise MemoryError("request %d needs %d bytes, more than the budget"
                                              % (head.id, self.ex.bytes_for(
                                                  [head.n], head.with_values, True)))
                        break
                    for r in batch:
                        waiting.remove(r)
                    inflight.append((self.ex.launch(batch, segmented=True), batch, need,
                                     len(self.launch_log)))
                else:
                    need = self.ex.bytes_for([head.n], head.with_values, False)
                    if used + need > self.budget:
                        if not inflight and need > self.budget:
                            raise MemoryError("request %d needs %d bytes, more than the budget"
                                              % (head.id, need))
                        break
                    waiting.popleft()
                    inflight.append((self.ex.launch([head], segmented=False), [head], need,
                                     len(self.launch_log)))
                self.launch_log.append([now(), None, len(inflight[-1][1])])
                used += need
                launches += 1
                self.peak_bytes = max(self.peak_bytes, used)
            if not inflight and not waiting and nxt < len(reqs) and realtime:
                time.sleep(max(0.0, min(reqs[nxt].arrival - now(), 0.001)))
        self.ex.check()
        wall = now()
        lat = np.array([d.latency for d in done])
        items = sum(d.request.n for d in done)
        return {"done": sorted(done, key=lambda d: d.request.id), "wall_s": wall,
                "items_per_s": items / wall, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "launches": launches,
                "peak_bytes": self.peak_bytes, "budget_bytes": self.budget,
                "launch_log": self.launch_log}


class SerialServer:
    """The baseline: one request at a time, in arrival order, each sorted
    alone with a plain synchronous sort once the previous one finished."""

    def __init__(self, executor):
        self.ex = executor

    def run(self, requests: List[Request], realtime: bool = True) -> dict:
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        lat = []
        for r in reqs:
            if realtime:
                while time.perf_counter() - t0 < r.arrival:
                    time.sleep(max(0.0, min(r.arrival - (time.perf_counter() - t0), 0.001)))
            h = self.ex.launch([r], segmented=False)
            while not self.ex.poll(h):
                pass
            self.ex.take(h, False)
            lat.append(time.perf_counter() - t0 - (r.arrival if realtime else 0.0))
        self.ex.check()
        wall = time.perf_counter() - t0
        lat = np.array(lat)
        items = sum(r.n for r in reqs)
        return {"wall_s": wall, "items_per_s": items / wall,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99))}


def make_requests(num: int, seed: int, lo_log10: float = 3.0, hi_log10: float = 8.0,
                  rate_per_s: Optional[float] = None) -> List[Request]:
    """The serving workload: sizes floor(10^U), U uniform on [lo, hi]; 30 %
    key-value; uniform or AND-of-2 keys; Poisson arrivals at `rate_per_s`
    (all at time 0 when None)."""
    from paper_1008_2849_gb300 import inputs
    spec = inputs.request_stream(num, seed, lo_log10, hi_log10)
    arr = (inputs.poisson_arrivals(num, rate_per_s, seed) if rate_per_s else np.zeros(num))
    return [Request(d["id"], d["n"], d["with_values"], d["dist"], d["key_seed"], float(a))
            for d, a in zip(spec, arr)]
