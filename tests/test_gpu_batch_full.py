"""The batched segmented workload at full size: 4096 arrays of (uint32 key,
uint32 value = index inside the array), sizes log-uniform on [2^8, 2^22]
(seed 10) as drawn -- about 1.89e9 pairs, 15 GB -- sorted by one captured
graph of rs_sort_pairs_segmented_ex and compared bit for bit with the CPU
oracle's segmented sort of the same batch, whose host time is printed as the
oracle's figure for this workload.

It takes about a minute and tens of GB of host memory; it is part of the
GPU suite (RS_SKIP_FULL_CHECKS=1 leaves it out of a quick run)."""
from __future__ import annotations

import os
import time

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("RS_SKIP_FULL_CHECKS") == "1",
                                 reason="full-size checks skipped: RS_SKIP_FULL_CHECKS=1")]


def test_batched_workload_full():
    import torch
    from paper_1008_2849_gb300 import build, rs
    build.build_library()
    k_np, v_np, off_np = inputs.segmented_batch(4096, 8, 22, seed=10, scale_to=None)
    n = k_np.size
    k = torch.from_numpy(k_np.view(np.int32)).cuda()
    v = torch.from_numpy(v_np.view(np.int32)).cuda()
    off = torch.from_numpy(off_np.view(np.int32)).cuda()
    graph = rs.Graph(k, v, off)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    graph.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    rs.check_stream(stream)
    gpu_ms = e0.elapsed_time(e1)
    graph.close()
    got_k = k.cpu().numpy().view(np.uint32)
    got_v = v.cpu().numpy().view(np.uint32)
    del k, v
    t0 = time.perf_counter()
    ko, vo = oracle.sort_pairs_segmented(k_np, v_np, off_np)
    oracle_s = time.perf_counter() - t0
    assert np.array_equal(got_k, ko)
    assert np.array_equal(got_v, vo)
    print("batched workload verified: %d pairs in 4096 arrays; GPU graph %.2f ms "
          "(cold, one launch); CPU oracle (one thread) %.1f s = %.3g pairs/s"
          % (n, gpu_ms, oracle_s, n / oracle_s))
