"""GPU tests of captured sorts (CUDA graphs) and per-size-class tuning: a
replayed graph must sort fresh data exactly as the oracle does, every time,
and no tuning setting may change a result."""
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


def test_graph_replays_whole_sort(rs):
    import torch
    n = 3_000_001
    kb = torch.empty(n, dtype=torch.int32, device="cuda")
    vb = torch.empty(n, dtype=torch.int32, device="cuda")
    g = rs.Graph(kb, vb)
    for seed in (120, 121, 122):
        k = inputs.keys("and2" if seed & 1 else "uniform", n, seed=seed)
        v = inputs.index_values(n)
        kb.copy_(torch.from_numpy(k.view(np.int32)))
        vb.copy_(torch.from_numpy(v.view(np.int32)))
        g.launch()
        rs.check_stream()
        ko, vo = oracle_sort(k, v)
        assert np.array_equal(to_host(kb), ko) and np.array_equal(to_host(vb), vo), seed
    g.close()


def test_graph_replays_segmented_sort(rs):
    import torch
    k0, v0, off = inputs.segmented_batch(300, 6, 16, seed=123)
    n = k0.size
    kb = torch.empty(n, dtype=torch.int32, device="cuda")
    vb = torch.empty(n, dtype=torch.int32, device="cuda")
    od = to_dev(off)
    g = rs.Graph(kb, vb, od)
    for seed in (124, 125):
        k = inputs.keys("uniform", n, seed=seed)
        kb.copy_(torch.from_numpy(k.view(np.int32)))
        vb.copy_(torch.from_numpy(v0.view(np.int32)))
        g.launch()
        rs.check_stream()
        ko, vo = oracle.sort_pairs_segmented(k, v0, off)
        assert np.array_equal(to_host(kb), ko) and np.array_equal(to_host(vb), vo), seed
    g.close()


def test_per_class_settings_do_not_change_results(rs):
    n = 1 << 20  # class 2
    k = inputs.keys("distinct256", n, seed=126)
    v = inputs.index_values(n)
    ref_k, ref_v = oracle_sort(k, v)
    cls = rs.size_class(n)
    old = rs.tune_get_class(cls, "tile_pairs")
    try:
        for shape in range(len(rs.tile_shapes())):
            rs.tune_set_class(cls, "tile_pairs", shape)
            kd, vd = to_dev(k), to_dev(v)
            rs.sort_pairs(kd, vd)
            assert np.array_equal(to_host(kd), ref_k) and np.array_equal(to_host(vd), ref_v), shape
    finally:
        rs.tune_set_class(cls, "tile_pairs", old)
