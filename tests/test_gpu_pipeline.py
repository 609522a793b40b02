"""GPU parity tests of the warp-specialised scatter pass (k_onesweep_ws,
RS_TUNE_PIPE) that unsigned 32-bit key-value arrays take: every result is
compared bit for bit with the CPU oracle's stable sort.

The pass is forced on in the size classes where it is not the default, so
that sizes of one tile (5376 items) and a few tiles, with ragged tails and
unaligned bases, run through it alongside the large sizes; key
distributions that make passes trivial (skipped) or whose digits pile into
few buckets are included.  The bounded waits are checked by withholding the
first tile's counts.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1008_2849_gb300 import inputs
from tests.gpu_util import oracle_sort, to_dev, to_host

pytestmark = pytest.mark.gpu

TILE = 12 * 32 * 14  # items per tile of the pass


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


@pytest.fixture
def pipe_everywhere(rs):
    """The pipelined pass in every size class (restored afterwards)."""
    old = [rs.tune_get_class(c, "pipe") for c in range(6)]
    for c in range(6):
        rs.tune_set_class(c, "pipe", 1)
    yield
    for c, v in enumerate(old):
        rs.tune_set_class(c, "pipe", v)


def _check_pairs(rs, k, v, offset=0):
    kd, vd = to_dev(k, offset), to_dev(v, offset)
    rs.sort_pairs(kd, vd)
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko)
    assert np.array_equal(to_host(vd), vo)


SIZES = [8193, TILE - 1, TILE, TILE + 1, 2 * TILE, 2 * TILE + 3, 3 * TILE + 1, 65537,
         152 * TILE - 7, 152 * TILE, 152 * TILE + 1, 310 * TILE + 5, 1_000_003,
         (1 << 20) + 1, 3 * (1 << 20) + 7]


@pytest.mark.parametrize("n", SIZES)
def test_pipeline_sizes(rs, pipe_everywhere, n):
    k = inputs.keys("uniform", n, seed=300 + n % 101)
    v = inputs.splitmix32(301, n, 3)  # values unrelated to the index
    _check_pairs(rs, k, v)


@pytest.mark.parametrize("dist", ["and4", "distinct256", "equal", "sorted", "reverse", "low16"])
def test_pipeline_distributions(rs, pipe_everywhere, dist):
    n = 2_000_001
    k = inputs.keys(dist, n, seed=310)
    _check_pairs(rs, k, inputs.index_values(n))


@pytest.mark.parametrize("off", [1, 2, 3])
def test_pipeline_unaligned_base(rs, pipe_everywhere, off):
    n = 3 * TILE + 77
    k = inputs.keys("and2", n, seed=320 + off)
    _check_pairs(rs, k, inputs.index_values(n), offset=off)


def test_pipeline_2pow24_plus(rs):
    """A class-4 size with the default settings (the pass is the default
    there), a ragged last tile."""
    assert rs.tune_get_class(rs.size_class((1 << 24) + 5), "pipe") == 1
    n = (1 << 24) + 5
    k = inputs.keys("uniform", n, seed=330)
    _check_pairs(rs, k, inputs.index_values(n))


def test_pipeline_graph_replay(rs, pipe_everywhere):
    """Captured in a CUDA graph and replayed on fresh data twice."""
    import torch
    n = 5 * TILE + 9
    kd = torch.empty(n, dtype=torch.int32, device="cuda")
    vd = torch.empty_like(kd)
    graph = rs.Graph(kd, vd)
    try:
        for seed in (340, 341):
            k = inputs.keys("uniform", n, seed=seed)
            v = inputs.index_values(n)
            kd.copy_(torch.from_numpy(k.view(np.int32)))
            vd.copy_(torch.from_numpy(v.view(np.int32)))
            graph.launch()
            torch.cuda.synchronize()
            rs.check_stream()
            ko, vo = oracle_sort(k, v)
            assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo)
    finally:
        graph.close()


def test_pipeline_same_as_tile_shapes(rs):
    """The pipelined pass and the tile-shape pass give the same bits."""
    n = 4_000_037
    k = inputs.keys("and3", n, seed=350)
    v = inputs.index_values(n)
    cls = rs.size_class(n)
    old = rs.tune_get_class(cls, "pipe")
    outs = []
    try:
        for pipe in (0, 1):
            rs.tune_set_class(cls, "pipe", pipe)
            kd, vd = to_dev(k), to_dev(v)
            rs.sort_pairs(kd, vd)
            outs.append((to_host(kd), to_host(vd)))
    finally:
        rs.tune_set_class(cls, "pipe", old)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(outs[1][0], ko) and np.array_equal(outs[1][1], vo)


def test_pipeline_lookback_wait_runs_out(rs, pipe_everywhere):
    """The first tile withholds its counts: the later tiles' bounded waits
    run out, the call reports RS_ERR_TIMEOUT, and the context stays usable."""
    n = 8 * TILE + 11
    k = inputs.keys("uniform", n, seed=360)
    v = inputs.index_values(n)
    kd, vd = to_dev(k), to_dev(v)
    rs.debug_set_spin_limit(2000)
    rs.debug_withhold_first_tile(True)
    try:
        with pytest.raises(rs.RsError) as ei:
            rs.sort_pairs(kd, vd)
        assert ei.value.code == 4
    finally:
        rs.debug_withhold_first_tile(False)
        rs.debug_set_spin_limit(0)
    assert rs.stream_status() == 0
    _check_pairs(rs, k, v)
