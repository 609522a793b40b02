"""Helpers shared by the GPU tests: moving uint32 arrays to and from CUDA
tensors, and oracle calls sized for the host (threaded above 2^22 items)."""
from __future__ import annotations

import os

import numpy as np

import oracle


def to_dev(a: np.ndarray, offset_elems: int = 0):
    """Copy a uint32 array to a new CUDA int32 tensor; with offset_elems > 0
    the returned view starts that many elements into a larger buffer (so its
    base is only 4-byte aligned)."""
    import torch
    if offset_elems:
        buf = torch.empty(a.size + offset_elems, dtype=torch.int32, device="cuda")
        view = buf[offset_elems:]
        view.copy_(torch.from_numpy(a.view(np.int32)))
        return view
    return torch.from_numpy(a.view(np.int32)).to("cuda")


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def oracle_sort(keys: np.ndarray, vals):
    if keys.size > (1 << 22):
        return oracle.sort_pairs_threaded(keys, vals, os.cpu_count() or 4)
    return oracle.sort_pairs(keys, vals)
