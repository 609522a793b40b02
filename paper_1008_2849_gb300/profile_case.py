"""One sort of a seeded synthetic array, for profiler captures.

    python -m paper_1008_2849_gb300.profile_case --log2n 26 [--keys-only]
           [--dist uniform] [--seed 2] [--repeat 1]

Builds librs.so if needed, copies the input to the GPU, runs rs_sort_pairs_ex
(or rs_sort_keys_ex) `repeat` times on fresh copies and checks the device
status.  It times nothing: a profiler (ncu) around it sees exactly the
library's kernels (per sort: one histogram, one plan and four scatter-pass
launches).  2^26 pairs is 512 MiB per array, more than the L2, and small
enough for a many-pass capture to finish quickly.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--log2n", type=int, default=26)
    ap.add_argument("--keys-only", action="store_true")
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)

    import torch

    from paper_1008_2849_gb300 import build, inputs, rs
    build.build_library()
    rs.lib()
    n = 1 << a.log2n
    k = torch.from_numpy(inputs.keys(a.dist, n, a.seed).view(np.int32)).cuda()
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    kb, vb = torch.empty_like(k), torch.empty_like(v)
    ws = rs.alloc_workspace(n, not a.keys_only)
    for _ in range(a.repeat):
        kb.copy_(k)
        vb.copy_(v)
        if a.keys_only:
            rs.sort_keys_ex(kb, ws)
        else:
            rs.sort_pairs_ex(kb, vb, ws)
    rs.check_stream()
    print("sorted %d %s (%s, seed %d) x%d" % (n, "keys" if a.keys_only else "pairs", a.dist,
                                              a.seed, a.repeat))
    return 0


if __name__ == "__main__":
    sys.exit(main())
