"""One sort of a seeded synthetic array, for profiler captures.

    python -m paper_1008_2849_gb300.profile_case --log2n 26 [--keys-only]
           [--dist uniform] [--seed 2] [--repeat 1] [--digits11 SHAPE]

Builds librs.so if needed, copies the input to the GPU, runs rs_sort_pairs_ex
(or rs_sort_keys_ex) `repeat` times on fresh copies and checks the device
status.  It times nothing: a profiler (ncu) around it sees exactly the
library's kernels (per sort: one histogram, one plan and four scatter-pass
launches).  With --digits11 SHAPE it runs rs_sort_digits11_ex instead (three
passes of 11/11/10-bit digits, scatter-kernel tile shape SHAPE; per sort:
three counting, three scan and three scatter launches).  2^26 pairs is 256
MiB per array, more than the L2, and small enough for a many-pass capture to
finish quickly.
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
    ap.add_argument("--digits11", type=int, default=-1,
                    help="tile shape of the 11-bit-digit sort; -1: the default sort")
    a = ap.parse_args(argv)

    import torch

    from paper_1008_2849_gb300 import build, inputs, rs
    build.build_library()
    rs.lib()
    n = 1 << a.log2n
    k = torch.from_numpy(inputs.keys(a.dist, n, a.seed).view(np.int32)).cuda()
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    kb, vb = torch.empty_like(k), torch.empty_like(v)
    if a.digits11 >= 0:
        rs.tune_set("d11_shape", a.digits11)
        ws = rs.alloc_workspace_digits11(n, not a.keys_only)
    else:
        ws = rs.alloc_workspace(n, not a.keys_only)
    for _ in range(a.repeat):
        kb.copy_(k)
        vb.copy_(v)
        if a.digits11 >= 0:
            rs.sort_digits11_ex(kb, None if a.keys_only else vb, ws)
        elif a.keys_only:
            rs.sort_keys_ex(kb, ws)
        else:
            rs.sort_pairs_ex(kb, vb, ws)
    rs.check_stream()
    print("sorted %d %s (%s, seed %d) x%d" % (n, "keys" if a.keys_only else "pairs", a.dist,
                                              a.seed, a.repeat))
    return 0


if __name__ == "__main__":
    sys.exit(main())
