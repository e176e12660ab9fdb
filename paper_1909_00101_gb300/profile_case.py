"""A small, bounded solve for profiler captures (no child processes, a few
hundred kernel launches): the blocked path on an F 1024x512, G 1024x512 pair of
the benchmark's distribution (sigma in [1e-4, 1e4], cond(X) = 1e3), with fixed
sweep caps so the launch count is known in advance.

    python -m paper_1909_00101_gb300.profile_case [--precision mixed|fp64]
        [--m 1024] [--n 512] [--w 16] [--fp32-sweeps 2] [--fp64-sweeps 1]
        [--shorten 0] [--fp32-params 1] [--fp64-gemm 1]

The QR shortening is off by default here, so that the Gram and apply kernels
run on the full m-row pair.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--w", type=int, default=16)
    ap.add_argument("--cplx", type=int, default=0)
    ap.add_argument("--fp32-sweeps", type=int, default=2)
    ap.add_argument("--fp64-sweeps", type=int, default=1)
    ap.add_argument("--shorten", type=int, default=0)
    ap.add_argument("--fp32-params", type=int, default=1)
    ap.add_argument("--fp64-gemm", type=int, default=1)
    a = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import paper_1909_00101_gb300 as hz
    from paper_1909_00101_gb300.build import build
    from paper_1909_00101_gb300.inputs import make_pair
    build()
    p = make_pair(a.m, a.m, a.n, lo=1e-4, hi=1e4, cond=1e3, cplx=bool(a.cplx), seed=0)
    F = torch.from_numpy(p.F).cuda()
    G = torch.from_numpy(p.G).cuda()
    with hz.Solver(path="blocked", precision=a.precision, block_w=a.w, inner_max_sweeps=1,
                   fp32_max_sweeps=a.fp32_sweeps, max_sweeps=a.fp64_sweeps, shorten=a.shorten,
                   fp32_params=a.fp32_params, fp64_gemm=a.fp64_gemm) as s:
        r = s.solve(F, G)
    torch.cuda.synchronize()
    i = r.info
    print(json.dumps({k: i[k] for k in ("status", "sweeps_fp32", "sweeps_fp64", "visits", "t_total_us")}))
    # a sweep cap reached is expected here; anything else is a failure
    sys.exit(0 if i["status"] in (0, hz.ENOCONV) else 1)


if __name__ == "__main__":
    main()
