"""Small, self-contained cases for profiling single kernels under ncu.

    python -m paper_2502_14589_gb300.profile_case --n 4096 --mmax 3 --precision fp64

runs one Krylov run of Fig. 2 (m_max iterations at most, fixed tolerance so the run does not
stop early) and one LIM step on a periodic n x n grid, so that every kernel of the hot path
launches a few times on vectors larger than the 129 MB L2 while the device holds only a few
GB (the Krylov basis has m_max + 1 columns).
"""
from __future__ import annotations

import argparse


def main():
    import numpy as np
    import torch
    from paper_2502_14589_gb300 import build, ch, inputs
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--mmax", type=int, default=3)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--eps", type=float, default=0.01)
    ap.add_argument("--tau", type=float, default=1e-9)
    ap.add_argument("--lim", action="store_true", help="also run one LIM step")
    args = ap.parse_args()
    build.build()
    n = [args.n] * args.dim
    N = int(np.prod(n))
    prec = ch.CH_FP64 if args.precision == "fp64" else ch.CH_MIXED
    y = torch.from_numpy(inputs.initial_state(n, 0)).cuda()
    yn = torch.empty_like(y)
    with ch.Grid(args.dim, n, args.eps, prec, args.mmax) as G:
        tau, st = ch.ch_phi_krylov(G.h, y, args.tau, 1e-14, args.mmax, 0, yn)
        if args.lim:
            ch.ch_lim_step(G.h, y, args.tau, yn)
        torch.cuda.synchronize()
        print(f"profile case n={n} N={N} precision={args.precision}: tau={tau:.3g} "
              f"matvecs={st['matvecs']} launches={ch.ch_kernel_launches(G.h)}")


if __name__ == "__main__":
    main()
