"""Small, self-contained cases for profiling single kernels under ncu.

    python -m paper_2502_14589_gb300.profile_case --n 4096 --mmax 3 --precision fp64

runs one Krylov run of Fig. 2 (m_max iterations at most, fixed tolerance so the run does not
stop early) and one LIM step on a periodic n x n grid, so that every kernel of the hot path
launches a few times on vectors larger than the 129 MB L2 while the device holds only a few
GB (the Krylov basis has m_max + 1 columns).

    python -m paper_2502_14589_gb300.profile_case --n 1024 --mmax 30 --ee2-step 5e-5

instead integrates the benchmark's adaptive EE2 (eps 0.01, tol 1e-6, tau0 1e-7) to the given
time, then times one more adaptive step with CUDA events and runs it once more inside the
NVTX range "step" (for ncu --nvtx --nvtx-include "step/": the launches of one typical step).
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
    ap.add_argument("--ee2-step", type=float, default=None,
                    help="integrate adaptive EE2 to this time, then time one more step")
    args = ap.parse_args()
    build.build()
    n = [args.n] * args.dim
    N = int(np.prod(n))
    prec = ch.CH_FP64 if args.precision == "fp64" else ch.CH_MIXED
    y = torch.from_numpy(inputs.initial_state(n, 0)).cuda()
    yn = torch.empty_like(y)
    if args.ee2_step is not None:
        with ch.Grid(args.dim, n, args.eps, prec, args.mmax) as G:
            st = ch.ch_integrate(G.h, ch.make_params("ee2", True, args.ee2_step, 1e-7, 1e-6, args.mmax), y)
            t, tau = ch.ch_get_state(G.h)
            prm = ch.make_params("ee2", True, 1.0, 1e-7, 1e-6, args.mmax)
            for rep in range(3):
                l0 = ch.ch_kernel_launches(G.h)
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                tu, est = ch.ch_ee_step(G.h, y, tau, prm, yn)
                e1.record(); e1.synchronize()
                print(f"step at t={t:.3g} ({st['steps']} steps before): tau={tau:.3g} taken={tu:.3g} "
                      f"{e0.elapsed_time(e1):.3f} ms, {ch.ch_kernel_launches(G.h) - l0} launches")
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("step")
            ch.ch_ee_step(G.h, y, tau, prm, yn)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        return
    with ch.Grid(args.dim, n, args.eps, prec, args.mmax) as G:
        tau, st = ch.ch_phi_krylov(G.h, y, args.tau, 1e-14, args.mmax, 0, yn)
        if args.lim:
            ch.ch_lim_step(G.h, y, args.tau, yn)
        torch.cuda.synchronize()
        print(f"profile case n={n} N={N} precision={args.precision}: tau={tau:.3g} "
              f"matvecs={st['matvecs']} launches={ch.ch_kernel_launches(G.h)}")


if __name__ == "__main__":
    main()
