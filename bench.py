"""Benchmark of the Cahn-Hilliard hot path on GB300.

One step = one whole integration of the workload to its final time T, first with the
adaptive EE2 scheme (Fig. 4, m_max = 30) and then with the adaptive LIM scheme (Fig. 3),
both from the same seeded initial state already resident in HBM.  Metric: grid-point
operator applications per second = N x (A_hat products + right-hand-side evaluations) /
time, with the time to T of each scheme reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload c1_2d1024_adaptive]

N > 1 runs under torchrun: every rank integrates its own independently seeded instance
(replicas of the single-GPU workload, weak scaling) and rank 0 prints the JSON line.
--impl reference times the plain single-threaded C oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CH grid-pt updates/s & time-to-T (EE, LIM): mixed/batched vs FP64, ≤1e-5 err"
UNIT = "grid-pt operator applications/s"
L2_BYTES = 129 * 2 ** 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak of GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM x 2.07 GHz
FP64_ISSUE_PEAK = 152 * 2 * 2.07e9              # FP64-pipe instructions/s
FP64_PEAK_TFLOPS = 2 * FP64_ISSUE_PEAK / 1e12   # FMA = 2 flop
try:
    HBM_GBS = json.load(open(PEAKS_FILE))["hbm_gbs"]
except Exception:
    HBM_GBS = 6800.0                            # fallback when the measured file is absent


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c1_2d1024_adaptive")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-roofline", action="store_true",
                    help="skip the per-kernel timing after the timed region (launch-list runs)")
    ap.add_argument("--t-final", type=float, default=None,
                    help="integrate to this time instead of the workload's T (profiling runs only)")
    return ap.parse_args()


def workload_desc(name, wl):
    if wl["dim"] == 2:
        grid = f"2D periodic {wl['n']}x{wl['n']}"
    else:
        grid = f"3D periodic {wl['n']}^3"
    return (f"{grid} unit domain, eps={wl['eps']}, u0 U[{wl['lo']},{wl['hi']}] zero-mean"
            f"{'+' + str(wl['mean']) if wl['mean'] else ''}, adaptive EE2(m_max={wl['mmax']}) and LIM, "
            f"tol={wl['tol']}, tau0={wl['tau0']}, T={wl['T']}, FP64")


# ---------------------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_samples(out)


def parse_clock_samples(text):
    """Median SM clock, maximum SM clock and the throttle reasons seen in the CSV lines of
    `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits`."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1])); smax.append(float(f[2]))
        except ValueError:
            continue
        for name, val in zip(names, f[5:9]):
            if val.lower() in ("active", "1", "yes"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# reference arm / CPU baseline: the plain C oracle on the host
# ---------------------------------------------------------------------------------------
def oracle_sample(wl, seed, steps_per_scheme):
    """Bounded sample of the workload on the oracle: the first `steps_per_scheme` steps of
    each adaptive scheme.  Returns (operator applications, seconds)."""
    import numpy as np  # noqa: F401
    from oracle import oracle
    from paper_2502_14589_gb300 import inputs
    n = [wl["n"]] * wl["dim"]
    g = oracle.Grid(wl["dim"], n, wl["eps"])
    y0 = inputs.initial_state(n, seed, wl["lo"], wl["hi"], wl["mean"])
    ops, secs = 0, 0.0
    for scheme in ("ee2", "lim"):
        t0 = time.perf_counter()
        rc, y, t, st, rec = oracle.integrate(g, y0, scheme, True, wl["T"], wl["tau0"], tol=wl["tol"],
                                             mmax=wl["mmax"], max_steps=steps_per_scheme, max_rec=16)
        secs += time.perf_counter() - t0
        ops += g.N * (st["matvecs"] + st["rhs_evals"])
    return ops, secs


def run_reference(args, rank, world):
    from paper_2502_14589_gb300 import inputs
    wl = inputs.WORKLOADS[args.workload]
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    sps = 2
    for _ in range(args.warmup):
        oracle_sample(wl, 0, sps)
    tot_ops, tot_s = 0, 0.0
    for k in range(args.steps):
        ops, s = oracle_sample(wl, 0, sps)
        tot_ops += ops; tot_s += s
    value = tot_ops / tot_s
    sample = (f"first {sps} adaptive EE2 steps + first {sps} adaptive LIM steps of the workload "
              f"per bench step, single-threaded C oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, wl), "global_batch": 1,
                   "parallelism": "replicas (rank 0 only runs the oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------------------
# batched workload: many independent instances of uneven size in one launch sequence
# ---------------------------------------------------------------------------------------
def run_batch_workload(args, rank, world, dist):
    import numpy as np
    import torch
    from paper_2502_14589_gb300 import build, ch, inputs, replicas
    build.build()
    wl = dict(inputs.WORKLOADS[args.workload])
    if args.t_final is not None:
        wl["T"] = args.t_final
    count = wl["count"]
    sides, eps = inputs.batch_descriptors(count, seed=0)
    y0s = [inputs.initial_state((int(n), int(n)), replicas.batch_instance_seed(rank, i), wl["lo"], wl["hi"])
           for i, n in enumerate(sides)]
    Ns = np.array([int(n) * int(n) for n in sides])
    stream = torch.cuda.current_stream()
    out = {}
    for prec, name in ((ch.CH_MIXED, "mixed"), (ch.CH_FP64, "fp64")):
        h = ch.ch_create_batch(2, [int(n) for n in sides], list(eps), prec, wl["mmax"], stream)
        offs, chunk = ch.ch_batch_layout(h, count)
        y0 = torch.zeros(offs[-1], dtype=torch.float64, device="cuda")
        for i in range(count):
            y0[offs[i]:offs[i] + Ns[i]] = torch.from_numpy(y0s[i]).cuda()
        y = torch.empty_like(y0)
        prm = ch.make_params("ee2", True, wl["T"], wl["tau0"], wl["tol"], wl["mmax"])
        reps = args.steps if name == "mixed" else 1
        for _ in range(args.warmup if name == "mixed" else 1):
            y.copy_(y0); ch.ch_integrate_batch(h, prm, y, count)
        torch.cuda.synchronize()
        ms, ops = 0.0, 0
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(reps):
            y.copy_(y0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = ch.ch_integrate_batch(h, prm, y, count)
            e1.record(stream); e1.synchronize()
            ms += e0.elapsed_time(e1)
            ops += int(sum(Ns[i] * (st[i]["matvecs"] + st[i]["rhs_evals"]) for i in range(count)))
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms, ops = replicas.combine(dist, ms, ops, "cuda")
        yh = y.cpu().numpy()
        out[name] = {"ms": ms / reps, "value": ops / (ms * 1e-3), "chunk_len": chunk,
                     "steps_max": max(x["steps"] for x in st), "steps_sum": sum(x["steps"] for x in st),
                     "y": [yh[offs[i]:offs[i] + Ns[i]] for i in range(count)],
                     "launches": ch.ch_batch_kernel_launches(h)}
        ch.ch_destroy_batch(h)
    errs = [np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(out["mixed"]["y"], out["fp64"]["y"])]
    for k in out:
        out[k].pop("y")
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": out["mixed"]["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["mixed"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 mixed",
            "data": "synthetic",
            "config": {"workload": f"batch of {count} 2D periodic instances, sides from {list(inputs.BATCH_SIDES)}, "
                                   f"eps U[0.01,0.05], u0 U[{wl['lo']},{wl['hi']}] zero-mean, adaptive EE2(m_max="
                                   f"{wl['mmax']}) tol {wl['tol']} to T={wl['T']}, FP32 Krylov basis/stencils, FP64 "
                                   f"reductions/phi/control", "global_batch": count, "grid_points": int(Ns.sum())},
            "batch": out, "mixed_vs_fp64": {"speedup": out["fp64"]["ms"] / out["mixed"]["ms"],
                                             "max_rel_err_at_T": float(max(errs)),
                                             "median_rel_err_at_T": float(np.median(errs))},
        }), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        from paper_2502_14589_gb300 import replicas
        if args.impl == "gb300":                 # the reference arm runs on the host only
            import torch
            torch.cuda.set_device(local_rank)
        dist = replicas.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.workload.startswith("c3"):
        run_batch_workload(args, rank, world, dist)
        if dist is not None:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2502_14589_gb300 import build, ch, inputs, replicas
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = dict(inputs.WORKLOADS[args.workload])
    if args.t_final is not None:
        wl["T"] = args.t_final
    n = [wl["n"]] * wl["dim"]
    N = int(np.prod(n))
    y0_host = inputs.initial_state(n, replicas.instance_seed(rank), wl["lo"], wl["hi"], wl["mean"])
    y0 = torch.from_numpy(y0_host).to(dev)
    y = torch.empty_like(y0)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    G = ch.Grid(wl["dim"], n, wl["eps"], ch.CH_FP64, wl["mmax"], stream)
    prm = {s: ch.make_params(s, True, wl["T"], wl["tau0"], wl["tol"], wl["mmax"]) for s in ("ee2", "lim")}

    y_ee2 = torch.empty_like(y0)              # EE2 solution at T of the last step

    def one_step(yin_dev, record=None):
        stats = {}
        for s in ("ee2", "lim"):
            y.copy_(yin_dev)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats[s] = ch.ch_integrate(G.h, prm[s], y)
            e1.record(stream)
            if s == "ee2":
                y_ee2.copy_(y)
            if record is not None:
                record[s].append((e0, e1, stats[s]))
        return stats

    for _ in range(args.warmup):
        one_step(y0)
    torch.cuda.synchronize()

    # ---- timed region: K steps, events per step, L2 flushed between steps --------------
    ch.ch_timing_start(G.h, None)           # per-class launch counts, no per-kernel events
    launches0 = ch.ch_kernel_launches(G.h)
    clocks = ClockSampler()
    if rank == 0:
        clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, ops, rec = [], 0, {"ee2": [], "lim": []}
    for k in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = one_step(y0, rec)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for s in ("ee2", "lim"):
            ops += N * (st[s]["matvecs"] + st[s]["rhs_evals"])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    launches = ch.ch_kernel_launches(G.h) - launches0
    _, _, counts = ch.ch_timing_read(G.h)
    total_ms, ops = replicas.combine(dist, sum(step_ms), ops, dev)
    value = ops / (total_ms * 1e-3)
    ttt = {}
    for s in ("ee2", "lim"):
        ms = [e0.elapsed_time(e1) for e0, e1, _ in rec[s]]
        st = rec[s][-1][2]
        ttt[s] = {"ms": sum(ms) / len(ms), "steps": st["steps"], "matvecs": st["matvecs"],
                  "rhs_evals": st["rhs_evals"], "phi_evals": st["phi_evals"],
                  "tau_shrinks": st["tau_shrinks"],
                  "ops_per_s": N * (st["matvecs"] + st["rhs_evals"]) / (sum(ms) / len(ms) * 1e-3)}

    # ---- mixed precision on the same instance: time to T and error at T against FP64 ----
    mixed = None
    if not args.no_mixed:
        y_fp64 = y_ee2.clone()                            # FP64 EE2 at T from the timed step
        Gm = ch.Grid(wl["dim"], n, wl["eps"], ch.CH_MIXED, wl["mmax"], stream)
        ym = torch.empty_like(y0)
        ym.copy_(y0)
        pw = ch.make_params("ee2", True, wl["T"] / 10, wl["tau0"], wl["tol"], wl["mmax"])
        ch.ch_integrate(Gm.h, pw, ym)                     # warm-up (graph capture)
        ym.copy_(y0)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stm = ch.ch_integrate(Gm.h, prm["ee2"], ym)
        e1.record(stream); e1.synchronize()
        ms_m = e0.elapsed_time(e1)
        err = float(torch.linalg.norm(ym - y_fp64) / torch.linalg.norm(y_fp64))
        mixed = {"ee2_ms_to_T": ms_m, "ee2_speedup_vs_fp64": ttt["ee2"]["ms"] / ms_m,
                 "ee2_rel_err_at_T_vs_fp64": err, "steps": stm["steps"], "matvecs": stm["matvecs"],
                 "ops_per_s": N * (stm["matvecs"] + stm["rhs_evals"]) / (ms_m * 1e-3),
                 "mass_drift": float(abs(ym.mean() - y0.mean()))}
        if not args.no_roofline:        # one Arnoldi iteration (j = 10) on the FP32 basis
            mixed["arnoldi_j10_us"] = ch.ch_bench_kernel(Gm.h, "arnoldi", 50)["avg_us"]
        Gm.close()

    # ---- end to end through the C ABI with host buffers ----------------------------------
    e2e = None
    if not args.no_e2e:
        y_host = torch.from_numpy(y0_host.copy()).pin_memory()
        out_host = torch.empty(N, dtype=torch.float64).pin_memory()
        e2e_ops, e2e_ms = 0, 0.0
        for k in range(max(1, args.steps // 2)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s in ("ee2", "lim"):
                y.copy_(y_host, non_blocking=True)
                st = ch.ch_integrate(G.h, prm[s], y)
                out_host.copy_(y, non_blocking=True)
                e2e_ops += N * (st["matvecs"] + st["rhs_evals"])
            e1.record(stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e = {"value": e2e_ops / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": 2 * N * 8}

    # ---- per-class kernel table: each class timed on the workload grid with CUDA events on
    # the grid's stream around a graph of 200 back-to-back launches (Arnoldi iteration at j = 10)
    kernels = {}
    classes = ("arnoldi", "tstage", "wstage", "mgs", "resid1", "lim2", "rhs1", "rhs2")
    for cls in (() if args.no_roofline else classes):
        if counts[cls] == 0:
            continue                     # not launched in the timed region on this grid
        kb = ch.ch_bench_kernel(G.h, cls, 200)
        dur = kb["avg_us"] * 1e-6
        kernels[cls] = {"launches": counts[cls], "avg_us": kb["avg_us"],
                        "est_share_s": counts[cls] * dur,
                        "gbs": kb["bytes"] / dur / 1e9, "tflops": kb["flops"] / dur / 1e12,
                        "fp64_issue_frac": kb["fp64_instr"] / dur / FP64_ISSUE_PEAK,
                        "bytes": kb["bytes"], "flops": kb["flops"], "fp64_instr": kb["fp64_instr"]}
    # ---- roofline of the dominant kernel, measured live: every launch of its class timed
    # with CUDA events on the grid's stream over the first twentieth of the workload's run
    # (t in [0, T/20], the same kernels and Krylov dimensions as the timed region; CUDA
    # graphs are off while launches are timed), with the algorithmic work of each launch
    # summed by the library (flops and bytes per point times the points of the launch)
    roof, live = None, {}
    if kernels:
        for cls, scheme in (("arnoldi", "ee2"), ("lim2", "lim")):
            if cls not in kernels:
                continue
            y.copy_(y0)
            ch.ch_timing_start(G.h, cls)
            seg = ch.make_params(scheme, True, wl["T"] / 20, wl["tau0"], wl["tol"], wl["mmax"])
            ch.ch_integrate(G.h, seg, y)
            ms, nt, _ = ch.ch_timing_read(G.h)
            fl, by = ch.ch_timing_work(G.h)
            ch.ch_timing_start(G.h, None)
            if nt > 0 and ms > 0:
                live[cls] = {"launches": nt, "avg_us": 1e3 * ms / nt, "tflops": fl / (ms * 1e-3) / 1e12,
                             "gbs": by / (ms * 1e-3) / 1e9, "flops_per_launch": fl / nt,
                             "bytes_per_launch": by / nt}
        dom = max(kernels, key=lambda c: kernels[c]["est_share_s"])
        if dom in live:
            kl = live[dom]
            roof = {"kernel": "k_" + dom, "bound": "alu", "achieved": kl["tflops"],
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": kl["tflops"] / FP64_PEAK_TFLOPS,
                    "traffic": None,
                    "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (FP64 pipe)",
                    "measured": f"{kl['launches']} launches timed live over t in [0, T/20]",
                    "avg_launch_us": kl["avg_us"], "algorithmic_flops_per_launch": kl["flops_per_launch"],
                    "algorithmic_bytes_per_launch": kl["bytes_per_launch"], "achieved_gbs": kl["gbs"],
                    "hbm_frac_of_measured": kl["gbs"] / HBM_GBS}

    # ---- CPU baseline (oracle on a bounded sample, rank 0 only, N = 1) -----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        oracle.build()
        c_ops, c_s = oracle_sample(wl, 0, 12)
        cpu = {"value": c_ops / c_s, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first 12 adaptive EE2 steps + first 12 adaptive LIM steps of the same "
                         f"workload (seed 0), {c_s:.1f} s single-threaded on the host"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, wl), "global_batch": world,
                       "grid_points": N, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed (256 MiB write) before every timed step"},
            "time_to_T": ttt, "e2e": e2e, "gpu_launches": launches, "launches_by_kernel": counts,
            "mixed": mixed, "roofline": roof, "kernels": kernels, "kernels_live": live, "hbm_peak_gbs": HBM_GBS, "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(out), flush=True)
    G.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
