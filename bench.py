"""Benchmark of the Cahn-Hilliard hot path on GB300.

One step = one whole integration of the workload to its final time T, first with the
adaptive EE2 scheme (Fig. 4, m_max = 30) and then with the adaptive LIM scheme (Fig. 3),
both from the same seeded initial state already resident in HBM.  Metric: grid-point
operator applications per second = N x (A_hat products + right-hand-side evaluations) /
time, with the time to T of each scheme reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload c1_2d1024_adaptive] [--roofline-kernel mgs]

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
# FP64 FMA peak of GB300: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c1_2d1024_adaptive")
    ap.add_argument("--roofline-kernel", default="mgs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
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
# GPU arm
# ---------------------------------------------------------------------------------------
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2502_14589_gb300 import build, ch, inputs
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = inputs.WORKLOADS[args.workload]
    n = [wl["n"]] * wl["dim"]
    N = int(np.prod(n))
    y0_host = inputs.initial_state(n, rank, wl["lo"], wl["hi"], wl["mean"])
    y0 = torch.from_numpy(y0_host).to(dev)
    y = torch.empty_like(y0)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    G = ch.Grid(wl["dim"], n, wl["eps"], ch.CH_FP64, wl["mmax"], stream)
    prm = {s: ch.make_params(s, True, wl["T"], wl["tau0"], wl["tol"], wl["mmax"]) for s in ("ee2", "lim")}

    def one_step(yin_dev):
        stats = {}
        for s in ("ee2", "lim"):
            y.copy_(yin_dev)
            stats[s] = ch.ch_integrate(G.h, prm[s], y)
        return stats

    for _ in range(args.warmup):
        one_step(y0)
    torch.cuda.synchronize()

    # ---- timed region: K steps, events per step, L2 flushed between steps --------------
    ch.ch_timing_start(G.h, args.roofline_kernel)
    launches0 = ch.ch_kernel_launches(G.h)
    clocks = ClockSampler()
    if rank == 0:
        clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, ops, per_scheme = [], 0, {"ee2": [], "lim": []}
    for k in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = one_step(y0)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for s in ("ee2", "lim"):
            ops += N * (st[s]["matvecs"] + st[s]["rhs_evals"])
            per_scheme[s].append(st[s])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    launches = ch.ch_kernel_launches(G.h) - launches0
    kern_ms, kern_n, counts = ch.ch_timing_read(G.h)
    ch.ch_timing_start(G.h, None)
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        o = torch.tensor([float(ops)], dtype=torch.float64, device=dev)
        dist.all_reduce(o, op=dist.ReduceOp.SUM)
        ops = float(o.item())
    value = ops / (total_ms * 1e-3)

    # ---- time to T of each scheme (one more run each, events on the stream) -------------
    ttt = {}
    for s in ("ee2", "lim"):
        y.copy_(y0)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stt = ch.ch_integrate(G.h, prm[s], y)
        e1.record(stream)
        e1.synchronize()
        ttt[s] = {"ms": e0.elapsed_time(e1), "steps": stt["steps"], "matvecs": stt["matvecs"],
                  "rhs_evals": stt["rhs_evals"], "phi_evals": stt["phi_evals"],
                  "tau_shrinks": stt["tau_shrinks"]}

    # ---- end to end through the C ABI with host buffers ----------------------------------
    e2e = None
    if not args.no_e2e:
        y_host = torch.from_numpy(y0_host.copy()).pin_memory()
        out_host = torch.empty(N, dtype=torch.float64).pin_memory()
        e2e_ops, e2e_ms = 0, 0.0
        for k in range(args.steps):
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

    # ---- roofline of the timed kernel class -----------------------------------------------
    roof = None
    if kern_n > 0:
        avg_s = kern_ms * 1e-3 / kern_n
        if args.roofline_kernel == "mgs":
            # one MGS pass: w -= h v_k and one dot product: 2 FP64 FMA = 4 flop per point
            flop = 4.0 * N
            achieved = flop / avg_s / 1e12
            roof = {"kernel": "k_mgs", "bound": "alu", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "traffic": None, "peak_source": "FP64 FMA rate 152 SM x 2 FMA/clk x 2.07 GHz",
                    "launches_timed": kern_n, "avg_launch_us": avg_s * 1e6,
                    "algorithmic_bytes_per_launch": 32.0 * N}
    hbm = None
    try:
        hbm = json.load(open(PEAKS_FILE)).get("hbm_gbs")
    except Exception:
        pass

    # ---- CPU baseline (oracle on a bounded sample, rank 0 only, N = 1) -----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        oracle.build()
        c_ops, c_s = oracle_sample(wl, 0, 4)
        cpu = {"value": c_ops / c_s, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first 4 adaptive EE2 steps + first 4 adaptive LIM steps of the same "
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
            "roofline": roof, "hbm_peak_gbs_measured": hbm, "cpu_baseline": cpu, "clocks": clk,
        }
        print(json.dumps(out), flush=True)
    G.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
