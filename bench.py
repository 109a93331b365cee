"""Benchmark of the Cahn-Hilliard hot path on GB300.

Default workload: 3D periodic 512^3 (134M unknowns), eps = 0.01, u0 U[-0.05, 0.05] zero
mean, adaptive EE2 (Fig. 4, m_max = 30) and adaptive LIM (Fig. 3), tol 1e-6, tau0 = 1e-7, to
T = 1e-4.  One step = one whole integration of the workload to T with each scheme, from the
same seeded state already resident in HBM: EE2 in mixed precision (FP32 Krylov basis and
stencils; FP64 state, reductions, projected phi and control) and LIM in FP64.  Metric:
grid-point operator applications per second = N x (A_hat products + right-hand-side
evaluations) / time, with the time to T of each scheme beside it, and the mixed-precision
EE2 against the plain FP64 EE2 on the same grid (time and error at T).  The mixed-precision
LIM (FP32 iterations on the increment) is reported beside the step: at this workload its
per-step FP64 work (bound, right-hand side, estimate) dominates, and Eq. (LIMdt)'s
unclamped growth makes adaptive LIM runs that differ by rounding take different steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload c4_3d512_adaptive | c1_2d1024_adaptive | c2_3d256_adaptive | c3_batch256]

N > 1 runs under torchrun: every rank integrates its own independently seeded instance
(replicas of the single-GPU workload, weak scaling) and rank 0 prints the JSON line.
--impl reference times the plain single-threaded C oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
DEFAULT_WORKLOAD = "c4_3d512_adaptive"
try:
    HBM_GBS, HBM_SOURCE = json.load(open(PEAKS_FILE))["hbm_gbs"], "measured"
except Exception:
    HBM_GBS, HBM_SOURCE = 6800.0, "fallback"     # the profiling recipe's fallback copy bandwidth
# DRAM traffic per algorithmic byte of the dominant kernel, from the ncu capture summarised
# in this file (None when the kernel changed after the capture)
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_arnoldi_gmgs_3d_mixed.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--t-final", type=float, default=None,
                    help="integrate to this time instead of the workload's T (short runs)")
    return ap.parse_args()


def workload_desc(name, wl):
    if name.startswith("c3"):
        from paper_2502_14589_gb300 import inputs
        return (f"batch of {wl['count']} 2D periodic instances, sides from {list(inputs.BATCH_SIDES)}, "
                f"eps U[0.01,0.05], u0 U[{wl['lo']},{wl['hi']}] zero-mean, adaptive EE2(m_max={wl['mmax']}) "
                f"tol {wl['tol']} to T={wl['T']}")
    grid = f"2D periodic {wl['n']}x{wl['n']}" if wl["dim"] == 2 else f"3D periodic {wl['n']}^3"
    return (f"{grid} unit domain, eps={wl['eps']}, u0 U[{wl['lo']},{wl['hi']}] zero-mean"
            f"{'+' + str(wl['mean']) if wl['mean'] else ''}, adaptive EE2(m_max={wl['mmax']}) and LIM, "
            f"tol={wl['tol']}, tau0={wl['tau0']}, T={wl['T']}")


def host_cpu():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model, "arch": platform.machine()}


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


def profile_traffic_ratio():
    """DRAM bytes per algorithmic byte of the dominant kernel from its ncu summary (a line
    `dram_per_algorithmic_byte: R`), or None."""
    try:
        for line in open(TRAFFIC_PROFILE):
            if line.strip().startswith("dram_per_algorithmic_byte:"):
                return float(line.split(":", 1)[1].split()[0])
    except (OSError, ValueError, IndexError):
        pass
    return None


# ---------------------------------------------------------------------------------------
# reference arm / CPU baseline: the plain C oracle on the host
# ---------------------------------------------------------------------------------------
SAMPLE_POINTS = 8_400_000     # points of the oracle's sample slab


def oracle_sample(wl, seed, y0=None, budget_s=5.0):
    """Bounded sample of the workload on the oracle: f(y) of Eq. (IVP), one grid-wide
    operator application as the metric counts them, on a slab of the workload's initial
    state (its first planes in 3D, rows in 2D, at most SAMPLE_POINTS points, as a periodic
    grid of that extent; the arithmetic per point is the workload's), repeated until
    budget_s seconds have passed.  Returns (operator applications, seconds, slab shape)."""
    import numpy as np
    from oracle import oracle
    from paper_2502_14589_gb300 import inputs
    n = [wl["n"]] * wl["dim"]
    if y0 is None:
        y0 = inputs.initial_state(n, seed, wl["lo"], wl["hi"], wl["mean"])
    plane = int(np.prod(n[:-1]))
    last = max(1, min(n[-1], SAMPLE_POINTS // plane))
    slab = n[:-1] + [last]
    ys = np.ascontiguousarray(y0[:plane * last])
    g = oracle.Grid(wl["dim"], slab, wl["eps"])
    ops, secs = 0, 0.0
    while secs < budget_s or ops == 0:
        t0 = time.perf_counter()
        oracle.rhs(g, ys)
        secs += time.perf_counter() - t0
        ops += g.N
    return ops, secs, slab


def run_reference(args, rank, world):
    from paper_2502_14589_gb300 import inputs
    wl = inputs.WORKLOADS[args.workload]
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    n = [wl["n"]] * wl["dim"]
    y0 = inputs.initial_state(n, 0, wl["lo"], wl["hi"], wl["mean"])
    for _ in range(args.warmup):
        oracle_sample(wl, 0, y0, budget_s=1.0)
    tot_ops, tot_s = 0, 0.0
    for _ in range(args.steps):
        ops, s, slab = oracle_sample(wl, 0, y0)
        tot_ops += ops; tot_s += s
    value = tot_ops / tot_s
    sample = (f"per bench step: f(y) of Eq. (IVP) on a {'x'.join(map(str, slab))} slab of the workload's "
              f"initial state (the same spacing, eps and values), repeated for >= 5 s, single-threaded C oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, wl), "global_batch": 1,
                   "parallelism": "replicas (rank 0 only runs the oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------------------
# batched workload: many independent instances of uneven size in one graph launch
# ---------------------------------------------------------------------------------------
def batch_compare(wl, rank, dist, T=None, warmup=1, steps=1, plain=True):
    """The batch of independent 2D instances to T: mixed precision batched (one graph launch
    per integration), FP64 batched, and the plain FP64 method (one grid per instance, one
    instance after another).  Times are CUDA events on the stream around each integration."""
    import numpy as np
    import torch
    from paper_2502_14589_gb300 import ch, inputs, replicas
    T = wl["T"] if T is None else T
    count = wl["count"]
    sides, eps = inputs.batch_descriptors(count, seed=0)
    y0s = [inputs.initial_state((int(n), int(n)), replicas.batch_instance_seed(rank, i), wl["lo"], wl["hi"])
           for i, n in enumerate(sides)]
    Ns = np.array([int(n) * int(n) for n in sides])
    stream = torch.cuda.current_stream()
    prm = ch.make_params("ee2", True, T, wl["tau0"], wl["tol"], wl["mmax"])
    out, ys = {}, {}
    for prec, name in ((ch.CH_MIXED, "mixed_batched"), (ch.CH_FP64, "fp64_batched")):
        h = ch.ch_create_batch(2, [int(n) for n in sides], list(eps), prec, wl["mmax"], stream)
        offs, chunk = ch.ch_batch_layout(h, count)
        y0 = torch.zeros(offs[-1], dtype=torch.float64, device="cuda")
        for i in range(count):
            y0[offs[i]:offs[i] + Ns[i]] = torch.from_numpy(y0s[i]).cuda()
        y = torch.empty_like(y0)
        for _ in range(warmup):
            y.copy_(y0); ch.ch_integrate_batch(h, prm, y, count)
        ms, ops, launches = 0.0, 0, 0
        for _ in range(steps):
            y.copy_(y0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            l0 = ch.ch_batch_kernel_launches(h)
            e0.record(stream)
            st = ch.ch_integrate_batch(h, prm, y, count)
            e1.record(stream); e1.synchronize()
            ms += e0.elapsed_time(e1)
            launches += ch.ch_batch_kernel_launches(h) - l0
            ops += int(sum(Ns[i] * (st[i]["matvecs"] + st[i]["rhs_evals"]) for i in range(count)))
        yh = y.cpu().numpy()
        ys[name] = [yh[offs[i]:offs[i] + Ns[i]] for i in range(count)]
        out[name] = {"ms_to_T": ms / steps, "value": ops / (ms * 1e-3), "chunk_len": chunk,
                     "scheduling_groups": ch.ch_batch_groups(h),
                     "batch_steps": max(x["steps"] for x in st), "kernel_launches": launches // steps}
        ch.ch_destroy_batch(h)
    if plain:
        ms, ops, yp = 0.0, 0, []
        for i, n in enumerate(sides):
            G = ch.Grid(2, (int(n), int(n)), float(eps[i]), ch.CH_FP64, wl["mmax"], stream)
            y = torch.from_numpy(y0s[i]).cuda()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = ch.ch_integrate(G.h, prm, y)
            e1.record(stream); e1.synchronize()
            ms += e0.elapsed_time(e1)
            ops += int(Ns[i]) * (st["matvecs"] + st["rhs_evals"])
            yp.append(y.cpu().numpy())
            G.close()
        out["fp64_plain"] = {"ms_to_T": ms, "value": ops / (ms * 1e-3),
                             "method": "one FP64 grid per instance, integrated one after another"}
    ref = ys["fp64_batched"]
    errs = [np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(ys["mixed_batched"], ref)]
    out["mixed_batched_vs_fp64_batched"] = {"speedup": out["fp64_batched"]["ms_to_T"] / out["mixed_batched"]["ms_to_T"],
                                            "max_rel_err_at_T": float(max(errs)),
                                            "median_rel_err_at_T": float(np.median(errs))}
    if plain:
        out["mixed_batched_vs_fp64_plain"] = {"speedup": out["fp64_plain"]["ms_to_T"] / out["mixed_batched"]["ms_to_T"]}
    out["grid_points"] = int(Ns.sum())
    out["T"] = T
    return out


def run_batch_workload(args, rank, world, dist):
    import torch
    from paper_2502_14589_gb300 import build, inputs, replicas
    build.build()
    wl = dict(inputs.WORKLOADS[args.workload])
    if args.t_final is not None:
        wl["T"] = args.t_final
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    out = batch_compare(wl, rank, dist, warmup=args.warmup, steps=args.steps)
    ms, ops = replicas.combine(dist, out["mixed_batched"]["ms_to_T"] * args.steps,
                               out["mixed_batched"]["value"] * out["mixed_batched"]["ms_to_T"] * 1e-3 * args.steps,
                               "cuda")
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": ops / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 mixed",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, wl), "global_batch": wl["count"],
                       "grid_points": out["grid_points"], "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "batch": out,
        }), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm: one grid, EE2 in mixed precision and LIM in FP64 to T
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
    Gm = ch.Grid(wl["dim"], n, wl["eps"], ch.CH_MIXED, wl["mmax"], stream)     # the timed step
    Gd = ch.Grid(wl["dim"], n, wl["eps"], ch.CH_FP64, wl["mmax"], stream)      # the plain FP64 method
    prm = {s: ch.make_params(s, True, wl["T"], wl["tau0"], wl["tol"], wl["mmax"]) for s in ("ee2", "lim")}
    grid_of = {"ee2": Gm, "lim": Gd}
    y_at_T = {s: torch.empty_like(y0) for s in ("ee2", "lim")}

    def one_step(yin, record=None):
        stats = {}
        for s in ("ee2", "lim"):
            y.copy_(yin)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats[s] = ch.ch_integrate(grid_of[s].h, prm[s], y)
            e1.record(stream)
            y_at_T[s].copy_(y)
            if record is not None:
                record[s].append((e0, e1, stats[s]))
        return stats

    for _ in range(args.warmup):
        one_step(y0)
    torch.cuda.synchronize()

    # ---- timed region: K steps, events per step, L2 flushed between steps.  Every launch of
    # the dominant kernel (the FP32 Arnoldi iteration of EE2) is timed with CUDA events on the
    # grid's stream inside the timed steps (launches that found their Krylov run ended and
    # returned at once excluded); the library sums each launch's algorithmic bytes and flops.
    # On grids below 4M points an iteration takes tens of microseconds and the per-launch events
    # would perturb the timed step; there the kernel is timed over t in [0, T/20] instead.
    in_step = N >= (1 << 22)
    ch.ch_timing_start(Gm.h, "arnoldi" if in_step else None)
    ch.ch_timing_start(Gd.h, None)          # per-class launch counts, no per-kernel events
    launches0 = ch.ch_kernel_launches(Gm.h) + ch.ch_kernel_launches(Gd.h)
    clocks = ClockSampler()
    if rank == 0:
        clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, ops, rec = [], 0, {"ee2": [], "lim": []}
    for _ in range(args.steps):
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
    launches = ch.ch_kernel_launches(Gm.h) + ch.ch_kernel_launches(Gd.h) - launches0
    counts = {}
    arn_ms, arn_n, cm = ch.ch_timing_read(Gm.h)
    arn_fl, arn_by = ch.ch_timing_work(Gm.h)
    ch.ch_timing_start(Gm.h, None)
    for c in (cm, ch.ch_timing_read(Gd.h)[2]):
        for k, v in c.items():
            counts[k] = counts.get(k, 0) + v
    total_ms, ops = replicas.combine(dist, sum(step_ms), ops, dev)
    value = ops / (total_ms * 1e-3)
    ttt = {}
    for s, prec in (("ee2", "mixed"), ("lim", "fp64")):
        ms = [e0.elapsed_time(e1) for e0, e1, _ in rec[s]]
        st = rec[s][-1][2]
        ttt[s] = {"precision": prec, "ms": sum(ms) / len(ms), "steps": st["steps"], "matvecs": st["matvecs"],
                  "rhs_evals": st["rhs_evals"], "phi_evals": st["phi_evals"], "tau_shrinks": st["tau_shrinks"],
                  "ops_per_s": N * (st["matvecs"] + st["rhs_evals"]) / (sum(ms) / len(ms) * 1e-3)}

    # ---- the plain FP64 EE2 on the same grid: time to T and the mixed run's error at T ----
    y.copy_(y0)
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st64 = ch.ch_integrate(Gd.h, prm["ee2"], y)
    e1.record(stream); e1.synchronize()
    ms64 = e0.elapsed_time(e1)
    mixed_vs_fp64 = {"ee2": {"fp64_ms_to_T": ms64, "mixed_ms_to_T": ttt["ee2"]["ms"], "speedup": ms64 / ttt["ee2"]["ms"],
                             "rel_err_at_T_vs_fp64": float(torch.linalg.norm(y_at_T["ee2"] - y) / torch.linalg.norm(y)),
                             "fp64_steps": st64["steps"], "mixed_steps": ttt["ee2"]["steps"],
                             "mixed_mass_drift": float(abs(y_at_T["ee2"].mean() - y0.mean()))}}
    # mixed-precision LIM: adaptive to T (time; its adaptive step sequence departs from the
    # FP64 run's, so the difference at T measures Eq. (LIMdt)'s sensitivity), and 200 constant
    # steps against the same 200 FP64 steps (the precision effect alone)
    y.copy_(y0)
    e0.record(stream)
    stm = ch.ch_integrate(Gm.h, prm["lim"], y)
    e1.record(stream); e1.synchronize()
    lim_m_ms = e0.elapsed_time(e1)
    lim_adapt_diff = float(torch.linalg.norm(y - y_at_T["lim"]) / torch.linalg.norm(y_at_T["lim"]))
    tau_c = 1e-9
    pc = ch.make_params("lim", False, 200 * tau_c, tau_c, wl["tol"], wl["mmax"])
    yc = {}
    for name, G in (("mixed", Gm), ("fp64", Gd)):
        y.copy_(y0)
        e0.record(stream)
        ch.ch_integrate(G.h, pc, y)
        e1.record(stream); e1.synchronize()
        yc[name] = (y.clone(), e0.elapsed_time(e1))
    mixed_vs_fp64["lim"] = {
        "mixed_adaptive_ms_to_T": lim_m_ms, "fp64_adaptive_ms_to_T": ttt["lim"]["ms"],
        "mixed_adaptive_steps": stm["steps"], "fp64_adaptive_steps": ttt["lim"]["steps"],
        "adaptive_runs_rel_diff_at_T": lim_adapt_diff,
        "same_200_steps_tau_1e-9": {"mixed_ms": yc["mixed"][1], "fp64_ms": yc["fp64"][1],
                                    "rel_err": float(torch.linalg.norm(yc["mixed"][0] - yc["fp64"][0])
                                                     / torch.linalg.norm(yc["fp64"][0]))}}

    # ---- end to end through the C ABI with host buffers (one step) ---------------------------
    y_host = torch.from_numpy(y0_host.copy()).pin_memory()
    out_host = torch.empty(N, dtype=torch.float64).pin_memory()
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_ops = 0
    for s in ("ee2", "lim"):
        y.copy_(y_host, non_blocking=True)
        st = ch.ch_integrate(grid_of[s].h, prm[s], y)
        out_host.copy_(y, non_blocking=True)
        e2e_ops += N * (st["matvecs"] + st["rhs_evals"])
    e1.record(stream); e1.synchronize()
    e2e = {"value": e2e_ops / (e0.elapsed_time(e1) * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": 2 * N * 8}

    # ---- roofline of the dominant kernel, measured live: every launch of the FP32 Arnoldi
    # iteration (Gram-corrected, HBM-bound) timed with CUDA events on the grid's stream over
    # t in [0, T/20] of the same workload (graphs off while launches are timed); the library
    # sums each launch's algorithmic bytes and flops from its Krylov dimension and N.  The
    # FP64 LIM kernels (FP64-issue bound) are timed the same way against the measured FP64 peak.
    fp64_peak = ch.ch_probe_fp64_peak(stream)
    live = {}
    where = "every launch of the timed steps"
    if not in_step:
        y.copy_(y0)
        ch.ch_timing_start(Gm.h, "arnoldi")
        ch.ch_integrate(Gm.h, ch.make_params("ee2", True, wl["T"] / 20, wl["tau0"], wl["tol"], wl["mmax"]), y)
        arn_ms, arn_n, _ = ch.ch_timing_read(Gm.h)
        arn_fl, arn_by = ch.ch_timing_work(Gm.h)
        ch.ch_timing_start(Gm.h, None)
        where = "every launch of EE2 over t in [0, T/20]"
    if arn_n > 0 and arn_ms > 0:
        live["arnoldi"] = {"launches": arn_n, "avg_us": 1e3 * arn_ms / arn_n, "gbs": arn_by / (arn_ms * 1e-3) / 1e9,
                           "tflops": arn_fl / (arn_ms * 1e-3) / 1e12, "bytes_per_launch": arn_by / arn_n,
                           "flops_per_launch": arn_fl / arn_n, "total_ms": arn_ms, "where": where}
    for cls in ("lim2", "resid1"):
        y.copy_(y0)
        ch.ch_timing_start(Gd.h, cls)
        ch.ch_integrate(Gd.h, ch.make_params("lim", True, wl["T"] / 20, wl["tau0"], wl["tol"], wl["mmax"]), y)
        ms, nt, _ = ch.ch_timing_read(Gd.h)
        fl, by = ch.ch_timing_work(Gd.h)
        ch.ch_timing_start(Gd.h, None)
        if nt > 0 and ms > 0:
            live[cls + "_fp64"] = {"launches": nt, "avg_us": 1e3 * ms / nt, "gbs": by / (ms * 1e-3) / 1e9,
                                   "tflops": fl / (ms * 1e-3) / 1e12, "bytes_per_launch": by / nt,
                                   "flops_per_launch": fl / nt, "where": "LIM over t in [0, T/20]"}
    roof = None
    if "arnoldi" in live:
        kl = live["arnoldi"]
        ratio = profile_traffic_ratio()
        roof = {"kernel": "k_arnoldi_gmgs", "bound": "hbm", "achieved": kl["gbs"], "peak": HBM_GBS, "unit": "GB/s",
                "frac": kl["gbs"] / HBM_GBS,
                "traffic": None if ratio is None else ratio * kl["bytes_per_launch"],
                "peak_source": f"{HBM_SOURCE} (MEASURED_PEAKS.json hbm_gbs)" if HBM_SOURCE == "measured" else "fallback",
                "measured": f"{kl['launches']} launches ({where}), CUDA events on the grid's stream",
                "avg_launch_us": kl["avg_us"], "algorithmic_bytes_per_launch": kl["bytes_per_launch"],
                "algorithmic_flops_per_launch": kl["flops_per_launch"]}
        if in_step:
            roof["share_of_step"] = kl["total_ms"] / total_ms
    fp64_kernels = {c: {**live[c], "frac_of_measured_fp64": live[c]["tflops"] / fp64_peak}
                    for c in ("lim2_fp64", "resid1_fp64") if c in live}
    # the dominant kernel in isolation at a fixed Krylov dimension (j = 10): 20 back-to-back
    # launches in a CUDA graph, events around it (an NVTX range "ch_bench_kernel" marks them)
    kb = ch.ch_bench_kernel(Gm.h, "arnoldi", 20)
    isolated = {"kernel": "k_arnoldi_gmgs", "j": 10, "avg_us": kb["avg_us"],
                "algorithmic_bytes": kb["bytes"], "gbs": kb["bytes"] / (kb["avg_us"] * 1e-6) / 1e9,
                "frac_of_hbm": kb["bytes"] / (kb["avg_us"] * 1e-6) / 1e9 / HBM_GBS}

    # ---- the batched workload (256 2D instances of uneven size to T = 1e-4), once: mixed
    # precision batched against FP64 batched and the plain FP64 method instance by instance
    batch = None
    if args.workload == DEFAULT_WORKLOAD and args.t_final is None:
        Gm.close(); Gd.close()
        del flush
        torch.cuda.empty_cache()
        batch = batch_compare(dict(inputs.WORKLOADS["c3_batch256"]), rank, dist)
        batch["workload"] = workload_desc("c3_batch256", inputs.WORKLOADS["c3_batch256"])

    # ---- CPU baseline (oracle on a bounded sample, rank 0 only, N = 1) -----------------
    cpu = None
    if rank == 0 and world == 1:
        from oracle import oracle
        oracle.build()
        c_ops, c_s, slab = oracle_sample(wl, 0, y0_host, budget_s=15.0)
        cpu = {"value": c_ops / c_s, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"f(y) of Eq. (IVP) on a {'x'.join(map(str, slab))} slab of the workload's initial "
                         f"state (same spacing, eps, values), {c_ops // (int(np.prod(slab)))} evaluations in "
                         f"{c_s:.1f} s single-threaded on the host"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "ee2 f32/f64 mixed, lim f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, wl), "global_batch": world, "grid_points": N,
                       "step": "EE2 (mixed precision) to T, then LIM (FP64) to T, from the same state",
                       "mixed_precision": "FP32 Krylov basis and stencils; FP64 state, projected phi, H, "
                                          "combine and control; inner products and norms summed as "
                                          "compensated FP32 pairs in double-float (about 2^-44 relative), "
                                          "not in FP64 arithmetic",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed (256 MiB write) before every timed step; every vector of the workload exceeds L2"},
            "time_to_T": ttt, "mixed_vs_fp64": mixed_vs_fp64, "e2e": e2e, "gpu_launches": launches,
            "launches_by_kernel": counts, "roofline": roof, "kernels_live": live, "fp64_kernels": fp64_kernels,
            "dominant_isolated": isolated,
            "fp64_peak_tflops": {"measured": fp64_peak, "how": "ch_probe_fp64_peak: FMA chains from registers"},
            "hbm_peak_gbs": HBM_GBS, "cpu_baseline": cpu, "clocks": clk, "batch_c3": batch,
        }
        print(json.dumps(out), flush=True)
    Gm.close(); Gd.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
