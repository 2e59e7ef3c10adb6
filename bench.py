#!/usr/bin/env python
"""Time-to-converge of coupled-cluster doubles for pure neutron matter on one GB300.

A step is one complete CCD solve (MBPT2 start, updates until |dE^(n+1) - dE^(n)| / N <
1e-6 MeV) of the workload N = 14 neutrons, rho = 0.08 fm^-3, plane waves with n^2 <= 20
(778 states), Minnesota interaction, mixing alpha = 0.5.  The channel tables and the
interaction blocks are resident in HBM before the timed region (built by the context); the
timed region covers the solve.  ``e2e`` repeats the measurement through the public API
from host inputs: context creation (basis, channels and V built on the GPU), solve, and the
converged amplitudes copied back to the host.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle (the only reference
implementation of this method) on the same workload and metric.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PNM CCD time-to-converge (ΔE/N<1e-6 MeV), mixed+learned vs FP64, one GB300"
WORKLOADS = {
    # name: (N, rho, n2max)
    "pnm_N14_rho0.08_n2max20": (14, 0.08, 20),
    "pnm_N14_rho0.08_n2max4": (14, 0.08, 4),
    "pnm_N66_rho0.16_n2max36": (66, 0.16, 36),
}
DEFAULT_WORKLOAD = "pnm_N14_rho0.08_n2max20"
MINNESOTA = (200.0, 1.487, -178.0, 0.639, -91.85, 0.465, 20.721)
TOL_PER_N = 1e-6
ALPHA = 0.5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "bf16x3"])
    ap.add_argument("--refine", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the FP64 / N=66 comparison runs")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while active."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value, dist, device="cpu"):
    """Largest value over all ranks (the slowest rank sets the job time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def chan_sizes(ctx, sys_=0):
    keys, sizes, _ = ctx.channels(sys_, 0)
    xk, xs, _ = ctx.channels(sys_, 1)
    szero = (keys % 3) == 1
    return sizes[:, 0].astype(float), sizes[:, 1].astype(float), szero, xs[:, 0].astype(float), xs[:, 1].astype(float)


def algorithmic_cost(ctx, kernel, prec):
    """(bytes, flops) per launch of a kernel, from the channel sizes: each array the kernel
    must touch, counted once."""
    nhh, npp, szero, nph, nhp = chan_sizes(ctx)
    nt = float((nhh * npp).sum())
    if kernel in ("k_pp64", "k_pp_tc"):
        vb = 8.0 if kernel == "k_pp64" else 4.0          # FP64 V, or BF16 hi + lo
        tb = 8.0 if kernel == "k_pp64" else 4.0          # t operand
        byts = float((npp[szero] ** 2).sum()) * vb + float((nhh[szero] * npp[szero]).sum()) * (tb + 8.0)
        flops = 2.0 * float((nhh[szero] * npp[szero] ** 2).sum()) * (1 if kernel == "k_pp64" else 3)
        return byts, flops
    if kernel in ("k_ph64", "k_ph32"):
        eb = 8.0 if kernel == "k_ph64" else 4.0
        byts = float((nph * nhp).sum()) * (4 + eb + eb) + float((nhp * nhp).sum()) * eb + nt * eb
        flops = 2.0 * float((nhp * nhp * nph + nph * nhp * nhp).sum())
        return byts, flops
    if kernel in ("k_update", "k_update_mix"):
        return nt * (8 + 8 + 8 + 16 + 4 * 8 + 8 + 8), nt * 20.0
    if kernel in ("k_tstats", "k_tstats32"):
        return nt * 8 * 2 + float((nhh * nhh).sum()) * 16, nt * 2.0 * (2 + nhh.mean())
    return nt * 8.0, 0.0


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# FP64 FMA rate of GB300: 152 SMs x 2 FP64 FMA per clock per SM x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def oracle_time(N, rho, n2max, budget_s=8.0, max_runs=50):
    """Median wall time (ms) of full oracle solves, repeated within a time budget."""
    from oracle import channel
    times = []
    t_start = time.perf_counter()
    dE = it = None
    while len(times) < max_runs and (time.perf_counter() - t_start) < budget_s or len(times) < 1:
        t0 = time.perf_counter()
        o = channel.OracleSystem(N, rho, n2max, MINNESOTA)
        dE, it, _, _ = o.ccd(alpha=ALPHA, tol=TOL_PER_N * N, maxit=500)
        times.append((time.perf_counter() - t0) * 1e3)
        del o
    return statistics.median(times), len(times), channel.threads(), dE, it


# ------------------------------------------------------------------------------ arms

def run_reference(a):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    N, rho, n2max = WORKLOADS[a.workload]
    from oracle import build as ob
    ob.build()
    from oracle import channel
    for _ in range(max(0, min(a.warmup, 1))):
        oracle_time(N, rho, n2max, budget_s=0.0, max_runs=1)
    times = []
    dE = it = None
    for _ in range(a.steps):
        t0 = time.perf_counter()
        o = channel.OracleSystem(N, rho, n2max, MINNESOTA)
        dE, it, _, _ = o.ccd(alpha=ALPHA, tol=TOL_PER_N * N, maxit=500)
        times.append((time.perf_counter() - t0) * 1e3)
        del o
    ms = statistics.mean(times)
    cores = channel.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": a.workload, "N": N, "rho": rho, "n2max": n2max,
                   "tol_dE_per_N": TOL_PER_N, "mix_alpha": ALPHA, "l2": "host"},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": "%d full FP64 solves of the workload (setup + iterations) on the host" % a.steps},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "result": {"dE_per_N": dE / N, "iters": it},
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_solves(ctx, solve_kw, steps, flush, stream, torch):
    """Per-solve device times (ms) with an L2 flush outside each timed region."""
    evs, iters, dEs = [], [], []
    for _ in range(steps):
        flush.zero_()  # 512 MB write > 129 MB L2, outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dE, it, _, _ = ctx.solve(**solve_kw)
        e1.record(stream)
        evs.append((e0, e1))
        iters.append(int(it[0]))
        dEs.append(float(dE[0]))
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in evs], iters, dEs


def solve_kwargs(P, prec, refine):
    return dict(precision=prec, alpha=ALPHA, tol=1e-30, tol_per_N=TOL_PER_N, max_iter=500,
                refine_sweeps=refine if prec == P.PNM_PREC_BF16X3 else 0)


def measure_other(P, torch, stream, flush, workload, prec, refine, steps):
    """Mean time-to-converge (ms) and iterations of another workload/precision."""
    N, rho, n2max = WORKLOADS[workload]
    ctx = P.Context(N, rho, n2max, params=MINNESOTA, stream=stream.cuda_stream)
    kw = solve_kwargs(P, prec, refine)
    for _ in range(3):
        ctx.solve(**kw)
    torch.cuda.synchronize()
    ms, iters, dEs = timed_solves(ctx, kw, steps, flush, stream, torch)
    tim = ctx.timings()
    ctx.close()
    return {"ms": statistics.mean(ms), "iters": statistics.mean(iters), "dE_per_N": statistics.mean(dEs) / N,
            "mixed_phase_ms": tim["mixed"], "refine_ms": tim["refine"]}


def measure_batch(P, torch, stream, flush, refine, steps):
    """16 densities (0.02..0.32) of N=14, n^2<=20 solved together in one context: every kernel
    launch covers all systems; the loop ends when all have converged."""
    rhos = [0.02 * k for k in range(1, 17)]
    ctx = P.Context(14, rhos, 20, params=MINNESOTA, stream=stream.cuda_stream)
    out = {}
    for pn, pv in (("bf16x3", P.PNM_PREC_BF16X3), ("fp64", P.PNM_PREC_FP64)):
        kw = solve_kwargs(P, pv, refine)
        for _ in range(3):
            ctx.solve(**kw)
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dE, it, _, _ = ctx.solve(**kw)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        out[pn] = {"ms": statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs),
                   "iters_max": int(max(it)), "dE_per_N": [float(x) / 14 for x in dE]}
    ctx.close()
    return out


def measure_learned(P, torch, stream, flush, refine, steps):
    """Learned warm start: train on solver amplitudes of N=14 (n^2<=20, 16 densities) and
    N=66 (n^2<=36, rho=0.16), then time N=66 solves at held-out densities from the learned
    start, from the MBPT2 start (both mixed precision) and in FP64."""
    kw64 = dict(precision=P.PNM_PREC_FP64, alpha=ALPHA, tol=1e-30, tol_per_N=1e-8, max_iter=500)
    t0 = time.perf_counter()
    tr14 = P.Context(14, [0.02 * k for k in range(1, 17)], 20, params=MINNESOTA, stream=stream.cuda_stream)
    tr14.solve(**kw64)
    tr66 = P.Context(66, 0.16, 36, params=MINNESOTA, stream=stream.cuda_stream)
    tr66.solve(**kw64)
    blob, hist = P.mlp_train([tr14, tr66], P.mlp_init(seed=1), epochs=12, batch=4096, lr=1e-3, seed=2)
    train_s = time.perf_counter() - t0
    tr14.close()
    tr66.close()
    res = {"train_s": train_s, "train_loss_first_last": [float(hist[0]), float(hist[-1])], "rho": {}}
    for rho in (0.05, 0.11, 0.17):
        ctx = P.Context(66, rho, 36, params=MINNESOTA, stream=stream.cuda_stream)
        ctx.mlp_set_model(blob)
        row = {}
        for name, prec, init in (("bf16x3_learned", P.PNM_PREC_BF16X3, P.PNM_INIT_MLP),
                                 ("bf16x3_mbpt2", P.PNM_PREC_BF16X3, P.PNM_INIT_MBPT2),
                                 ("fp64_mbpt2", P.PNM_PREC_FP64, P.PNM_INIT_MBPT2)):
            kw = solve_kwargs(P, prec, refine)
            kw["init"] = init
            for _ in range(3):
                ctx.solve(**kw)
            ms, iters, dEs = timed_solves(ctx, kw, steps, flush, stream, torch)
            row[name] = {"ms": statistics.mean(ms), "iters": statistics.mean(iters),
                         "dE_per_N": statistics.mean(dEs) / 66}
        ctx.close()
        res["rho"][str(rho)] = row
    return res


def run_ours(a):
    world, rank, local = dist_setup()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1611_06765_gb300 import build as pb
    pb.build()
    import paper_1611_06765_gb300 as P
    N, rho, n2max = WORKLOADS[a.workload]
    prec_name = "bf16x3" if a.precision == "auto" else a.precision
    prec = P.PNM_PREC_BF16X3 if prec_name == "bf16x3" else P.PNM_PREC_FP64
    refine = a.refine if prec == P.PNM_PREC_BF16X3 else 0
    stream = torch.cuda.current_stream()
    ctx = P.Context(N, rho, n2max, params=MINNESOTA, stream=stream.cuda_stream)
    solve_kw = solve_kwargs(P, prec, a.refine)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, a.warmup)):
        flush.zero_()
        ctx.solve(**solve_kw)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        step_ms, iters, dEs = timed_solves(ctx, solve_kw, a.steps, flush, stream, torch)
        wall = time.perf_counter() - wall0
    ms = statistics.mean(step_ms)
    if dist:
        ms = max_over_ranks(ms, dist, device="cuda")
    tim = ctx.timings()

    # e2e through the public API from host inputs
    e2e_ms = []
    n_t = None
    for k in range(max(1, min(a.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = P.Context(N, rho, n2max, params=MINNESOTA, stream=stream.cuda_stream)
        c2.solve(**solve_kw)
        amps = c2.get_amplitudes()
        c2.close()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        n_t = amps.size

    # per-kernel durations from one profiled host-driven solve of the same work
    ctx.set_profiling(True)
    ctx.solve(host_loop=True, **solve_kw)
    stats = ctx.kernel_stats()
    ctx.set_profiling(False)
    dom = max(stats.items(), key=lambda kv: kv[1][0])
    kname, (ktot, kn) = dom
    kavg_s = ktot / kn / 1e3
    byts, flops = algorithmic_cost(ctx, kname, prec)
    hbm, bf16, src = read_peaks()
    if kname == "k_pp64":
        roof = {"bound": "alu", "achieved": flops / kavg_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "FP64 DFMA rate derived from SM count and clock"}
    else:
        roof = {"bound": "hbm", "achieved": byts / kavg_s / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": "%s hbm_gbs" % src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["kernel"] = kname
    roof["kernel_avg_us"] = kavg_s * 1e6
    roof["algorithmic_bytes"] = byts
    roof["algorithmic_flops"] = flops
    body = 6 if prec == P.PNM_PREC_BF16X3 else 5
    launches_per_solve = 2 + body * statistics.mean(iters) + (1 if refine else 0)

    comparison = None
    if rank == 0 and not a.no_extra:
        comparison = {}
        other = P.PNM_PREC_FP64 if prec == P.PNM_PREC_BF16X3 else P.PNM_PREC_BF16X3
        comparison[a.workload + ("_fp64" if other == P.PNM_PREC_FP64 else "_bf16x3")] = measure_other(
            P, torch, stream, flush, a.workload, other, a.refine, max(5, a.steps // 2))
        if a.workload != "pnm_N66_rho0.16_n2max36":
            for pn, pv in (("bf16x3", P.PNM_PREC_BF16X3), ("fp64", P.PNM_PREC_FP64)):
                comparison["pnm_N66_rho0.16_n2max36_" + pn] = measure_other(
                    P, torch, stream, flush, "pnm_N66_rho0.16_n2max36", pv, a.refine, 3)
        comparison["density_batch_N14_n2max20_16rho"] = measure_batch(P, torch, stream, flush, a.refine, 3)
        comparison["learned_start_N66_n2max36_heldout"] = measure_learned(P, torch, stream, flush, a.refine, 3)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        from oracle import build as ob
        ob.build()
        cms, runs, cores, dE_o, it_o = oracle_time(N, rho, n2max)
        cpu = {"value": cms, "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": "median of %d full FP64 oracle solves of the workload (setup + %d iterations)" % (runs, it_o),
               "dE_per_N": dE_o / N, "gpu_minus_oracle_dE_per_N": statistics.mean(dEs) / N - dE_o / N}

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": a.steps,
            "warmup": max(3, a.warmup), "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == P.PNM_PREC_FP64 else "bf16x3+f32+f64",
            "data": "synthetic",
            "config": {"workload": a.workload, "N": N, "rho": rho, "n2max": n2max,
                       "precision": prec_name, "refine_sweeps": refine, "mix_alpha": ALPHA,
                       "tol_dE_per_N": TOL_PER_N, "l2": "flushed (512 MB write) before every step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "clocks": clk.summary(),
            "e2e": {"value": statistics.mean(e2e_ms), "unit": "ms",
                    "h2d_bytes_per_step": 4 + 8 + 4 + 7 * 8,
                    "d2h_bytes_per_step": 8 * (n_t or 0) + 8 + 4 + 8},
            "gpu_launches": int(round(launches_per_solve * a.steps)),
            "roofline": roof,
            "cpu_baseline": cpu,
            "comparison": comparison,
            "tuning": (dict(zip(("k_splits", "stages", "pp_tc_us", "serial_mask"), ctx.tuning()))
                       if prec == P.PNM_PREC_BF16X3 else None),
            "result": {"dE_per_N": statistics.mean(dEs) / N, "iters": statistics.mean(iters),
                       "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms),
                       "wall_ms_per_step": wall * 1e3 / a.steps, "setup_ms": tim["setup"],
                       "mixed_phase_ms": tim["mixed"], "refine_ms": tim["refine"],
                       "kernels_ms_per_solve": {k: v[0] for k, v in stats.items()}},
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
