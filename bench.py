#!/usr/bin/env python
"""Time-to-converge of coupled-cluster doubles for pure neutron matter on one GB300.

Metric: device time for the CCD iteration to reach |dE^(n+1) - dE^(n)| / N < 1e-6 MeV.

Default workload, the one the metric's "mixed + learned" is defined on: N = 66 neutrons,
plane waves with n^2 <= 36 (1850 states), Minnesota interaction, mixing 0.5, at the three
held-out densities rho = 0.05, 0.11, 0.17 fm^-3, solved together in one batched context
(every kernel launch covers the three systems).  A step is one converged solve of that batch
from the learned start (the tensor-core inference of the network, which forms each sample's
features from the context in registers, and the copy to the spin flips, inside the timed
region), the pp ladder in BF16x3 on the tensor cores, FP64 denominators / residual /
energies, and two FP64 refinement sweeps at the end (their contractions in FP32 pairs).  The
network is trained before timing, by the library's own GPU kernels, on amplitudes the solver
converges for N = 14 (n^2 <= 20, 16 densities 0.02 ... 0.32) and N = 66 (n^2 <= 36, rho =
0.04, 0.06, ..., 0.20).  Channel tables, interaction blocks and the model are resident
in HBM before the timed region; L2 is flushed before every step.

``e2e`` times the public API from host inputs: context creation (basis, channels and V built
on the GPU), model upload, solve, converged amplitudes copied back.  ``comparison`` holds the
same batch from the MBPT2 start (mixed and FP64) and the other configurations, each with its
dE/N error against the FP64 oracle, a twist-averaged batch (N = 14, n^2 <= 20, rho = 0.08,
120 twists of a 4 x 5 x 6 Gauss-Legendre mesh in one context) in both precisions, the ladder
truncations of Eqs. ccd1 and ccd2 (N = 66, n^2 <= 36, rho = 0.16, FP64) and the third-order
diagrams of the held-out batch (pnm_mbpt3, with the oracle's time and values), and symmetric
nuclear matter (14 protons + 14 neutrons, rho = 0.16, n^2 <= 20) in both precisions.  ``--impl reference`` times the FP64 CPU oracle.

Prints one JSON line.
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
HELDOUT = (0.05, 0.11, 0.17)
# N = 66 densities of the warm-start training set (the held-out ones are not among them)
TRAIN66 = (0.04, 0.06, 0.08, 0.10, 0.12, 0.14, 0.16, 0.18, 0.20)
TRAIN_SEED = 3  # shuffling seed of the warm-start training (initial weights: seed 1)
SWEEP16 = tuple(round(0.02 * k, 2) for k in range(1, 17))
WORKLOADS = {
    # name: (N, densities, n2max, start, precision, contractions of the refinement sweeps)
    # "f32pair": FP32-pair contractions (48 significant bits on the FP32 pipe, FP64 results);
    # "fp64": the FP64 pipe.  The update, denominators, residual and energy are FP64 in both.
    "pnm_N66_n2max36_heldout3_learned_bf16x3": (66, HELDOUT, 36, "mlp", "bf16x3", "f32pair"),
    "pnm_N66_n2max36_heldout3_learned_bf16x3_fp64refine": (66, HELDOUT, 36, "mlp", "bf16x3", "fp64"),
    "pnm_N66_n2max36_heldout3_mbpt2_bf16x3": (66, HELDOUT, 36, "mbpt2", "bf16x3", "f32pair"),
    "pnm_N66_n2max36_heldout3_mbpt2_fp64": (66, HELDOUT, 36, "mbpt2", "fp64", None),
    "pnm_N14_rho0.08_n2max20_bf16x3": (14, (0.08,), 20, "mbpt2", "bf16x3", "f32pair"),
    "pnm_N14_rho0.08_n2max20_fp64": (14, (0.08,), 20, "mbpt2", "fp64", None),
    "pnm_N66_rho0.16_n2max36_bf16x3": (66, (0.16,), 36, "mbpt2", "bf16x3", "f32pair"),
    "pnm_N66_rho0.16_n2max36_fp64": (66, (0.16,), 36, "mbpt2", "fp64", None),
    "pnm_N14_n2max20_16rho_bf16x3": (14, SWEEP16, 20, "mbpt2", "bf16x3", "f32pair"),
    "pnm_N14_n2max20_16rho_fp64": (14, SWEEP16, 20, "mbpt2", "fp64", None),
    "pnm_N14_rho0.08_n2max4_fp64": (14, (0.08,), 4, "mbpt2", "fp64", None),
}
# Twist-averaged boundary conditions: one system per point of a product Gauss-Legendre twist
# mesh (4 x 5 x 6 nodes on [0, pi]: no two equal components, so no mesh point has a
# degenerate Fermi level), all in one batched context.  name: (N, rho, n2max, mesh, precision)
TWIST_WORKLOADS = {
    "pnm_N14_rho0.08_n2max20_tabc4x5x6_bf16x3": (14, 0.08, 20, (4, 5, 6), "bf16x3"),
    "pnm_N14_rho0.08_n2max20_tabc4x5x6_fp64": (14, 0.08, 20, (4, 5, 6), "fp64"),
}
# Truncated iterations (Eq. ccd1: pp ladder; Eq. ccd2: pp and hh ladders), FP64, and the
# third-order diagrams.  name: (N, densities, n2max, terms)
TRUNC_WORKLOADS = {
    "pnm_N66_rho0.16_n2max36_ccd1_pp_fp64": (66, (0.16,), 36, "pp"),
    "pnm_N66_rho0.16_n2max36_ccd2_pphh_fp64": (66, (0.16,), 36, "pphh"),
}
MBPT3_WORKLOAD = ("pnm_N66_n2max36_heldout3_mbpt3_fp64", 66, HELDOUT, 36)
# Symmetric nuclear matter (14 protons and 14 neutrons).  name: (N, Z, rho, n2max, precision)
NUCLEAR_WORKLOADS = {
    "snm_A28_rho0.16_n2max20_bf16x3": (14, 14, 0.16, 20, "bf16x3"),
    "snm_A28_rho0.16_n2max20_fp64": (14, 14, 0.16, 20, "fp64"),
}
DEFAULT_WORKLOAD = "pnm_N66_n2max36_heldout3_learned_bf16x3"
COMPARE = ["pnm_N66_n2max36_heldout3_learned_bf16x3", "pnm_N66_n2max36_heldout3_learned_bf16x3_fp64refine",
           "pnm_N66_n2max36_heldout3_mbpt2_bf16x3",
           "pnm_N66_n2max36_heldout3_mbpt2_fp64", "pnm_N14_rho0.08_n2max20_bf16x3",
           "pnm_N14_rho0.08_n2max20_fp64", "pnm_N66_rho0.16_n2max36_bf16x3", "pnm_N66_rho0.16_n2max36_fp64",
           "pnm_N14_n2max20_16rho_bf16x3", "pnm_N14_n2max20_16rho_fp64"]
MINNESOTA = (200.0, 1.487, -178.0, 0.639, -91.85, 0.465, 20.721)
TOL_PER_N = 1e-6
# DRAM bytes (read + write) per launch of the default workload from one ncu capture, with the
# first 16 hex digits of the SHA-256 of the kernel's source file at the time of the capture:
# reported only while that file is unchanged, else null.
TRAFFIC = {"k_update_mix": (154537728.0, "19db074b78c7acf1"), "k_pp_tc": (257623040.0, "53dafb1834d94e42")}
ALPHA = 0.5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--refine", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the comparison workloads")
    ap.add_argument("--model", default=None, help="load the warm-start network (.npy) instead of training it")
    ap.add_argument("--save-model", default=None, help="write the trained warm-start network (.npy)")
    ap.add_argument("--train-epochs", type=int, default=40, help="warm-start training epochs")
    ap.add_argument("--train-batch", type=int, default=1024, help="warm-start training batch")
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


def chan_sizes(ctx):
    """Channel sizes of every system of a context, concatenated; for cross channels also the
    sign of S_z = s_a - s_i (the ph kernels form S_z > 0 channels in full and mirror them onto
    S_z < 0, and S_z = 0 channels as half-size sum and difference blocks)."""
    import numpy as np
    nhh, npp, nlad, nph, nhp, xsz, nself = [], [], [], [], [], [], []
    for s in range(ctx.nsys):
        _, sizes, dpairs = ctx.channels(s, 0)
        _, xs, xpairs = ctx.channels(s, 1)
        nv, _, _ = ctx.basis(s)
        w = nv[:, 3].astype(int)
        spin = np.where(np.abs(w) == 1, w, w - 4 * np.sign(w))
        first = np.concatenate([[0], np.cumsum(xs[:, 0])[:-1]]).astype(int)
        # hole pairs that the spin flip maps onto themselves (same momentum and species,
        # opposite spin): the rows of a channel the updates compute are (n_hh + these) / 2
        hh = dpairs[: int(sizes[:, 0].sum())]
        selfp = (np.all(nv[hh[:, 0], :3] == nv[hh[:, 1], :3], axis=1)
                 & (w[hh[:, 0]] - spin[hh[:, 0]] == w[hh[:, 1]] - spin[hh[:, 1]]))
        hoff = np.concatenate([[0], np.cumsum(sizes[:, 0])[:-1]]).astype(int)
        nself.append(np.add.reduceat(selfp.astype(int), hoff) if len(hh) else np.zeros(len(sizes), int))
        nhh.append(sizes[:, 0])
        npp.append(sizes[:, 1])
        nlad.append(ctx.ladder_sizes(s))
        nph.append(xs[:, 0])
        nhp.append(xs[:, 1])
        xsz.append(np.sign(spin[xpairs[first, 0]] - spin[xpairs[first, 1]]))
    cat = lambda v: np.concatenate(v).astype(float)
    return cat(nhh), cat(npp), cat(nlad), cat(nph), cat(nhp), cat(xsz), cat(nself)


def algorithmic_cost(ctx, kernel):
    """(bytes, flops) per launch of a kernel, from the channel sizes of all systems of the
    context: every array the kernel must touch, counted once."""
    nhh, npp, nlad, nph, nhp, xsz, nself = chan_sizes(ctx)
    nt = float((nhh * npp).sum())
    # the updates compute one amplitude of each spin-flip pair and write both
    ncomp = 0.5 * nt
    if kernel == "k_pp_f2":
        kernel = "k_pp64"  # same arrays (V as FP32 pairs, 8 bytes) and the same flops
    if kernel in ("k_pp64", "k_pp_tc"):
        # the ladder in its basis (pnm_ladder_sizes): V block n_lad x n_lad, operand and result
        # rows x n_lad per channel; k_pp64 takes the rows the update computes, (n_hh + self
        # pairs) / 2 (exact for S_z = 0 channels, right in total over a channel and its flip),
        # k_pp_tc every row
        rows = 0.5 * (nhh + nself) if kernel == "k_pp64" else nhh
        vb = 8.0 if kernel == "k_pp64" else 4.0          # FP64 V, or BF16 hi + lo
        tb = 8.0 if kernel == "k_pp64" else 4.0          # t operand in the ladder basis
        rb = 8.0 if kernel == "k_pp64" else 4.0          # result
        byts = float((nlad ** 2).sum()) * vb + float((rows * nlad).sum()) * (tb + rb)
        flops = 2.0 * float((rows * nlad ** 2).sum()) * (1 if kernel == "k_pp64" else 3)
        return byts, flops
    if kernel in ("k_ph64", "k_ph32", "k_ph_f2"):
        # S_z > 0: T (index map + gathered t, or the scattered FP32 copy), W and V1 read, Q
        # written; S_z = 0: the spin-up half of the rows of T, W and V1 read and of Q written;
        # 2 products of (rows x cols x cols) per block, the S_z = 0 blocks at half size, two of
        # them; S_z < 0 channels are not formed
        e = 4.0 if kernel == "k_ph32" else 8.0
        tin = 4 if kernel == "k_ph32" else (4 + 8)
        full, half = xsz > 0, xsz == 0
        el, vv = nph * nhp, nhp * nhp
        byts = (float(el[full].sum()) * (tin + e + e) + float(vv[full].sum()) * e
                + float(el[half].sum()) * (tin + e + e) / 2 + float(vv[half].sum()) * e / 2)
        flops = (4.0 * float((nph * nhp * nhp)[full].sum())
                 + 2 * 4.0 * float(((nph / 2) * (nhp / 2) ** 2)[half].sum()))
        return byts, flops
    if kernel in ("k_update", "k_update_mix"):
        # elementwise step over every restricted amplitude: t read (8 B), t written (8 B) and
        # one 4-byte index per amplitude, the figure the algorithm itself needs
        return nt * (8 + 8 + 4), nt * 20.0
    if kernel in ("k_tstats", "k_tstats32"):
        return nt * 8 * 2 + float((nhh * nhh).sum()) * 16, nt * 2.0 * (2 + nhh.mean())
    return nt * 8.0, 0.0


def kernel_source(kernel):
    """Source file (in the package's csrc/) that defines a kernel."""
    if kernel in ("k_pp_tc", "k_pack"):
        return "mixed.cu"
    return "iterate.cu"


def measured_traffic(kernel, workload):
    """DRAM bytes per launch from the ncu capture recorded in TRAFFIC, if it was taken on this
    workload and the kernel's source is unchanged since; else None."""
    import hashlib
    ent = TRAFFIC.get(kernel)
    if ent is None or workload != DEFAULT_WORKLOAD:
        return None
    path = os.path.join(ROOT, "paper_1611_06765_gb300", "csrc", kernel_source(kernel))
    try:
        with open(path, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return ent[0] if digest == ent[1] else None


MIXED_KERNELS = ("k_update_mix", "k_ph32", "k_pp_tc", "k_tstats32", "k_pack", "k_dchi32")


def work_fraction(ctx, kernel, iters, launches, mixed, refine_sweeps):
    """Average fraction of the full batch that one launch of a kernel processes in a solve:
    converged systems are skipped (the contractions from the update after the one that met the
    tolerance, the update itself one update later, when both amplitude buffers hold the
    values).  iters: updates per system (refinement sweeps included); launches: launches of the
    kernel in the solve."""
    import numpy as np
    n = np.array([float((ctx.channels(s, 0)[1][:, 0] * ctx.channels(s, 0)[1][:, 1]).sum())
                  for s in range(ctx.nsys)])
    if (mixed and kernel not in MIXED_KERNELS) or kernel in ("k_dchi32", "k_dchi"):
        return 1.0  # refinement sweeps (every system reopened); k_dchi never skips
    m = np.array(iters, float) - (refine_sweeps if mixed else 0)
    extra = 1 if kernel in ("k_update_mix", "k_update") else 0
    act = np.minimum(m + extra, launches)
    return float((n * act).sum() / (n.sum() * launches))


def implementation_bytes(ctx, kernel):
    """Bytes per launch the current implementation of an update kernel moves by its own
    accounting (every array it touches, once), beside the algorithmic figure."""
    nhh, npp, nlad, nph, nhp, xsz, nself = chan_sizes(ctx)
    ncomp = 0.5 * float((nhh * npp).sum())
    if kernel == "k_update":
        # per computed amplitude: t, v, eps, 1/eps, qmap, flip map, ladder map, rpp, four Q
        # values read; t_next written for it and its flip
        return ncomp * (8 + 8 + 8 + 8 + 16 + 4 + 4 + 8 + 4 * 8 + 2 * 8)
    if kernel == "k_update_mix":
        # per computed amplitude: t, alpha/eps, qmap, flip map, t32, ladder map, pp ladder, hh
        # ladder (v is formed from the interaction table), four Q values read; t written for
        # it, t32 for it and its flip, four T entries
        return ncomp * (8 + 8 + 16 + 4 + 4 + 4 + 4 + 4 + 4 * 4 + 8 + 2 * 4 + 4 * 4)
    return None


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"




def oracle_solve(N, rho, n2max):
    """One full FP64 oracle solve (setup + MBPT2 start + iterations); (ms, dE, iterations)."""
    from oracle import channel
    t0 = time.perf_counter()
    o = channel.OracleSystem(N, rho, n2max, MINNESOTA)
    dE, it, _, _ = o.ccd(alpha=ALPHA, tol=TOL_PER_N * N, maxit=500)
    ms = (time.perf_counter() - t0) * 1e3
    del o
    return ms, dE, it


# ------------------------------------------------------------------------------ arms

def run_reference(a):
    """The FP64 oracle on the host cores, same workload and metric.  One step is one full
    solve (setup, MBPT2 start, iterations to the same stopping rule) of every system of the
    workload, one after the other, so each step covers the whole batch (about 5 s on 16 Arm
    cores for the held-out batch)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    N, rhos, n2max = WORKLOADS[a.workload][:3]
    from oracle import build as ob
    ob.build()
    from oracle import channel
    for _ in range(a.warmup):
        for rho in rhos:
            oracle_solve(N, rho, n2max)
    times, dEs = [], {}
    for k in range(a.steps):
        step = 0.0
        for rho in rhos:
            ms, dE, it = oracle_solve(N, rho, n2max)
            step += ms
            dEs[str(rho)] = dE / N
        times.append(step)
    ms = statistics.mean(times)
    cores = channel.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": a.workload, "N": N, "rho": list(rhos), "n2max": n2max, "start": "mbpt2",
                   "tol_dE_per_N": TOL_PER_N, "mix_alpha": ALPHA, "l2": "host"},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": "each step: one full FP64 oracle solve (MBPT2 start) of each of the %d "
                                   "systems of the workload, summed" % len(rhos)},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "result": {"dE_per_N": dEs},
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
        iters.append([int(x) for x in it])
        dEs.append([float(x) for x in dE])
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in evs], iters, dEs


def solve_kwargs(P, workload, refine):
    _, _, _, start, prec, rk = WORKLOADS[workload]
    p = P.PNM_PREC_BF16X3 if prec == "bf16x3" else P.PNM_PREC_FP64
    return dict(precision=p, alpha=ALPHA, tol=1e-30, tol_per_N=TOL_PER_N, max_iter=500,
                refine_sweeps=refine if p == P.PNM_PREC_BF16X3 else 0,
                init=P.PNM_INIT_MLP if start == "mlp" else P.PNM_INIT_MBPT2,
                refine_kernels=P.PNM_PREC_F32PAIR if rk == "f32pair" else P.PNM_PREC_FP64)


_model = {}


def trained_model(P, stream):
    """Warm-start network trained by the library's GPU kernels on converged amplitudes of
    N = 14 (n^2 <= 20, 16 densities 0.02 ... 0.32) and N = 66 (n^2 <= 36, rho = 0.04, 0.06,
    ..., 0.20; the held-out 0.05, 0.11, 0.17 are not in the training set): 40 epochs, batch
    1024, Adam with the learning rate decaying from 1e-3 to 1e-5 along a half cosine, seeds 1
    (initial weights) and 3 (shuffling), the matrix products on the tensor cores; or the one
    given with --model."""
    if "blob" not in _model and _model.get("path"):
        import numpy as np
        _model["blob"] = np.load(_model["path"]).astype(np.float32)
    if "blob" not in _model:
        kw64 = dict(precision=P.PNM_PREC_FP64, alpha=ALPHA, tol=1e-30, tol_per_N=1e-8, max_iter=500)
        t0 = time.perf_counter()
        tr14 = P.Context(14, list(SWEEP16), 20, params=MINNESOTA, stream=stream.cuda_stream)
        tr14.solve(**kw64)
        tr66 = P.Context(66, list(TRAIN66), 36, params=MINNESOTA, stream=stream.cuda_stream)
        tr66.solve(**kw64)
        blob, hist = P.mlp_train([tr14, tr66], P.mlp_init(seed=1), epochs=_model.get("epochs", 40),
                                 batch=_model.get("batch", 1024), lr=1e-3, seed=TRAIN_SEED, lr_final=1e-5)
        tr14.close()
        tr66.close()
        _model.update(blob=blob, train_s=time.perf_counter() - t0, loss=[float(hist[0]), float(hist[-1])])
    return _model["blob"]


RANK_RHO_STEP = 0.01


def rank_densities(rhos, rank):
    """The densities one replica solves: rank 0 the workload's own, rank r > 0 each scaled by
    1 + 0.01 r.  The held-out densities differ by factors of 1.5 or more, so the ranks' sets
    are disjoint up to rank 49, and every replica does the work of a batch of the same shape
    (weak scaling: N replicas solve N different batches)."""
    if rank == 0:
        return list(rhos)
    f = 1.0 + RANK_RHO_STEP * rank
    return [round(r * f, 12) for r in rhos]


def make_context(P, workload, stream, rank=0):
    N, rhos, n2max, start = WORKLOADS[workload][:4]
    ctx = P.Context(N, rank_densities(rhos, rank), n2max, params=MINNESOTA, stream=stream.cuda_stream)
    if start == "mlp":
        ctx.mlp_set_model(trained_model(P, stream))
    return ctx


def measure(P, torch, stream, flush, workload, refine, steps):
    """Mean time-to-converge (ms), per-system iterations and dE/N of another workload."""
    N = WORKLOADS[workload][0]
    ctx = make_context(P, workload, stream)
    kw = solve_kwargs(P, workload, refine)
    for _ in range(3):
        ctx.solve(**kw)
    torch.cuda.synchronize()
    ms, iters, dEs = timed_solves(ctx, kw, steps, flush, stream, torch)
    ctx.close()
    return {"ms": statistics.mean(ms), "iters": iters[-1], "dE_per_N": [x / N for x in dEs[-1]]}


def measure_twist(P, torch, stream, flush, workload, refine, steps):
    """Mean time-to-converge (ms) of a twist-averaged batch, with its twist-averaged energies."""
    import numpy as np
    N, rho, n2max, mesh, prec = TWIST_WORKLOADS[workload]
    theta, w = P.twist_mesh(*mesh)
    ctx = P.Context(N, rho, n2max, params=MINNESOTA, stream=stream.cuda_stream, theta=theta)
    p = P.PNM_PREC_BF16X3 if prec == "bf16x3" else P.PNM_PREC_FP64
    kw = dict(precision=p, alpha=ALPHA, tol=1e-30, tol_per_N=TOL_PER_N, max_iter=500,
              refine_sweeps=refine if prec == "bf16x3" else 0, refine_kernels=P.PNM_PREC_F32PAIR)
    for _ in range(3):
        ctx.solve(**kw)
    torch.cuda.synchronize()
    ms, iters, dEs = timed_solves(ctx, kw, steps, flush, stream, torch)
    eref = ctx.eref()
    ctx.close()
    dE = np.array(dEs[-1])
    return {"ms": statistics.mean(ms), "systems": len(w), "mesh": list(mesh), "N": N, "rho": rho,
            "n2max": n2max, "iters_min": min(iters[-1]), "iters_max": max(iters[-1]),
            "E_per_N_twist_avg": float(np.sum(w * (eref + dE)) / N),
            "Eref_per_N_twist_avg": float(np.sum(w * eref) / N),
            "dE_per_N_twist_avg": float(np.sum(w * dE) / N),
            "_theta": theta, "_w": w, "_dE_per_N": dE / N}


def measure_trunc(P, torch, stream, flush, workload, steps):
    """Mean time-to-converge (ms) of a truncated FP64 iteration at the metric's stopping rule,
    with the oracle's fixed point of the same truncation (|dE change| / N < 1e-10 MeV)."""
    N, rhos, n2max, terms = TRUNC_WORKLOADS[workload]
    code = {"pp": P.PNM_TERMS_PP, "pphh": P.PNM_TERMS_PPHH}[terms]
    ctx = P.Context(N, list(rhos), n2max, params=MINNESOTA, stream=stream.cuda_stream)
    kw = dict(precision=P.PNM_PREC_FP64, alpha=ALPHA, tol=1e-30, tol_per_N=TOL_PER_N, max_iter=500, terms=code)
    for _ in range(3):
        ctx.solve(**kw)
    torch.cuda.synchronize()
    ms, iters, dEs = timed_solves(ctx, kw, steps, flush, stream, torch)
    ctx.close()
    return {"ms": statistics.mean(ms), "iters": iters[-1], "terms": terms,
            "dE_per_N": [x / N for x in dEs[-1]], "_key": (N, rhos, n2max, terms)}


def measure_nuclear(P, torch, stream, flush, workload, refine, steps):
    """Mean time-to-converge (ms) of symmetric nuclear matter at the metric's stopping rule."""
    N, Z, rho, n2max, prec = NUCLEAR_WORKLOADS[workload]
    ctx = P.Context(N, rho, n2max, params=MINNESOTA, stream=stream.cuda_stream, Z=Z)
    p = P.PNM_PREC_BF16X3 if prec == "bf16x3" else P.PNM_PREC_FP64
    kw = dict(precision=p, alpha=ALPHA, tol=1e-30, tol_per_N=TOL_PER_N, max_iter=2000,
              refine_sweeps=refine if prec == "bf16x3" else 0, refine_kernels=P.PNM_PREC_F32PAIR)
    for _ in range(3):
        ctx.solve(**kw)
    torch.cuda.synchronize()
    ms, iters, dEs = timed_solves(ctx, kw, steps, flush, stream, torch)
    eref = float(ctx.eref()[0])
    ctx.close()
    A = N + Z
    return {"ms": statistics.mean(ms), "N": N, "Z": Z, "rho": rho, "n2max": n2max, "iters": iters[-1],
            "E_per_A": (eref + dEs[-1][0]) / A, "dE_per_A": dEs[-1][0] / A}


_nuc_oracle = {}


def oracle_nuclear(r):
    """The oracle's energy at the same stopping rule and at its fixed point (1e-10 MeV per
    nucleon): the GPU's error against both."""
    from oracle import channel
    key = (r["N"], r["Z"], r["rho"], r["n2max"])
    if key not in _nuc_oracle:
        A = r["N"] + r["Z"]
        o = channel.OracleSystem(r["N"], r["rho"], r["n2max"], MINNESOTA, Z=r["Z"])
        t0 = time.perf_counter()
        at_rule = o.ccd(alpha=ALPHA, tol=TOL_PER_N * A, maxit=4000)
        ms = (time.perf_counter() - t0) * 1e3
        fixed = o.ccd(alpha=ALPHA, tol=1e-10 * A, maxit=4000)
        _nuc_oracle[key] = (at_rule[0] / A, at_rule[1], fixed[0] / A, ms)
    rule, it, fixed, ms = _nuc_oracle[key]
    r["oracle_iters_at_rule"] = it
    r["oracle_ms"] = ms
    r["dE_per_A_minus_oracle_at_rule"] = r["dE_per_A"] - rule
    r["dE_per_A_minus_oracle_fixed_point"] = r["dE_per_A"] - fixed


def oracle_trunc(r, budget_s=60.0):
    from oracle import channel
    N, rhos, n2max, terms = r.pop("_key")
    err = {}
    t0 = time.perf_counter()
    for rho, d in zip(rhos, r["dE_per_N"]):
        if time.perf_counter() - t0 > budget_s:
            break
        o = channel.OracleSystem(N, rho, n2max, MINNESOTA)
        e, _, _, _ = o.ccd(alpha=ALPHA, tol=1e-10 * N, maxit=2000, terms=terms)
        err[str(rho)] = d - e / N
    r["dE_per_N_minus_oracle"] = err


def measure_mbpt3(P, torch, stream, steps):
    """Device time (ms) of pnm_mbpt3 on the held-out batch and its three diagrams per system."""
    name, N, rhos, n2max = MBPT3_WORKLOAD
    ctx = P.Context(N, list(rhos), n2max, params=MINNESOTA, stream=stream.cuda_stream)
    for _ in range(3):
        e3 = ctx.mbpt3()
    ms = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e3 = ctx.mbpt3()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.close()
    return {"ms": statistics.mean(ms), "N": N, "rho": list(rhos), "n2max": n2max,
            "diagrams_per_N": {str(r): {"pp_ladder_4": e[0] / N, "hh_ladder_5": e[1] / N, "ph_ring_3": e[2] / N}
                               for r, e in zip(rhos, e3.tolist())}}


def oracle_mbpt3(r, budget_s=60.0):
    """The oracle's diagrams for each system (timed) and the GPU's relative error."""
    from oracle import channel
    errs, tms = [], []
    t0 = time.perf_counter()
    for rho in r["rho"]:
        if time.perf_counter() - t0 > budget_s:
            break
        o = channel.OracleSystem(r["N"], rho, r["n2max"], MINNESOTA)
        o.mbpt3()  # the first call builds the interaction blocks; the timed one reuses them
        t1 = time.perf_counter()
        ref = o.mbpt3()
        tms.append((time.perf_counter() - t1) * 1e3)
        got = r["diagrams_per_N"][str(rho)]
        g = [got["pp_ladder_4"], got["hh_ladder_5"], got["ph_ring_3"]]
        errs.append(max(abs(a * r["N"] - b) / abs(b) for a, b in zip(g, ref)))
    r["max_rel_err_vs_oracle"] = max(errs) if errs else None
    r["oracle_ms_per_system"] = statistics.mean(tms) if tms else None


_twist_fixed = {}


def oracle_twist(P, r, budget_s=60.0):
    """The oracle's fixed points (|dE change| / N < 1e-10 MeV) at every twist of a measured
    twist batch, within a time budget; fills the error fields of r."""
    import numpy as np
    from oracle import channel
    theta, w, dE = r.pop("_theta"), r.pop("_w"), r.pop("_dE_per_N")
    err = []
    t0 = time.perf_counter()
    for th, d in zip(theta, dE):
        key = (r["N"], r["rho"], r["n2max"], tuple(th))
        if key not in _twist_fixed:
            if time.perf_counter() - t0 > budget_s:
                break
            o = channel.OracleSystem(r["N"], r["rho"], r["n2max"], MINNESOTA, theta=th)
            _twist_fixed[key] = o.ccd(alpha=ALPHA, tol=1e-10 * r["N"], maxit=1000)[0] / r["N"]
        err.append(d - _twist_fixed[key])
    r["oracle_systems"] = len(err)
    if err:
        r["max_abs_dE_per_N_minus_oracle"] = float(np.max(np.abs(err)))
        if len(err) == len(w):
            r["twist_avg_dE_per_N_minus_oracle"] = float(np.sum(w * np.array(err)))


def oracle_leg(workloads, budget_s=60.0):
    """cpu_baseline leg: FP64 oracle solves of the systems of the given workloads (each
    distinct (N, rho, n2max) once, within a time budget, in the order given): one at the
    metric's stopping rule (timed) and one converged to |dE change| / N < 1e-10 MeV (the fixed
    point the GPU results are compared with).  Returns {(N, rho, n2max): (ms, dE/N at the
    metric's rule, iterations, dE/N at the fixed point)}."""
    from oracle import build as ob
    ob.build()
    from oracle import channel
    seen = []
    for w in workloads:
        N, rhos, n2max = WORKLOADS[w][:3]
        for r in rhos:
            if (N, r, n2max) not in seen:
                seen.append((N, r, n2max))
    out = {}
    t0 = time.perf_counter()
    for key in seen:
        if out and time.perf_counter() - t0 > budget_s:
            break
        ms, dE, it = oracle_solve(*key)
        o = channel.OracleSystem(key[0], key[1], key[2], MINNESOTA)
        dE_fix, _, _, _ = o.ccd(alpha=ALPHA, tol=1e-10 * key[0], maxit=1000)
        out[key] = (ms, dE / key[0], it, dE_fix / key[0])
    return out


def oracle_one_thread():
    """The oracle on one host thread, full solve of N = 14, rho = 0.08, n^2 <= 20 (ms), beside
    the all-core figure of the same solve."""
    from oracle import channel
    n = channel.threads()
    ms_all, _, _ = oracle_solve(14, 0.08, 20)
    channel.set_threads(1)
    try:
        ms_one, _, it = oracle_solve(14, 0.08, 20)
    finally:
        channel.set_threads(n)
    return {"workload": "pnm_N14_rho0.08_n2max20", "ms_1_thread": ms_one, "ms_all_threads": ms_all,
            "threads": n, "iterations": it}


def oracle_errors(res, workload, ora):
    N, rhos, n2max = WORKLOADS[workload][:3]
    err = {}
    for r, e in zip(rhos, res["dE_per_N"]):
        if (N, r, n2max) in ora:
            err[str(r)] = e - ora[(N, r, n2max)][3]
    return err


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
    N, rhos, n2max, start, prec_name, refine_kind = WORKLOADS[a.workload]
    _model["path"] = a.model
    _model["epochs"], _model["batch"] = a.train_epochs, a.train_batch
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ctx = make_context(P, a.workload, stream, rank)
    solve_kw = solve_kwargs(P, a.workload, a.refine)
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
    if a.save_model and rank == 0 and "blob" in _model:
        import numpy as np
        np.save(a.save_model, _model["blob"])

    # e2e through the public API from host inputs (the trained model is an input, like V's parameters)
    # one untimed end-to-end pass first (the memory pool grows to hold a second context beside
    # the timed one), then the timed passes
    e2e_ms = []
    n_t = 0
    for k in range(1 + max(1, min(a.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = make_context(P, a.workload, stream, rank)
        c2.solve(**solve_kw)
        n_t = sum(c2.get_amplitudes(s).size for s in range(c2.nsys))
        c2.close()
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_mean = statistics.mean(e2e_ms)
    if dist:
        e2e_mean = max_over_ranks(e2e_mean, dist, device="cuda")

    # per-kernel durations from one profiled host-driven solve of the same work (the same
    # kernels, launched one update at a time instead of from the graph's device-side loop); it
    # sits in the NVTX range "host_driven_solve", so that a profiler can select its launches
    # (ncu --nvtx --nvtx-include host_driven_solve/; ncu does not profile the kernel nodes of a
    # graph with a conditional node)
    ctx.set_profiling(True)
    torch.cuda.nvtx.range_push("host_driven_solve")
    _, it_h, _, _ = ctx.solve(host_loop=True, **solve_kw)
    torch.cuda.nvtx.range_pop()
    stats = ctx.kernel_stats()
    ctx.set_profiling(False)
    kname, (ktot, kn) = max(stats.items(), key=lambda kv: kv[1][0])
    kavg_s = ktot / kn / 1e3
    # algorithmic cost of a launch over the full batch, scaled by the fraction of the batch the
    # solve's launches process on average (converged systems are skipped)
    byts_full, flops_full = algorithmic_cost(ctx, kname)
    wfrac = work_fraction(ctx, kname, [int(x) for x in it_h], kn, prec_name != "fp64", solve_kw.get("refine_sweeps", 0))
    byts, flops = byts_full * wfrac, flops_full * wfrac
    hbm, bf16, src = read_peaks()
    fp64_peak = P.measure_fma_peak(True, stream.cuda_stream)
    fp32_peak = P.measure_fma_peak(False, stream.cuda_stream)
    if kname in ("k_pp64", "k_ph64"):
        roof = {"bound": "alu", "achieved": flops / kavg_s / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "peak_source": "measured FP64 FMA rate (pnm_measure_fma_peak)"}
    elif kname in ("k_pp_f2", "k_ph_f2"):
        # FP64-equivalent flops against the FP32 pipe's rate per FP32-pair multiply-add (12 FP32
        # instructions, i.e. the measured FP32 FMA rate / 12)
        roof = {"bound": "alu", "achieved": flops / kavg_s / 1e12, "peak": fp32_peak / 12,
                "unit": "TFLOP/s", "peak_source": "measured FP32 FMA rate / 12 (FP32-pair multiply-add)"}
    else:
        roof = {"bound": "hbm", "achieved": byts / kavg_s / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": "%s hbm_gbs" % src}
    traffic = measured_traffic(kname, a.workload)
    roof.update(frac=roof["achieved"] / roof["peak"], traffic=traffic, kernel=kname, kernel_avg_us=kavg_s * 1e6,
                algorithmic_bytes=byts, algorithmic_flops=flops,
                algorithmic_bytes_full_batch=byts_full, launch_work_fraction=wfrac, launches=kn,
                traffic_basis="ncu DRAM read + write of one launch over the full batch (all systems active)",
                measured_fma_peaks_tflops={"fp64": fp64_peak, "fp32": fp32_peak})
    ib = implementation_bytes(ctx, kname)
    if ib is not None:
        roof["implementation_bytes"] = ib * wfrac
        roof["implementation_gbs"] = ib * wfrac / kavg_s / 1e9
    # the FP64 refinement contractions against the measured FP64 FMA rate
    for k in ("k_pp64", "k_ph64", "k_ph32", "k_pp_f2", "k_ph_f2"):
        if k in stats and k != kname:
            tk = stats[k][0] / stats[k][1] / 1e3
            bk, fk = algorithmic_cost(ctx, k)
            fk *= work_fraction(ctx, k, [int(x) for x in it_h], stats[k][1], prec_name != "fp64",
                                solve_kw.get("refine_sweeps", 0))
            pk = {"k_ph32": fp32_peak, "k_pp_f2": fp32_peak / 12, "k_ph_f2": fp32_peak / 12}.get(k, fp64_peak)
            roof[k] = {"bound": "alu", "achieved": fk / tk / 1e12, "peak": pk, "unit": "TFLOP/s",
                       "frac": fk / tk / 1e12 / pk, "kernel_avg_us": tk * 1e6}
    if "k_pp_tc" in stats and kname != "k_pp_tc":
        t_tc = stats["k_pp_tc"][0] / stats["k_pp_tc"][1] / 1e3
        b_tc, f_tc = algorithmic_cost(ctx, "k_pp_tc")
        w_tc = work_fraction(ctx, "k_pp_tc", [int(x) for x in it_h], stats["k_pp_tc"][1], prec_name != "fp64",
                             solve_kw.get("refine_sweeps", 0))
        b_tc, f_tc = b_tc * w_tc, f_tc * w_tc
        roof["k_pp_tc"] = {"bound": "hbm", "achieved": b_tc / t_tc / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": b_tc / t_tc / 1e9 / hbm, "kernel_avg_us": t_tc * 1e6,
                           "traffic": measured_traffic("k_pp_tc", a.workload),
                           "tensor_tflops": f_tc / t_tc / 1e12, "tensor_frac_of_bf16_peak": f_tc / t_tc / 1e12 / bf16}
    # kernels of one solve: the loop bodies and refinement sweeps counted by the profiler, plus
    # the start (MBPT2: init + energy; learned: inference, copy to the spin flips, symmetrise,
    # init + energy, FP32 copies)
    launches_per_solve = sum(n for _, n in stats.values()) + (6 if start == "mlp" else 2)

    comparison = None
    if rank == 0 and not a.no_extra:
        comparison = {}
        for w in COMPARE:
            if w != a.workload:
                comparison[w] = measure(P, torch, stream, flush, w, a.refine, 5)
        for w in TWIST_WORKLOADS:
            comparison[w] = measure_twist(P, torch, stream, flush, w, a.refine, 5)
        for w in TRUNC_WORKLOADS:
            comparison[w] = measure_trunc(P, torch, stream, flush, w, 5)
        comparison[MBPT3_WORKLOAD[0]] = measure_mbpt3(P, torch, stream, 5)
        for w in NUCLEAR_WORKLOADS:
            comparison[w] = measure_nuclear(P, torch, stream, flush, w, a.refine, 5)
        if "train_s" in _model:
            comparison["training"] = {"seconds": _model["train_s"], "loss_first_last": _model["loss"],
                                      "epochs": _model["epochs"], "batch": _model["batch"],
                                      "data": "FP64-converged amplitudes, N=14 n2max=20 16 densities "
                                              "and N=66 n2max=36 rho=" + "/".join("%g" % r for r in TRAIN66),
                                      "schedule": "Adam, lr 1e-3 -> 1e-5 half cosine, seeds 1 and %d" % TRAIN_SEED}

    result = {"dE_per_N": [x / N for x in dEs[-1]], "iters": iters[-1], "step_ms_min": min(step_ms),
              "step_ms_max": max(step_ms), "step_ms": [round(x, 4) for x in step_ms],
              "step_ms_median": statistics.median(step_ms), "wall_ms_per_step": wall * 1e3 / a.steps,
              "setup_ms": tim["setup"], "mixed_phase_ms": tim["mixed"], "refine_ms": tim["refine"],
              "kernels_ms_per_solve": {k: v[0] for k, v in stats.items()}}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        from oracle import channel
        ora = oracle_leg([a.workload] + (COMPARE if comparison is not None else []))
        own = [ora[(N, r, n2max)] for r in rhos if (N, r, n2max) in ora]
        cpu = {"value": sum(x[0] for x in own) * len(rhos) / len(own), "unit": "ms",
               "cores": channel.threads(), "kind": "oracle",
               "sample": "%d of %d systems of the workload, one full FP64 oracle solve each (setup, MBPT2 "
                         "start, iterations to the same stopping rule), summed and scaled to all systems"
                         % (len(own), len(rhos)),
               "oracle_dE_per_N": {str(k[1]): v[1] for k, v in ora.items() if k[0] == N and k[2] == n2max
                                   and k[1] in rhos},
               "oracle_fixed_point_dE_per_N": {str(k[1]): v[3] for k, v in ora.items()
                                               if k[0] == N and k[2] == n2max and k[1] in rhos},
               "errors": "dE_per_N_minus_oracle fields: GPU dE/N minus the oracle's fixed point "
                         "(converged to 1e-10 MeV per neutron)",
               "oracle_iters": {str(k[1]): v[2] for k, v in ora.items() if k[0] == N and k[2] == n2max
                                and k[1] in rhos},
               "one_thread": oracle_one_thread()}
        result["dE_per_N_minus_oracle"] = oracle_errors(result, a.workload, ora)
        if comparison:
            for w, r in comparison.items():
                if w in WORKLOADS:
                    r["dE_per_N_minus_oracle"] = oracle_errors(r, w, ora)
                elif w in TWIST_WORKLOADS:
                    oracle_twist(P, r)
                elif w in TRUNC_WORKLOADS:
                    oracle_trunc(r)
                elif w == MBPT3_WORKLOAD[0]:
                    oracle_mbpt3(r)
                elif w in NUCLEAR_WORKLOADS:
                    oracle_nuclear(r)

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": a.steps,
            "warmup": max(3, a.warmup), "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec_name == "fp64" else "bf16x3+f32+f64",
            "data": "synthetic",
            "config": {"workload": a.workload, "N": N, "rho": list(rhos), "n2max": n2max, "start": start,
                       "precision": prec_name, "refine_sweeps": solve_kw["refine_sweeps"],
                       "refine_contractions": refine_kind, "mix_alpha": ALPHA,
                       "tol_dE_per_N": TOL_PER_N, "l2": "flushed (512 MB write) before every step",
                       "parallelism": "replicas" if world > 1 else "single",
                       "rank_rho": ("rank r solves rho x (1 + %g r)" % RANK_RHO_STEP) if world > 1 else None},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_mean, "unit": "ms",
                    "h2d_bytes_per_step": 8 * len(rhos) + 7 * 8 + 8 + (4 * len(_model.get("blob", ()))),
                    "d2h_bytes_per_step": 8 * n_t + len(rhos) * 20},
            "gpu_launches": int(launches_per_solve * a.steps),
            "roofline": roof,
            "cpu_baseline": cpu,
            "tuning": (dict(zip(("k_splits", "stages", "pp_tc_us", "serial_mask"), ctx.tuning()))
                       if prec_name == "bf16x3" else None),
            "comparison": ({k: {f: v for f, v in r.items() if not f.startswith("_")}
                            for k, r in comparison.items()} if comparison else comparison),
            "result": result,
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
