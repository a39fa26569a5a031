#!/usr/bin/env python3
"""Benchmark of the S-ADI per-time-step hot path on GB300.

Workload (one bench "step" = one S-ADI time step of every instance):
  N = 1023 interior points per direction on Omega = (-1, 1)^2, kappa = 1,
  tau = 1e-3, g(u) = -sin u, three instances alpha in {1.2, 1.5, 1.8},
  phi1 = 8 seeded Gaussian bumps (centres U(-0.6, 0.6)^2, widths U(0.05, 0.2),
  amplitudes U(-1, 1)), phi2 = 0.  Synthetic, seeded.
Metric: grid-point updates per second, N^2 * steps * instances / time, for the
chosen form, with the plain FP64 GS-FFT path on the same GPU and each form's
relative L2 difference to it stated.  Candidate forms: FP32 FFTs with
Gohberg-Semencul FFT sweeps, and FP32 FFTs with both sweeps as
split-BF16 dense-inverse GEMMs on the tensor cores; the chosen form is the
fastest one within 1e-5 relative L2 of the FP64 path after the accuracy run
(--acc-steps, default 1000 steps from the same data).

Timing: W untimed warm-up steps, then K timed steps; each step is bracketed
by CUDA events on the launching stream (the FP32 forms replay a captured
CUDA graph of one batched step) and an L2 flush (a 256 MiB write) runs
between timed steps, outside the events (the working set, ~30 MB per
instance, is smaller than L2).  Multi-GPU: every rank advances its own copy
of the three instances (independent problems, no collective); value = all
ranks' updates / the slowest rank's time.

--impl reference times the FP64 CPU oracle (the reference arm for this
paper-only workload) on the host cores: each step is one S-ADI step of one
instance (cycling through the three alpha), rank 0 only.
"""
from __future__ import annotations

import argparse
import contextlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Workload presets (Omega = (-1, 1)^2, seeded Gaussian-bump phi1).  "n1023" is
# the default bench workload; the others are single large instances run on
# request (--workload).
PRESETS = {
    "n1023": dict(N=1023, alphas=(1.2, 1.5, 1.8), kappa=1.0, tau=1e-3, g=2, bumps=8, phi2=0.0, seed=2,
                  total_steps=1000),
    "n4095": dict(N=4095, alphas=(1.7,), kappa=0.5, tau=5e-4, g=1, bumps=8, phi2=0.0, seed=3, total_steps=2000),
    "n8191": dict(N=8191, alphas=(1.6,), kappa=1.0, tau=2.5e-4, g=2, bumps=32, phi2=0.1, seed=5,
                  total_steps=500),
    # 256 independent instances of uneven size: N from {127, 255, 511, 1023, 2047},
    # alpha ~ U(1.1, 1.9), kappa ~ U(0.5, 2), tau = h/2 = 1/(N+1), g = -u^3, 8 bumps
    "batch256": dict(N=None, count=256, sizes=(127, 255, 511, 1023, 2047), alphas=(1.1, 1.9), kappa=(0.5, 2.0),
                     g=1, bumps=8, phi2=0.0, seed=4, total_steps=500),
}
CFG = PRESETS["n1023"]
N_DEFAULT = CFG["N"]
ALPHAS = CFG["alphas"]
KAPPA, TAU = CFG["kappa"], CFG["tau"]
GKIND = CFG["g"]
GNAME = {0: "0", 1: "-u^3", 2: "-sin(u)"}
METRIC = "grid-point updates/s (N^2*steps/s)"
UNIT = "pt/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n1023", choices=sorted(PRESETS))
    ap.add_argument("--N", type=int, default=None, help="override the preset's N")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--acc-steps", type=int, default=1000,
                    help="steps of the accuracy check (FP32 form vs plain FP64 from the same data)")
    return ap.parse_args()


def _nvtx(name):
    """An NVTX range around the timed steps, so that a profiler can be told
    to capture those launches alone (e.g. ncu --nvtx --nvtx-include
    "timed_steps/"); a no-op where torch has no NVTX."""
    try:
        import torch
        return torch.cuda.nvtx.range(name)
    except Exception:
        return contextlib.nullcontext()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _select(a):
    """Apply the chosen preset to the module-level workload constants."""
    global CFG, ALPHAS, KAPPA, TAU, GKIND
    CFG = dict(PRESETS[a.workload])
    if a.N is not None:
        CFG["N"] = a.N
    a.N = CFG["N"]
    ALPHAS, KAPPA, TAU, GKIND = CFG["alphas"], CFG["kappa"], CFG.get("tau"), CFG["g"]


def batch_instances(cfg):
    """The batch workload's instances: (N, alpha, kappa, tau, seed) per
    instance k, parameters drawn in order from default_rng(SEED_BASE + seed),
    the bumps of instance k from seed SEED_BASE + seed + k."""
    import numpy as np
    from paper_2312_06206_gb300 import workloads as WL
    rng = np.random.default_rng(WL.SEED_BASE + cfg["seed"])
    out = []
    for k in range(cfg["count"]):
        N = int(rng.choice(cfg["sizes"]))
        al = float(rng.uniform(*cfg["alphas"]))
        ka = float(rng.uniform(*cfg["kappa"]))
        out.append((N, al, ka, 1.0 / (N + 1), WL.SEED_BASE + cfg["seed"] + k))
    return out


def lpt_partition(costs, world):
    """Longest-processing-time-first assignment of items to world bins:
    items in decreasing cost, each to the least loaded bin (ties: lowest
    rank).  Returns the item indices of every bin."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    bins = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda b: (load[b], b))
        bins[r].append(i)
        load[r] += costs[i]
    return [sorted(b) for b in bins]


def _workload(N):
    from paper_2312_06206_gb300 import workloads as WL
    return WL.gaussian_bumps(N, CFG["bumps"], WL.SEED_BASE + CFG["seed"])


def _phi2(phi1):
    return None if CFG["phi2"] == 0.0 else CFG["phi2"] * phi1


def _config(N, extra=None):
    al = ",".join(str(x) for x in ALPHAS)
    cfg = {"workload": f"sadi-step N={N} alpha={{{al}}} kappa={KAPPA:g} tau={TAU:g} g={GNAME[GKIND]} "
                       f"phi1={CFG['bumps']} gaussian bumps phi2={CFG['phi2']:g}*phi1",
           "N": N, "instances": len(ALPHAS), "alphas": list(ALPHAS), "kappa": KAPPA, "tau": TAU,
           "g": GNAME[GKIND], "domain": [-1.0, 1.0]}
    if extra:
        cfg.update(extra)
    return cfg


# --------------------------------------------------------------- clocks ------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out.update({"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                    "reasons": sorted(reasons), "samples": len(rows)})
        return out


# --------------------------------------------------------- cpu baseline ------

def cpu_baseline(N, phi1, nsteps=3, alpha=1.5):
    """The FP64 oracle (FFT tier) as it stands, on the host cores: nsteps
    S-ADI steps (n >= 1 formula) of one instance; the problem set-up and the
    n = 0 start step are not timed."""
    from oracle import sadi as O
    P = O.Problem(N, alpha, KAPPA, TAU, -1.0, 1.0, GKIND)
    import numpy as np
    u0 = np.array(phi1)
    p2 = _phi2(phi1)
    u1 = O.step(P, None, u0, True, np.zeros_like(u0) if p2 is None else p2, tier="fft")
    t0 = time.perf_counter()
    up, uc = u0, u1
    for _ in range(nsteps):
        up, uc = uc, O.step(P, up, uc, False, tier="fft")
    dt = time.perf_counter() - t0
    return {"value": N * N * nsteps / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{nsteps} S-ADI steps (n>=1) of one instance (alpha={alpha}) of the N={N} workload; "
                      "oracle FFT tier (numpy FFT convolution + LAPACK Cholesky sweeps, FP64), "
                      "default BLAS threading", "seconds": dt}, (u0, u1, uc)


# --------------------------------------------------------- reference arm -----

def run_reference_batch(a):
    """Reference arm of the batch workload: the FP64 oracle (FFT tier) on the
    host cores, each step one S-ADI step of one instance, cycling through the
    first eight instances of the batch."""
    import numpy as np
    from oracle import sadi as O
    from paper_2312_06206_gb300 import workloads as WL
    sample = batch_instances(CFG)[:8]
    probs, states = [], []
    for (N, al, ka, ta, sd) in sample:
        P = O.Problem(N, al, ka, ta, -1.0, 1.0, CFG["g"])
        u0 = WL.gaussian_bumps(N, CFG["bumps"], sd)
        probs.append(P)
        states.append([u0, O.step(P, None, u0, True, np.zeros_like(u0), tier="fft")])

    def one(k):
        i = k % len(probs)
        up, uc = states[i]
        states[i] = [uc, O.step(probs[i], up, uc, False, tier="fft")]
        return probs[i].N ** 2
    for k in range(a.warmup):
        one(k)
    pts = 0
    t0 = time.perf_counter()
    for k in range(a.steps):
        pts += one(a.warmup + k)
    dt = time.perf_counter() - t0
    val = pts / dt
    sizes = [x[0] for x in sample]
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "sadi-batch 256 instances N~U{127,255,511,1023,2047} alpha~U(1.1,1.9) "
                                   "kappa~U(0.5,2) tau=h/2 g=-u^3 phi1=8 gaussian bumps phi2=0",
                       "reference": "FP64 CPU oracle (FFT tier); one step = one S-ADI step of one instance, "
                                    f"cycling the first 8 instances (N = {sizes})"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{a.steps} single-instance S-ADI steps over instances of N = {sizes}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(a):
    _select(a)
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    if a.workload == "batch256":
        return run_reference_batch(a)
    import numpy as np
    from oracle import sadi as O
    N = a.N
    phi1 = _workload(N)
    probs = [O.Problem(N, al, KAPPA, TAU, -1.0, 1.0, GKIND) for al in ALPHAS]
    states = []
    p2 = _phi2(phi1)
    for P in probs:
        u0 = phi1.copy()
        u1 = O.step(P, None, u0, True, np.zeros_like(u0) if p2 is None else p2, tier="fft")
        states.append([u0, u1])

    def one(k):
        i = k % len(probs)
        up, uc = states[i]
        states[i] = [uc, O.step(probs[i], up, uc, False, tier="fft")]
    for k in range(a.warmup):
        one(k)
    t0 = time.perf_counter()
    for k in range(a.steps):
        one(a.warmup + k)
    dt = time.perf_counter() - t0
    val = N * N * a.steps / dt
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": _config(N, {"reference": "FP64 CPU oracle (FFT tier); one step = one S-ADI step of one "
                                               "instance, cycling alpha"}),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{a.steps} single-instance S-ADI steps at N={N}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- our arm -------

def aggregate(times, world_size, pts_per_step, steps_list, reduce_max=None):
    """Whole-job throughput from per-rank times.  times: this rank's
    [ms_fp32, ms_fp64, s_e2e]; reduce_max(list) -> element-wise max over ranks
    (identity on one rank).  Every rank advances its own copy of the workload
    (weak scaling), so value = world_size * points * steps / slowest time."""
    mx = reduce_max(list(times)) if reduce_max else list(times)
    ms32, ms64, e2e = mx
    k32, k64, ke = steps_list
    return {"value": world_size * pts_per_step * k32 / (ms32 / 1e3),
            "value64": world_size * pts_per_step * k64 / (ms64 / 1e3),
            "e2e": world_size * pts_per_step * ke / e2e,
            "ms32": ms32, "ms64": ms64, "e2e_s": e2e}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel in a workload, from the ncu captures summarised under profiles/
# (kr_rows_r2c_n1023.md, kr_cols_conv_n1023.md, kr_rows_solve_dense_n1023.md,
# k_tc_gemm_n1023.md, k_tc_gemm_n4095.md); absent = no capture of the
# current kernel, reported as null.
NCU_TRAFFIC = {("n1023", "kr_rows_r2c"): 12.66e6, ("n1023", "kr_cols_conv"): 50.48e6,
               ("n1023", "kr_rows_solve<dense>"): 70.76e6, ("n1023", "k_tc_gemm(x+y)"): 89.4e6,
               ("n4095", "k_tc_gemm(x+y)"): 1733.6e6}


# Algorithmic work per grid point of one instance and step, per kernel
# (the method's own bytes of the FP32 design: the per-kernel input and output
# each step must move, and the method's FFT flops at the nominal 5 L log2 L of
# a complex FFT of length L).  a1 row FFT: u^n in (4), spectrum row out (8);
# a2 column convolution: spectrum in and out (16), symbol (N'+1)^2 ~ N^2
# floats (4); a3 row inverse FFT + B^n + x sweep: spectrum in (8), u^n in (4),
# W out (4); a4 + a5 y sweep + leapfrog: W, u^n, u^{n-1} in, u^{n+1} out (16).
# The dense form splits a3: its B^n kernel writes B (4) instead of W, and one
# GEMM launch runs the x sweep (B in, W out: 8) and a4 + a5 (16).  The dense
# form's sweeps run no FFT flops; the tensor work they do instead (three
# BF16 products of 2 N^3 per sweep) is reported separately as a dense
# equivalent, not as the method's work.
BYTES_PER_PT = {"rows_r2c": 12, "cols_conv": 20, "rows_solve": 16, "cols_solve": 16,
                "rows_solve<dense>": 16, "tc_gemm": 24}


def algorithmic(N, Np, dense=False):
    """[(bytes, flops)] of the four timed phases for one instance (flops None
    where the kernel runs none of the method's arithmetic)."""
    pts = N * N
    fft = 5.0 * Np * math.log2(Np)           # one complex FFT of length N'
    r2c = (BYTES_PER_PT["rows_r2c"] * pts, N * fft)                  # one transform per row
    conv = (BYTES_PER_PT["cols_conv"] * pts, 4 * Np * fft)          # 2 + 2 per column pair, N' pairs
    if not dense:
        return [r2c, conv,
                (BYTES_PER_PT["rows_solve"] * pts, N * 5 * fft),    # inverse row FFT + Algorithm 1 (4)
                (BYTES_PER_PT["cols_solve"] * pts, N * 4 * fft)]    # Algorithm 1 per column
    return [r2c, conv, (BYTES_PER_PT["rows_solve<dense>"] * pts, N * fft),
            (BYTES_PER_PT["tc_gemm"] * pts, None)]


def launches_per_step(Np, dense):
    """Kernel launches of one batched step (all instances in each): row FFT,
    column convolution (three passes at N' = 8192), row kernel, and either
    one launch of both sweep GEMMs (dense form) or the y sweep (on the
    shared-memory engine: transpose, row solve, transpose with leapfrog)."""
    conv = 3 if Np == 8192 else 1
    if dense:
        return 2 + conv + 1
    return 2 + conv + (3 if Np > 1024 else 1)


def peaks_of():
    """Roofline denominators: the measured copy bandwidth and sustained BF16
    rate (MEASURED_PEAKS.json), and the FP32 FMA peak at the measured maximum
    SM clock (152 SMs x 128 lanes x 2 flops)."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    return {"fp32_tflops": 152 * 128 * 2 * sm_max * 1e6 / 1e12, "sm_max_mhz": sm_max,
            "hbm_gbs": float(peaks.get("hbm_gbs", 6800.0)),
            "bf16_tflops_sustained": float(peaks.get("bf16_tflops_sustained", 1700.0)),
            "source": "measured" if peaks else "fallback"}


def roofline_of(phase_ms, N, Np, dense, ninst, workload):
    """Roofline entry of the dominant kernel from the per-phase times (ms per
    step, one launch per phase covering ninst instances of size N).  Each
    kernel's bound is the roof its algorithmic intensity (method flops per
    method byte) meets first: HBM below the ridge FP32 peak / HBM peak, the
    FP32 pipes above it; a kernel with no method flops is HBM-bound."""
    # the register path: both forms up to N' = 1024, the dense form's FFT part
    # at N' = 2048 too
    reg = Np <= 1024 or (dense and Np == 2048)
    pre = "kr_" if reg else "k_"
    conv = "kr_cols_conv" if reg else ("k_conv3_a+b+c" if Np == 8192 else "k_cols_conv")   # three passes at 8192
    if dense:
        names = [pre + "rows_r2c", conv, pre + "rows_solve<dense>", "k_tc_gemm(x+y)"]
    else:
        ysweep = "kr_cols_solve" if reg else "k_transpose+k_rows_gs+k_transpose_leapfrog"
        names = [pre + "rows_r2c", conv, pre + "rows_solve", ysweep]
    alg = algorithmic(N, Np, dense)
    pk = peaks_of()
    fp32_peak, hbm_peak, bf16_peak = pk["fp32_tflops"], pk["hbm_gbs"], pk["bf16_tflops_sustained"]
    ridge = fp32_peak * 1e12 / (hbm_peak * 1e9)
    per_kernel = {}
    for k, nm in enumerate(names):
        b_alg, f_alg = alg[k]
        dur = phase_ms[k] / 1e3
        inten = None if f_alg is None else f_alg / b_alg
        bound = "hbm" if inten is None or inten < ridge else "alu"
        gbs = b_alg * ninst / dur / 1e9
        tfl = None if f_alg is None else f_alg * ninst / dur / 1e12
        ach, peak, unit = (gbs, hbm_peak, "GB/s") if bound == "hbm" else (tfl, fp32_peak, "TFLOP/s")
        e = {"us": phase_ms[k] * 1e3, "share": phase_ms[k] / sum(phase_ms), "bound": bound,
             "intensity_flop_per_byte": inten, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
             "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak, "fp32_tflops": tfl,
             "alg_bytes": b_alg * ninst, "alg_flops": None if f_alg is None else f_alg * ninst,
             "traffic": NCU_TRAFFIC.get((workload, nm))}
        if nm.startswith("k_tc_gemm"):
            dflops = 12.0 * N ** 3 * ninst
            e["dense_equivalent"] = {"what": "split-BF16 tensor work of the dense-inverse sweeps (3 BF16 "
                                             "products of 2N^3 per sweep), not the method's work",
                                     "tflops": dflops / dur / 1e12, "peak": bf16_peak,
                                     "frac": dflops / dur / 1e12 / bf16_peak}
        per_kernel[nm] = e
    dom = max(range(4), key=lambda k: phase_ms[k])
    dname = names[dom]
    dk = per_kernel[dname]
    src = pk["source"]
    out = {"kernel": dname, "bound": dk["bound"], "achieved": dk["achieved"], "peak": dk["peak"],
           "unit": dk["unit"], "frac": dk["frac"], "traffic": dk["traffic"], "avg_launch_us": dk["us"],
           "units_per_launch": f"{ninst} x {N}^2 grid points",
           "per_unit": (f"{alg[dom][0] // (N * N)} B/pt" +
                        ("" if alg[dom][1] is None else f", {alg[dom][1] / (N * N):.0f} flop/pt")),
           "traffic_note": "ncu dram bytes per launch from profiles/ (null if no capture of this kernel)",
           "peak_note": (f"copy bandwidth, {src} (MEASURED_PEAKS.json)" if dk["bound"] == "hbm" else
                         f"FP32 FMA peak at the {src} max clock: 152 SM x 128 lanes x 2 x "
                         f"{pk['sm_max_mhz']:.0f} MHz"),
           "ridge_flop_per_byte": ridge, "kernels": per_kernel}
    if "dense_equivalent" in dk:
        out["dense_equivalent"] = dk["dense_equivalent"]
    return out


def c1_latency(S, stream, reps=3):
    """The small configuration (N = 63, alpha = 1.5, kappa = 1, tau = 1/64,
    64 steps, g = -u^3, FP64, one instance): microseconds per step, CUDA
    events on the launching stream around the 64 steps after set_initial
    (the n = 0 step, 31 replays of a captured graph of two steps, one more
    step), best of reps runs after one warm-up run.  Latency-bound (four
    launches of up to 64 blocks per step)."""
    import torch
    from paper_2312_06206_gb300 import workloads as WL
    w = WL.small_fp64(63)
    best = float("inf")
    with S.Sadi(w.N, w.alpha, w.kappa, w.tau, (w.a, w.b)) as s:
        s.set_options(w.g, S.SADI_PREC_FP64)
        s.set_stream(stream.cuda_stream)
        s.set_initial(w.phi1, w.phi2)
        s.step(1)
        graph = S.SadiGraph([s], 2)      # captured at n = 1; every run below replays it at n = 1
        for r in range(reps + 1):
            s.set_initial(w.phi1, w.phi2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(1)
            graph.launch((w.steps - 2) // 2)
            s.step(w.steps - 1 - 2 * ((w.steps - 2) // 2))
            e1.record(stream)
            e1.synchronize()
            if r > 0:
                best = min(best, e0.elapsed_time(e1))
        graph.close()
    return {"workload": "sadi N=63 alpha=1.5 kappa=1 tau=1/64 64 steps g=-u^3 phi1=exp(-20r^2) phi2=0, FP64",
            "us_per_step": best * 1e3 / w.steps, "value": w.N * w.N * w.steps / (best / 1e3), "unit": UNIT,
            "timing": f"CUDA events around the {w.steps} steps after set_initial (the n = 0 step, a graph of two "
                      f"steps replayed, the last step), best of {reps}"}


def run_batch(a):
    """The batch workload: every rank builds its LPT share of the 256
    instances, the autotuner picks each size's form, and one CUDA graph
    launch per step advances all of them (total work fixed: strong scaling)."""
    ws, rank, local = _dist()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi as S
    from paper_2312_06206_gb300 import workloads as WL
    inst = batch_instances(CFG)
    costs = [N * N * math.log2(N + 1) for (N, _, _, _, _) in inst]
    mine = lpt_partition(costs, ws)[rank]
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    t0 = time.perf_counter()
    ctxs = []
    for i in mine:
        N, al, ka, ta, _ = inst[i]
        s = S.Sadi(N, al, ka, ta, (-1.0, 1.0))
        s.set_stream(stream.cuda_stream)
        ctxs.append(s)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    S.sadi_autotune(ctxs, CFG["g"])
    t_tune = time.perf_counter() - t0
    tuning = sorted(set(s.sadi_tuning_log() for s in ctxs))
    phis = {}
    for i, s in zip(mine, ctxs):
        N = inst[i][0]
        phis[i] = WL.gaussian_bumps(N, CFG["bumps"], inst[i][4])
        s.set_initial(phis[i])
    S.sadi_batch_step(ctxs, 1)                  # the n = 0 step (not replayed)
    graph = S.SadiGraph(ctxs, 1)
    kernels_per_step = graph.sadi_graph_kernels()
    graph.launch(max(a.warmup, 3))
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    with _nvtx("timed_steps"):
        for k in range(a.steps):
            evs[k][0].record(stream)
            graph.launch(1)
            evs[k][1].record(stream)
    barrier()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    clocks = sampler.stop()
    graph.close()
    # per-kernel phases of the largest instance of this rank (the dominant
    # group: the largest N carries most of the points), for the roofline
    big = max(range(len(ctxs)), key=lambda j: inst[mine[j]][0])
    cb = ctxs[big]
    cb.sadi_profile(True)
    S.sadi_batch_step([cb], 10)
    phase, nph = cb.sadi_get_phase_times()
    cb.sadi_profile(False)
    phase_ms = [t / max(nph, 1) for t in phase]
    Nb = inst[mine[big]][0]
    Npb = cb.sadi_get_info()[0]
    gb, pb = cb.sadi_get_options()
    roof = roofline_of(phase_ms, Nb, Npb, pb == S.SADI_PREC_FP32_DENSE, 1, None)
    roof["scope"] = f"one N={Nb} instance of the batch stepped alone"
    # e2e through the public API: set_initial from pinned host arrays, the
    # n = 0 step, then per step one graph launch + an asynchronous read of
    # every instance (sadi_get_async into pinned host buffers, two sets used
    # in turn), the reads waited for at the end.  The graph of one step is
    # captured before the timed region (a captured step serves every later
    # step of the same contexts).
    import ctypes
    lib = S.lib()
    pins = {i: torch.from_numpy(phis[i]).pin_memory() for i in mine}
    outs = [{i: torch.empty(phis[i].shape, dtype=torch.float64).pin_memory() for i in mine} for _ in range(2)]
    Ke = max(3, a.steps)   # as many steps as the device-timed run
    for i, s in zip(mine, ctxs):
        assert lib.sadi_set_initial(s.ctx, ctypes.c_void_p(pins[i].data_ptr()), None) == 0
    S.sadi_batch_step(ctxs, 1)
    g2 = S.SadiGraph(ctxs, 1)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for i, s in zip(mine, ctxs):
        assert lib.sadi_set_initial(s.ctx, ctypes.c_void_p(pins[i].data_ptr()), None) == 0
    S.sadi_batch_step(ctxs, 1)
    for k in range(Ke):
        g2.launch(1)
        for i, s in zip(mine, ctxs):
            assert lib.sadi_get_async(s.ctx, ctypes.c_void_p(outs[k % 2][i].data_ptr())) == 0
    for s in ctxs:
        assert lib.sadi_wait(s.ctx) == 0
    dt_e2e = time.perf_counter() - t0
    g2.close()
    barrier()
    h2d = sum(phis[i].size * 8 for i in mine) / (Ke + 1)
    d2h = sum(phis[i].size * 8 for i in mine)

    def reduce_max(vals):
        tt = torch.tensor(vals, dtype=torch.float64, device=dev)
        if ws > 1:
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        return [float(x) for x in tt.tolist()]
    ms_max, e2e_max = reduce_max([ms, dt_e2e])
    pts_all = sum(N * N for (N, _, _, _, _) in inst)
    value = pts_all * a.steps / (ms_max / 1e3)
    # e2e counts the n = 0 step and Ke graph steps of every instance
    e2e_val = pts_all * (Ke + 1) / e2e_max
    if rank == 0:
        # accuracy over the full step count: one instance per size against the
        # FP64 path from the same data, in the form the autotuner chose
        firsts = {}
        for i, (N, _, _, _, _) in enumerate(inst):
            firsts.setdefault(N, i)
        acc = {}
        pairs = []
        for N, i in sorted(firsts.items()):
            _, al, ka, ta, sd = inst[i]
            phi = WL.gaussian_bumps(N, CFG["bumps"], sd)
            prec = None
            for j, s in zip(mine, ctxs):
                if inst[j][0] == N:
                    prec = s.sadi_get_options()[1]
                    break
            if prec is None:
                prec = S.SADI_PREC_FP32
            c64 = S.Sadi(N, al, ka, ta)
            c64.set_options(CFG["g"], S.SADI_PREC_FP64)
            c64.set_initial(phi)
            c32 = S.Sadi(N, al, ka, ta)
            c32.set_options(CFG["g"], prec)
            c32.set_initial(phi)
            pairs.append((N, i, prec, c64, c32))
        acc_steps = CFG["total_steps"] if a.acc_steps > 0 else 0
        if acc_steps:
            S.sadi_batch_step([p[3] for p in pairs] + [p[4] for p in pairs], acc_steps)
        for N, i, prec, c64, c32 in pairs:
            if acc_steps:
                u64, _ = c64.get()
                u32, _ = c32.get()
                acc[str(N)] = {"instance": i, "form": {1: "fp32_gsfft", 2: "fp32_dense"}.get(prec, prec),
                               "rel_l2": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64))}
            c64.close()
            c32.close()
        cpu = None
        if ws == 1 and not a.no_cpu_baseline:
            cpu = batch_cpu_baseline(inst)
        nsz = {str(n): sum(1 for x in inst if x[0] == n) for n in CFG["sizes"]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sadi-batch 256 instances N~U{127,255,511,1023,2047} alpha~U(1.1,1.9) "
                                   "kappa~U(0.5,2) tau=h/2 g=-u^3 phi1=8 gaussian bumps phi2=0",
                       "instances": len(inst), "instances_per_size": nsz, "points_per_step": pts_all,
                       "parallelism": f"LPT-partitioned instances over {ws} rank(s), no collective",
                       "launch": "one CUDA graph launch per step covering every instance of the rank",
                       "l2": "working set of all instances far above L2 (no flush needed)",
                       "autotune": tuning, "setup_s": t_setup, "autotune_s": t_tune},
            "rel_l2_vs_fp64_full": {"steps": acc_steps, "per_size": acc} if acc_steps else None,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "how": "C ABI with pinned host buffers: sadi_set_initial of every instance, the n = 0 "
                           "batch step, then per step one graph launch (captured before the timed region) + "
                           "sadi_get_async of every instance into one of two pinned buffer sets, sadi_wait "
                           "at the end; wall clock"},
            "gpu_launches": kernels_per_step * a.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    for s in ctxs:
        s.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def batch_cpu_baseline(inst, budget_s=10.0):
    """The FP64 oracle (FFT tier) stepping instances of the batch in order,
    two n >= 1 steps each, until about budget_s seconds of work."""
    import numpy as np
    from oracle import sadi as O
    from paper_2312_06206_gb300 import workloads as WL
    pts = 0
    spent = 0.0
    used = 0
    for (N, al, ka, ta, sd) in inst:
        P = O.Problem(N, al, ka, ta, -1.0, 1.0, CFG["g"])
        u0 = WL.gaussian_bumps(N, CFG["bumps"], sd)
        u1 = O.step(P, None, u0, True, np.zeros_like(u0), tier="fft")
        t0 = time.perf_counter()
        up, uc = u0, u1
        for _ in range(2):
            up, uc = uc, O.step(P, up, uc, False, tier="fft")
        spent += time.perf_counter() - t0
        pts += 2 * N * N
        used += 1
        if spent >= budget_s:
            break
    return {"value": pts / spent, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the first {used} instances of the batch, 2 S-ADI steps (n>=1) each, oracle FFT tier "
                      "(FP64), default BLAS threading", "seconds": spent}


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    _select(a)
    if a.workload == "batch256":
        return run_batch(a)
    ws, rank, local = _dist()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi as S
    N = a.N
    phi1 = _workload(N)
    # a dedicated stream (the legacy default stream has handle 0, which the
    # library reads as "use the context's own stream")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def make(prec):
        ctxs = []
        for al in ALPHAS:
            s = S.Sadi(N, al, KAPPA, TAU, (-1.0, 1.0))
            s.set_options(GKIND, prec)
            s.set_stream(stream.cuda_stream)
            ctxs.append(s)
        if prec != S.SADI_PREC_FP64:
            # tiles of the shared-memory FFT engine tuned for this form
            S.sadi_autotune(ctxs, GKIND, 2)
        for s in ctxs:
            s.set_initial(phi1, _phi2(phi1))
        return ctxs

    def step_all(ctxs):
        S.sadi_batch_step(ctxs, 1)

    def timed(ctxs, K, W, profile=False):
        for _ in range(W):
            step_all(ctxs)
        if profile:
            ctxs[0].sadi_profile(True)
        # the FP32 forms replay one captured step per launch (sadi_graph_*);
        # the FP64 path (ping-pong state) and profiled passes launch directly
        graph = None
        if not profile and W > 0 and ctxs[0].sadi_get_options()[1] != S.SADI_PREC_FP64:
            graph = S.SadiGraph(ctxs, 1)
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        with _nvtx("timed_steps"):
            for k in range(K):
                flush.zero_()
                evs[k][0].record(stream)
                if graph is not None:
                    graph.launch(1)
                else:
                    step_all(ctxs)
                evs[k][1].record(stream)
        barrier()
        if graph is not None:
            graph.close()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        phases = None
        if profile:
            # the batched FP32 kernels cover all instances; their events are
            # recorded on the first context
            p, n = ctxs[0].sadi_get_phase_times()
            ctxs[0].sadi_profile(False)
            phases = ([t / n for t in p], n)
        return ms, phases

    # plain FP64 GS-FFT path (the baseline of the metric)
    sampler = ClockSampler(local)
    sampler.start()
    has64 = N <= 4096                      # the FP64 step path supports N <= 4096
    c64 = make(S.SADI_PREC_FP64) if has64 else []
    K64 = max(1, min(a.steps, 20))
    ms64 = timed(c64, K64, a.warmup)[0] if has64 else float("nan")
    # candidate forms: FP32 Gohberg-Semencul FFT sweeps, and (N <= 4096) the
    # dense-inverse sweeps as split-BF16 tensor-core GEMMs
    forms = [("fp32_gsfft", S.SADI_PREC_FP32)]
    if N <= 8192:
        forms.append(("fp32_dense", S.SADI_PREC_FP32_DENSE))
    res = {}
    for name, prec in forms:
        ctxs = make(prec)
        ms, _ = timed(ctxs, a.steps, a.warmup)
        res[name] = {"ctxs": ctxs, "ms": ms, "prec": prec}
    clocks = sampler.stop()
    # accuracy of each form against the plain FP64 path after the same number
    # of steps from the same data
    extra = a.warmup + a.steps - (a.warmup + K64)
    if has64 and extra > 0:
        S.sadi_batch_step(c64, extra)
    ref64 = [s.get() for s in c64]
    for name, r in res.items():
        rels = []
        for (u64, n64), s in zip(ref64, r["ctxs"]):
            u, n = s.get()
            assert n64 == n
            rels.append(float(np.linalg.norm(u - u64) / np.linalg.norm(u64)))
        r["rel_steps"] = (max(rels) if rels else None, a.warmup + a.steps)
    # accuracy at the workload's full step count: every form from phi1
    if a.acc_steps > 0 and has64:
        allc = c64 + [s for r in res.values() for s in r["ctxs"]]
        for s in allc:
            s.set_initial(phi1, _phi2(phi1))
        S.sadi_batch_step(allc, a.acc_steps)
        ref = [s.get()[0] for s in c64]
        for name, r in res.items():
            per = [float(np.linalg.norm(s.get()[0] - u64) / np.linalg.norm(u64)) for s, u64 in zip(r["ctxs"], ref)]
            r["rel_full"] = {"steps": a.acc_steps, "per_alpha": dict(zip([str(x) for x in ALPHAS], per)),
                             "max": max(per)}
    # the chosen form: the fastest one within the stated accuracy (1e-5
    # relative L2 against the plain FP64 path)
    TOL = 1e-5

    def acc_of(r):
        return r["rel_full"]["max"] if "rel_full" in r else r["rel_steps"][0]
    ok = [n for n, r in res.items() if acc_of(r) is None or acc_of(r) <= TOL]
    chosen = min(ok or list(res), key=lambda n: res[n]["ms"])
    cc = res[chosen]["ctxs"]
    dense = res[chosen]["prec"] == S.SADI_PREC_FP32_DENSE
    # per-kernel timing (separate profiled pass) for the roofline
    for s in cc:
        s.set_initial(phi1, _phi2(phi1))
    Kp = max(5, min(a.steps, 20))
    _, (phase_ms, _) = timed(cc, Kp, 3, profile=True)
    Np = cc[0].sadi_get_info()[0]
    roofline = roofline_of(phase_ms, N, Np, dense, len(ALPHAS), a.workload if a.N == PRESETS[a.workload]["N"] else None)
    # e2e through the public API with host buffers: set_initial from pinned
    # host arrays, then every step sadi_batch_step(1) + sadi_get into pinned host.
    pin_in = torch.from_numpy(phi1).pin_memory()
    p2h = _phi2(phi1)
    pin_in2 = None if p2h is None else torch.from_numpy(np.ascontiguousarray(p2h)).pin_memory()
    pin_out = [[torch.empty((N, N), dtype=torch.float64).pin_memory() for _ in ALPHAS] for _ in range(2)]
    Ke = max(3, a.steps)   # as many steps as the device-timed run
    import ctypes
    lib = S.lib()
    arr = (ctypes.c_void_p * len(cc))(*[s.ctx for s in cc])

    def set_all():
        for s in cc:
            st = lib.sadi_set_initial(s.ctx, ctypes.c_void_p(pin_in.data_ptr()),
                                      None if pin_in2 is None else ctypes.c_void_p(pin_in2.data_ptr()))
            assert st == 0, s.sadi_last_error()
    # the graph of one batched step, captured before the timed region (a
    # captured step serves every later step of the same contexts)
    set_all()
    assert lib.sadi_batch_step(arr, len(cc), 1) == 0
    ge = S.SadiGraph(cc, 1)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    set_all()
    assert lib.sadi_batch_step(arr, len(cc), 1) == 0          # the n = 0 step
    for i, s in enumerate(cc):
        assert lib.sadi_get_async(s.ctx, ctypes.c_void_p(pin_out[1][i].data_ptr())) == 0
    for k in range(Ke - 1):
        ge.launch(1)
        for i, s in enumerate(cc):
            assert lib.sadi_get_async(s.ctx, ctypes.c_void_p(pin_out[k % 2][i].data_ptr())) == 0
    for s in cc:
        assert lib.sadi_wait(s.ctx) == 0
    dt_e2e = time.perf_counter() - t0
    ge.close()
    barrier()
    h2d = len(ALPHAS) * N * N * 8 * (1 if pin_in2 is None else 2) / Ke
    d2h = len(ALPHAS) * N * N * 8

    # aggregate over ranks (max time)
    def reduce_max(vals):
        tt = torch.tensor(vals, dtype=torch.float64, device=dev)
        if ws > 1:
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        return [float(x) for x in tt.tolist()]
    pts = N * N * len(ALPHAS)
    others = [n for n in res if n != chosen]
    agg = aggregate([res[chosen]["ms"], ms64 if has64 else 1.0, dt_e2e], ws, pts, (a.steps, K64, Ke), reduce_max)
    agg_o = {n: aggregate([res[n]["ms"], 1.0, 1.0], ws, pts, (a.steps, 1, 1), reduce_max) for n in others}
    value, value64, e2e_val = agg["value"], agg["value64"], agg["e2e"]
    c1 = c1_latency(S, stream) if rank == 0 and a.workload == "n1023" else None
    if rank == 0:
        cpu = None
        rel_oracle = None
        if ws == 1 and not a.no_cpu_baseline and a.workload == "n1023":
            cpu, (u0, u1, uK) = cpu_baseline(N, phi1, alpha=ALPHAS[len(ALPHAS) // 2])
            # each GPU form vs the oracle after the same 1 + 3 steps (middle alpha)
            rel_oracle = {"alpha": ALPHAS[len(ALPHAS) // 2]}
            for nm, prec in [("fp64", S.SADI_PREC_FP64)] + forms:
                with S.Sadi(N, ALPHAS[len(ALPHAS) // 2], KAPPA, TAU, (-1.0, 1.0)) as s:
                    s.set_options(GKIND, prec)
                    s.set_initial(phi1, _phi2(phi1))
                    s.step(4)
                    ug, _ = s.get()
                    rel_oracle[nm] = float(np.linalg.norm(ug - uK) / np.linalg.norm(uK))
        form_desc = {"fp32_gsfft": "FP32 FFTs and Gohberg-Semencul FFT sweeps, double-float state, FP64 setup",
                     "fp32_dense": "FP32 FFTs for L_h; both sweeps as split-BF16 dense-inverse tcgen05 GEMMs "
                                   "(FP32 accumulate); double-float state; FP64 setup"}
        forms_out = {}
        for n, r in res.items():
            v = value if n == chosen else agg_o[n]["value"]
            forms_out[n] = {"value": v, "unit": UNIT, "ms_per_step": r["ms"] / a.steps,
                            "rel_l2_vs_fp64": {"steps": r["rel_steps"][1], "max": r["rel_steps"][0]},
                            "rel_l2_vs_fp64_full": r.get("rel_full"), "form": form_desc[n]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": agg["ms32"] / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(N, {"form": form_desc[chosen], "chosen_form": chosen,
                                  "selection": f"fastest form within {TOL:g} relative L2 of the plain FP64 path "
                                               f"after the accuracy run",
                                  "parallelism": f"replicas x{ws}",
                                  "l2": "flushed between timed steps (256 MiB write outside the step events)"}),
            "fp64_plain": {"value": value64, "unit": UNIT, "ms_per_step": agg["ms64"] / K64, "steps": K64}
            if has64 else None,
            "speedup_vs_fp64": value / value64 if has64 else None,
            "forms": forms_out,
            "rel_l2_vs_oracle_4steps": rel_oracle,
            "c1_small": c1,
            "roofline": roofline,
            "batched": "one launch per kernel covers all instances (sadi_batch_step)",
            "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "how": "C ABI with pinned host buffers: sadi_set_initial once, the n = 0 step by "
                           "sadi_batch_step, then per step one launch of the step graph (captured before the "
                           "timed region) + sadi_get_async of u^{n+1} (FP64, N^2 doubles) for each instance "
                           "into one of two pinned buffer sets, sadi_wait at the end; wall clock"},
            "gpu_launches": launches_per_step(Np, chosen == "fp32_dense") * a.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    for s in c64 + [s for r in res.values() for s in r["ctxs"]]:
        s.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
