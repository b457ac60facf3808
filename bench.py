"""Benchmark: ALS sweeps/s of TR-ALS-Sampled on the 500x500x500 FP32 rank-10 workload.

One step = one whole decomposition through the C ABI (tr_als_sampled: initial leverage
scores + 10 sweeps of Alg. 2, J = 4000, mixed precision) with X resident in HBM. The
metric is sweeps/s = sweeps per step * steps / time. Besides it the JSON line carries the
end-to-end number through the host-memory entry point, the roofline of the dominant
kernel, the plain FP64 GPU form (the metric's comparator), the FP64 CPU oracle on a
bounded sample, the same decomposition with uniform sampling (Sec. 5 variant) and with
dense TR-ALS (Alg. 1, the paper's comparison method), the 512-problem batched workload, and the serving leg: p50/p99 decomposition latency of a
Poisson stream of requests (200/s) through the native server.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--serve-seconds S] [--skip-cpu] [--skip-fp64] [--skip-uniform] [--skip-dense]
                  [--paper-protocol]
                  [--skip-batched] [--skip-configs] [--skip-serving]

With N > 1 (torchrun), every rank decomposes its own tensor (replicas, weak scaling).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2010_08581_gb300 import inputs  # noqa: E402

WORKLOAD = "tr3_500_r10_fp32"
METRIC = "ALS sweeps/s at fixed rel. fit vs plain FP64 GPU; p50/p99 decomposition latency"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
NOMINAL_FP64_TFLOPS = 1.25


def workload_config(wl):
    return {
        "workload": f"{WORKLOAD}: 500x500x500 FP32 X = TR(rank-10 N(0,1) cores) + 1e-2 rel. "
                    f"Gaussian noise; target ranks 10, J={wl['J']}, {wl['sweeps']} sweeps per "
                    "step (one whole decomposition), mixed precision: FP32 design rows and "
                    "fibres; TF32x3 tensor-core normal equations with FP32 accumulation; "
                    "normal matrix factored in FP32 together with the factor's FP32 "
                    "inverse (FP64 factorisation if a pivot is small), FP32 solves by "
                    "that inverse and one refinement step; leverage scores from the "
                    "double-float Gram through an FP32 Cholesky preconditioner and a "
                    "double-float series (the double-float factorisation with FP64 fallback "
                    "when the preconditioner is poor); strided modes read from contiguous "
                    "copies of X made in every step",
        "dims": list(wl["dims"]), "ranks": list(wl["ranks"]), "J": wl["J"],
        "sweeps_per_step": wl["sweeps"],
        "l2": "inputs larger than L2: X is 500 MB (> 129 MB L2); samples are redrawn every "
              "step (seed + step)",
    }


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def allreduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, local_seconds: float, world: int) -> float:
    """Whole-job throughput of `world` replicas: all ranks' units over the slowest rank's
    time (max over ranks)."""
    return world * units_per_rank / allreduce_max(local_seconds, world)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            out["reasons"] = ["nvidia-smi unavailable"]
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# --------------------------------------------------------------------------------------
# roofline of the dominant kernel
# --------------------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    return d


def _peak_hbm(peaks):
    if peaks:
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in peaks and isinstance(peaks[k], (int, float)):
                return float(peaks[k]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def algorithmic_cost(kernel, wl):
    """(kind, per-launch algorithmic bytes or flops) of one launch on this workload.

    Per core update n (I = I_n, L = R^2 = 100, J = 4000 samples, FP32 rows and fibres):
      gather          : J*I*4 bytes read (fibres) + J*I*4 written
      subchain        : J*(N-1)*L*8 slice bytes read + J*L*4 written
      normal_eq_tc    : 2*J*L*(L + I) useful flops (TF32 tensor cores)
      cholesky_leverage: L^3/3 flops in double-float (FP32 pairs; one CTA, mixed path)
      cholesky_solve  : L^3/3 flops in FP32 (one CTA, mixed path: the factor; the inverse
                        formed in the same pass replaces the substitutions of solve_rhs,
                        whose flops are counted there)
      solve_rhs       : 6*L^2*I FP32 flops (two triangular solve pairs + residual)
      gram_f64        : 2*I*L^2 FP64 flops
      leverage_rows   : I*L^2 FP64 flops
      sample          : J*(N-1) * (4 + 8*log2 I) bytes (index writes + CDF probes) + J*8
      sample_chain    : sample + subchain + gather (draws, rows and fibres in one kernel)
      lev_factor      : 2*L^3/3 FP32 flops (one CTA: the preconditioner's Cholesky factor
                        and its inverse X in one pass)
      gram_dd         : I*L^2 double-float flops (Gram of B^T, upper tiles)
      lev_u, lev_e    : L^3 and L^3/3 double-float flops (U = X K, E = U X^T - I)
      lev_rows        : I*L^2 double-float flops (w = X b per row; the FP32 series is smaller)
      mode_last       : 2 * |X| * 4 bytes (X read and its copy written, once per strided mode)
    """
    dims, ranks, J = wl["dims"], wl["ranks"], wl["J"]
    N = len(dims)
    I = sum(dims) / N
    L = ranks[0] * ranks[1]
    s = 4
    table = {
        "gather": ("hbm", 2.0 * J * I * s),
        "normal_eq": ("flops_f32", 2.0 * J * L * (L + I)),
        "normal_eq_tc": ("flops_tf32", 2.0 * J * L * (L + I)),
        "subchain": ("hbm", J * (N - 1) * L * 8.0 + J * L * s),
        "cholesky_solve": ("flops_f32", L ** 3 / 3.0),
        "cholesky_leverage": ("flops_ff", L ** 3 / 3.0),
        "solve_rhs": ("flops_f32", 6.0 * L * L * I),
        "gram_f64": ("flops_f64", 2.0 * I * L * L),
        "leverage_rows": ("flops_f64", I * L * L),
        "sample": ("hbm", J * (N - 1) * (4 + 8 * math.log2(max(I, 2))) + J * 8),
        "sample_chain": ("hbm", J * (N - 1) * (4 + 8 * math.log2(max(I, 2))) + J * 8
                         + J * (N - 1) * L * 8.0 + J * L * s + 2.0 * J * I * s),
        "reduce_MB": ("hbm", L * (L + I) * 8.0),
        "reduce_gram": ("hbm", L * L * 8.0),
        "cdf": ("hbm", I * 8.0 * 3),
        "init_normal": ("hbm", I * L * 8.0),
        "lev_factor": ("flops_f32", 2.0 * L ** 3 / 3.0),
        "gram_dd": ("flops_ff", I * L * L),
        "lev_u": ("flops_ff", float(L) ** 3),
        "lev_e": ("flops_ff", L ** 3 / 3.0),
        "lev_rows": ("flops_ff", I * L * L),
        "mode_last": ("hbm", 2.0 * math.prod(dims) * s),
    }
    return table.get(kernel)


def traffic_for(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, if its source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(kernel)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2010_08581_gb300", "csrc", e.get("source", ""))
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except Exception:
        return None
    return e.get("bytes_per_launch") if h == e.get("source_sha") else None


def roofline(prof, wl, peaks):
    """The roofline object of the kernel with the largest share of the timed kernel time
    (among those with a stated algorithmic cost)."""
    top = rooflines(prof, wl, peaks, 1)
    return top[0] if top else None


def rooflines(prof, wl, peaks, k):
    """Roofline objects of the k kernels with the largest shares of the timed kernel time."""
    tot_ms = sum(v[0] for v in prof.values())
    out = []
    for name, (ms, n) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        e = roofline_entry(name, ms, n, wl, peaks)
        if e is None:
            continue
        e["share_of_timed"] = round(ms / max(tot_ms, 1e-9), 4)
        out.append(e)
        if len(out) == k:
            break
    return out


_SM_COUNT = []


def alu_basis(peaks):
    """SM count and SM clock (GHz) behind the ALU peaks: the count queried from the device
    (152 on GB300 when no device is visible), the clock from the measured peaks' sm_max_mhz
    (GB300's 2070 MHz maximum otherwise)."""
    if not _SM_COUNT:
        sms = 152
        try:
            if torch.cuda.is_available():
                sms = int(torch.cuda.get_device_properties(0).multi_processor_count)
        except Exception:
            pass
        _SM_COUNT.append(sms)
    mhz = (peaks or {}).get("sm_max_mhz")
    ghz = float(mhz) / 1e3 if isinstance(mhz, (int, float)) and mhz > 0 else 2.07
    return _SM_COUNT[0], ghz


def roofline_entry(name, ms, n, wl, peaks):
    """Roofline object of one kernel: algorithmic work per launch over its average launch time."""
    cost = algorithmic_cost(name, wl)
    if cost is None:
        return None
    kind, amount = cost
    avg_s = ms / 1e3 / n
    sms, ghz = alu_basis(peaks)
    if kind == "hbm":
        peak, src = _peak_hbm(peaks)
        ach = amount / avg_s / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": round(ach, 3), "peak": peak,
                "unit": "GB/s", "frac": round(ach / peak, 5),
                "traffic": traffic_for(name), "peak_source": f"{src} HBM copy",
                "avg_launch_us": round(avg_s * 1e6, 3), "launches": n,
                "share_of_timed": None}
    if kind == "flops_f64":
        # FP64 ALU: nominal GB300 FP64 rate (no measured FP64 peak is provided); an FMA
        # microbenchmark on this GPU measured 1.20 TFLOP/s, about 2 DFMA/clk/SM.
        peak = NOMINAL_FP64_TFLOPS
        ach = amount / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": round(ach, 6), "peak": peak,
                "unit": "TFLOP/s", "frac": round(ach / peak, 5),
                "frac_of_one_sm": round(ach / (peak / sms), 4),
                "traffic": traffic_for(name),
                "peak_source": f"nominal FP64 1.25 TFLOP/s for {sms} SMs (one-CTA kernels are "
                               "bounded by one SM: see frac_of_one_sm)",
                "avg_launch_us": round(avg_s * 1e6, 3), "launches": n,
                "share_of_timed": None}
    if kind == "flops_f32":
        # SIMT FP32: SMs * 128 FMA/clk * 2 * SM clock
        peak = sms * 128 * 2 * ghz * 1e9 / 1e12
        ach = amount / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(ach / peak, 5),
                "frac_of_one_sm": round(ach / (peak / sms), 4),
                "traffic": traffic_for(name),
                "peak_source": f"FP32 SIMT: {sms} SMs x 128 FMA/clk x 2 x {ghz:.2f} GHz",
                "avg_launch_us": round(avg_s * 1e6, 3), "launches": n,
                "share_of_timed": None}
    if kind == "flops_ff":
        # double-float on the FP32 pipe: one multiply-add a - x*y is 15 FP32 instructions
        # (Dekker's product via FMA, then a two-sum); 128 lanes/clk/SM at the SM clock
        per_sm = 128 * ghz * 1e9 * 2 / 15 / 1e12
        peak = sms * per_sm
        ach = amount / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": round(ach, 6),
                "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(ach / peak, 5),
                "frac_of_one_sm": round(ach / per_sm, 4),
                "frac_of_one_sm_fp64": round(ach / (NOMINAL_FP64_TFLOPS / sms), 4),
                "traffic": traffic_for(name),
                "peak_source": f"double-float on FP32 SIMT: {sms} SMs x 128 lanes x {ghz:.2f} GHz x "
                               "2 flops / 15 instructions per multiply-add (one-CTA kernel: "
                               "see frac_of_one_sm; frac_of_one_sm_fp64 compares with one "
                               "SM's nominal FP64 rate)",
                "avg_launch_us": round(avg_s * 1e6, 3), "launches": n,
                "share_of_timed": None}
    if kind == "flops_tf32":
        bf16, src = (peaks or {}).get("bf16_tflops"), "measured"
        if not isinstance(bf16, (int, float)):
            bf16, src = FALLBACK_BF16_TFLOPS, "fallback"
        peak = bf16 * 0.5          # dense TF32 = half the dense BF16 rate (nominal ratio)
        ach = amount / avg_s / 1e12
        return {"kernel": name, "bound": "tensor", "achieved": round(ach, 3),
                "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(ach / peak, 5),
                "traffic": traffic_for(name),
                "peak_source": f"{src} BF16 x 0.5 (TF32/BF16 nominal ratio)",
                "avg_launch_us": round(avg_s * 1e6, 3), "launches": n,
                "share_of_timed": None}
    return None


# --------------------------------------------------------------------------------------
# CPU oracle on a bounded sample
# --------------------------------------------------------------------------------------
def oracle_sample(X_np, init_paper, wl, budget_s=15.0, max_sweeps=50):
    """Time the FP64 NumPy oracle (as it stands) doing whole sweeps of the same workload
    until about budget_s seconds of CPU work."""
    import oracle as orc
    N = len(wl["dims"])
    cores = [np.array(c, dtype=np.float64) for c in init_paper]
    ps, cdfs = [None] * N, [None] * N
    t0 = time.perf_counter()
    for k in range(1, N):
        ps[k], cdfs[k] = orc.core_distribution(cores[k])
    sweeps = 0
    while sweeps < max_sweeps:
        for n in range(N):
            cores[n], _, _ = orc.sampled_core_update(X_np, cores, ps, cdfs, n, wl["J"],
                                                     wl["sample_seed"], sweeps * N + n)
            ps[n], cdfs[n] = orc.core_distribution(cores[n])
        sweeps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    try:
        ncores = len(os.sched_getaffinity(0))
    except Exception:
        ncores = os.cpu_count()
    return sweeps, dt, ncores


def oracle_sample_single_thread(budget_s=10.0):
    """The same bounded oracle sample in a child process whose BLAS and OpenMP pools are held
    to one thread (the thread counts are fixed when NumPy loads, hence the child). Returns
    (sweeps, seconds) or None if the child fails."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = (
        "import json, sys, torch\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import bench\n"
        "from paper_2010_08581_gb300 import inputs\n"
        "torch.set_num_threads(1)\n"
        "wl = inputs.WORKLOADS[bench.WORKLOAD]\n"
        "X, _ = inputs.tr_plus_noise(wl['dims'], wl['ranks'], seed=wl['seed'], "
        "rel_noise=wl['rel_noise'], dtype=torch.float32)\n"
        "init = [c.numpy() for c in inputs.random_cores(wl['dims'], wl['ranks'], wl['init_seed'])]\n"
        f"sw, dt, _ = bench.oracle_sample(X.numpy(), init, wl, budget_s={budget_s!r}, max_sweeps=50)\n"
        "print(json.dumps({'sweeps': sw, 'seconds': dt}))\n")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=budget_s * 20 + 120)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def run_batched(T, plain_fp64, dev, steps, warmup, stream):
    """512 independent 3-way FP32 problems (I_n ~ U{32..200}, ranks ~ U{3..8}, J = 10 max L,
    10 sweeps each) through tr_als_sampled_batched: one step = the whole batch."""
    from paper_2010_08581_gb300 import autotune
    count, sweeps = 512, 10
    probs = inputs.batched_workload(count, seed=4, device=dev)
    ctxb = T.Context(dev.index if dev.index is not None else 0)
    for pr in probs:
        pr["cores"] = T.empty_cores(pr["dims"], pr["ranks"], device=dev)
        pr["init"] = False
    t0 = time.perf_counter()
    tuned = autotune.tune_batched(ctxb, probs, T.TR_PREC_MIXED)
    tune_s = time.perf_counter() - t0
    for i in range(max(1, warmup)):
        T.tr_als_sampled_batched(ctxb, probs, sweeps, T.TR_PREC_MIXED)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for i in range(steps):
        for pr in probs:
            pr["seed"] += 1
        evs[i][0].record(stream)
        T.tr_als_sampled_batched(ctxb, probs, sweeps, T.TR_PREC_MIXED)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    tot_s = sum(ms) / 1e3
    fits = [T.tr_rel_error(ctxb, pr["X"], pr["ranks"], pr["cores"]) for pr in probs[:16]]
    # the plain FP64 GPU form on a few of the same problems, one after another
    nplain = 8
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    inits = [[c.to(dev) for c in inputs.random_cores(pr["dims"], pr["ranks"], 5 + i)]
             for i, pr in enumerate(probs[:nplain])]
    plain_fp64.als_sampled(probs[0]["X"], inits[0], probs[0]["J"], 1, 0)
    torch.cuda.synchronize()
    a.record(stream)
    for i, pr in enumerate(probs[:nplain]):
        plain_fp64.als_sampled(pr["X"], inits[i], pr["J"], sweeps, i)
    b.record(stream)
    torch.cuda.synchronize()
    plain_rate = nplain * sweeps / (a.elapsed_time(b) / 1e3)
    ctxb.close()
    rate = count * sweeps * steps / tot_s
    return {"workload": "512 independent 3-way FP32 problems, I_n ~ U{32..200}, TR ranks ~ "
                        "U{3..8}, TR(N(0,1)) + 1e-3 noise, J = 10 max_k L_k, 10 sweeps each, "
                        "mixed precision, one tr_als_sampled_batched call per step",
            "value": round(rate, 1), "unit": "instance-sweeps/s", "steps": steps,
            "ms_per_batch": round(tot_s * 1e3 / steps, 3),
            "median_rel_err_first16": float(np.median(fits)),
            "plain_fp64_gpu_form": {"value": round(plain_rate, 2), "unit": "instance-sweeps/s",
                                    "what": f"{nplain} of the problems decomposed one after "
                                            "another by the plain FP64 form"},
            "speedup_vs_plain_fp64": round(rate / plain_rate, 1),
            "tiles": {"samples_per_warp": tuned["samples_per_warp"],
                      "contract_tile": tuned["contract_tile"], "from_table": tuned["cached"],
                      "tuning_s": round(tune_s, 3),
                      "ms_per_one_sweep_call": tuned.get("ms"),
                      "what": "launch shapes chosen by the project's autotuner on scratch "
                              "copies of this batch (results do not depend on them)"}}


def run_fp64_factorisations(T, X, ranks, J, sweeps, init_dev, wl, stream, reps, value, fit):
    """The headline decomposition with TR_FACTOR_FP64: the normal matrix and the leverage
    Gram factored in FP64 (the rest of the mixed path unchanged), same inputs and seeds."""
    ctx = T.Context(torch.cuda.current_device())
    T.tr_set_factorization(ctx, T.TR_FACTOR_FP64)
    cores = T.empty_cores(wl["dims"], ranks, device=X.device)

    def call(i):
        T.tr_als_sampled(ctx, X, ranks, J, sweeps, wl["sample_seed"] + i, T.TR_PREC_MIXED, cores,
                         init_cores=init_dev)

    for i in range(2):
        call(i)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(reps):
        call(i)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    err = T.tr_rel_error(ctx, X, ranks, cores)
    ctx.close()
    v = sweeps * reps / sec
    return {"value": round(v, 3), "unit": "sweeps/s", "final_rel_err": err,
            "default_over_this": round(value / v, 3),
            "equal_fit": abs(err - fit) <= 0.01 * err,
            "what": "normal matrix and leverage Gram factored in FP64 (TR_FACTOR_FP64); "
                    "rows, fibres, contraction, FP32 solves with one refinement step as in "
                    "the headline"}


def run_uniform(T, X, ranks, J, sweeps, init_dev, dims, stream, reps):
    """The same decomposition with uniform draws (no distributions formed), at J and 5 J
    samples per update: sweeps/s and the final relative error of each."""
    ctx = T.Context(torch.cuda.current_device())
    T.tr_set_sampling(ctx, T.TR_SAMPLING_UNIFORM)
    out = {}
    for mult in (1, 5):
        Ju = J * mult
        cores = T.empty_cores(dims, ranks, device=X.device)

        def call(i):
            T.tr_als_sampled(ctx, X, ranks, Ju, sweeps, 500 + i, T.TR_PREC_MIXED, cores,
                             init_cores=init_dev)

        for i in range(3):
            call(i)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(reps):
            call(3 + i)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        out[f"J={Ju}"] = {"value": round(sweeps * reps / sec, 3), "unit": "sweeps/s",
                          "final_rel_err": T.tr_rel_error(ctx, X, ranks, cores)}
    ctx.close()
    return out


def run_dense(T, X, ranks, sweeps, init_dev, dims, stream, reps, sampled_value, sampled_err):
    """Dense TR-ALS (Alg. 1, every row of each least-squares problem) on the same workload and
    the same LS path: sweeps/s, final error, and the sampled method's speedup over it."""
    ctx = T.Context(torch.cuda.current_device())
    cores = T.empty_cores(dims, ranks, device=X.device)

    def call():
        T.tr_als(ctx, X, ranks, sweeps, 0, T.TR_PREC_MIXED, cores, init_cores=init_dev)

    call()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        call()
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    value = sweeps * reps / sec
    err = T.tr_rel_error(ctx, X, ranks, cores)
    T.tr_profile_begin(ctx)
    call()
    prof = T.tr_profile_end(ctx)
    ctx.close()
    return {"value": round(value, 3), "unit": "sweeps/s", "final_rel_err": err,
            "sampled_speedup": round(sampled_value / value, 3),
            "sampled_err_ratio": round(sampled_err / err, 4),
            "kernels_ms_one_decomposition": {k: [round(v[0], 3), v[1]] for k, v in
                                             sorted(prof.items(), key=lambda kv: -kv[1][0])},
            "what": "TR-ALS (Alg. 1) through tr_als, mixed precision, same initial cores; "
                    "sampled_speedup = the headline sweeps/s / this"}


def _tolerate_singular(T, fn, flags):
    """Run fn; a TR_ERR_SINGULAR status (that update kept its core) is recorded, not raised."""
    try:
        fn()
    except T.TrError as e:
        if e.status != T.TR_ERR_SINGULAR:
            raise
        flags["singular_updates"] = True


def _converge_dense(T, ctx, X, ranks, cores, init, flags, tol=1e-6, cap=100):
    """Alg. 1 one sweep per call until the relative error changes by less than tol (the
    paper's TR-ALS criterion) or cap sweeps. Returns (sweeps, error, device ms of the sweeps)."""
    ms, prev, it = 0.0, None, 0
    cur_init = init
    while it < cap:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _tolerate_singular(T, lambda: T.tr_als(ctx, X, ranks, 1, 0, T.TR_PREC_MIXED, cores,
                                               init_cores=cur_init), flags)
        b.record()
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        it += 1
        err = T.tr_rel_error(ctx, X, ranks, cores)
        cur_init = [c.clone() for c in cores]
        if prev is not None and abs(prev - err) < tol:
            break
        prev = err
    return it, err, ms


def _grow_j(T, ctx, X, ranks, cores, init, sweeps, target, j0, dj, flags, jcap=40000):
    """The smallest J (j0, j0 + dj, ...) whose sampled run of `sweeps` sweeps reaches an
    error below target. Returns (J, error, device ms of that run) or the last try."""
    J = j0

    def run():
        T.tr_als_sampled(ctx, X, ranks, J, sweeps, 11, T.TR_PREC_MIXED, cores, init_cores=init)

    while True:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _tolerate_singular(T, run, flags)
        torch.cuda.synchronize()
        a.record()
        _tolerate_singular(T, run, flags)
        b.record()
        torch.cuda.synchronize()
        err = T.tr_rel_error(ctx, X, ranks, cores)
        if err < target or J + dj > jcap:
            return J, err, a.elapsed_time(b)
        J += dj


def run_paper_protocol(T, dev):
    """The paper's decomposition protocol (Sec. 5 and its supplement) on GB300, one seeded
    run per case: TR-ALS until the error changes by < 1e-6 (cap 100 sweeps), then the
    sampled method with the same number of sweeps and J grown until its error is below
    1.2x TR-ALS's. Cases: the coherent random tensors (R' = R = 10, I = 100..500) and the
    three oscillatory functions on 4^10 points (R = 10)."""
    ctx = T.Context(torch.cuda.current_device())
    T.tr_set_ls_rank(ctx, T.TR_LS_RANK_DROP)   # basic LS solutions, as a QR-based solve gives
    out = {"what": "TR-ALS to convergence, then the smallest J (paper's increments) with the "
                   "sampled error < 1.2x; times are device ms of the whole decomposition; one "
                   "seeded run per case (the paper reports medians of 10); LS steps drop "
                   "columns with small pivots (basic solutions)"}
    cases = [("coherent_I%d" % I, None, I) for I in (100, 200, 300, 400, 500)]
    cases += [("oscillatory_" + nm, nm, None) for nm in inputs.OSCILLATORY]
    for name, fn, I in cases:
        if fn is None:
            X, _ = inputs.coherent_tr(I, 10, seed=I, device=dev)
            dims, ranks, j0, dj = (I, I, I), (10, 10, 10), 200, 100
        else:
            X = inputs.oscillatory(fn).to(dev)
            dims, ranks, j0, dj = (4,) * 10, (10,) * 10, 1000, 1000
        init = [inputs.slice_major(c).to(dev) for c in inputs.random_cores(dims, ranks, 77)]
        cores = T.empty_cores(dims, ranks, device=dev)
        fd, fs = {}, {}
        it, e_als, ms_als = _converge_dense(T, ctx, X, ranks, cores, init, fd)
        J, e_s, ms_s = _grow_j(T, ctx, X, ranks, cores, init, it, 1.2 * e_als, j0, dj, fs)
        out[name] = {"sweeps": it, "tr_als_err": e_als, "tr_als_ms": round(ms_als, 3),
                     "J": J, "sampled_err": e_s, "sampled_ms": round(ms_s, 3),
                     "speedup": round(ms_als / ms_s, 2),
                     "singular_updates": {"tr_als": bool(fd), "sampled": bool(fs)}}
        del X
        torch.cuda.empty_cache()
    ctx.close()
    return out


def _time_calls(fn, reps, stream):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    a.record(stream)
    for i in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def run_config1(T, plain_fp64, dev, stream, reps=5):
    """100x100x100 FP64 TR of rank 5 + 1e-3 noise, J = 2000, 10 sweeps, FP64 path, against
    the plain FP64 GPU form on the same problem and initial cores."""
    wl = inputs.WORKLOADS["tr3_100_r5_fp64"]
    X, _ = inputs.tr_plus_noise(wl["dims"], wl["ranks"], seed=wl["seed"],
                                rel_noise=wl["rel_noise"], device=dev, dtype=torch.float64)
    init = [c.to(dev) for c in inputs.random_cores(wl["dims"], wl["ranks"], wl["init_seed"])]
    init_sm = [inputs.slice_major(c) for c in init]
    ctx = T.Context(dev.index or 0)
    out = T.empty_cores(wl["dims"], wl["ranks"], device=dev)
    sec = _time_calls(lambda: T.tr_als_sampled(ctx, X, wl["ranks"], wl["J"], wl["sweeps"],
                                               wl["sample_seed"], T.TR_PREC_FP64, out,
                                               init_cores=init_sm), reps, stream)
    err = T.tr_rel_error(ctx, X, wl["ranks"], out)
    res = [None]

    def plain():
        res[0] = plain_fp64.als_sampled(X, init, wl["J"], wl["sweeps"], 1)
    psec = _time_calls(plain, 2, stream)
    perr = plain_fp64.rel_error(X, res[0])
    ctx.close()
    return {"workload": "100x100x100 FP64 TR(rank-5 N(0,1)) + 1e-3 noise, ranks 5, J = 2000, "
                        "10 sweeps per decomposition, FP64 path",
            "value": round(wl["sweeps"] / sec, 2), "unit": "sweeps/s",
            "ms_per_decomposition": round(sec * 1e3, 3), "final_rel_err": err,
            "plain_fp64_gpu_form": {"value": round(wl["sweeps"] / psec, 2), "unit": "sweeps/s",
                                    "final_rel_err": perr},
            "speedup_vs_plain_fp64": round(psec / sec, 2)}


def run_config3(T, dev, stream, peaks, reps=3):
    """4-way 256x256x3x2000 FP32 cosine workload, ranks 10, J = 8000, 20 sweeps, mixed; and
    the fibre gather of its contiguous mode (I = 2000) timed per launch against HBM peak."""
    dims, ranks, J, sweeps = (256, 256, 3, 2000), (10, 10, 10, 10), 8000, 20
    X = inputs.cosine_sum(dims, seed=0, device=dev)
    init = [inputs.slice_major(c).to(dev) for c in inputs.random_cores(dims, ranks, 1)]
    ctx = T.Context(dev.index or 0)
    out = T.empty_cores(dims, ranks, device=dev)
    sec = _time_calls(lambda: T.tr_als_sampled(ctx, X, ranks, J, sweeps, 2, T.TR_PREC_MIXED,
                                               out, init_cores=init), reps, stream)
    err = T.tr_rel_error(ctx, X, ranks, out)
    # gather of mode 3: J fibres of 2000 contiguous floats, read and written once
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    idx = torch.stack([torch.randint(0, d, (J,), generator=g, device=dev) for d in dims[:3]],
                      1).to(torch.int32).contiguous()
    w = torch.rand(J, generator=g, device=dev, dtype=torch.float64)
    Y = torch.empty((J, dims[3]), device=dev)
    gsec = _time_calls(lambda: T.tr_gather(ctx, X, 3, idx, w, Y), 50, stream)
    gbytes = 2.0 * J * dims[3] * 4
    peak, src = _peak_hbm(peaks)
    ctx.close()
    return {"workload": "256x256x3x2000 FP32 sum of 20 separable low-frequency cosine products "
                        "+ 5% uniform noise, ranks 10, J = 8000, 20 sweeps, mixed precision",
            "value": round(sweeps / sec, 2), "unit": "sweeps/s",
            "ms_per_decomposition": round(sec * 1e3, 3), "final_rel_err": err,
            "gather_mode3": {"bytes_per_launch": gbytes, "us_per_launch": round(gsec * 1e6, 2),
                             "achieved_gbs": round(gbytes / gsec / 1e9, 1), "peak_gbs": peak,
                             "frac": round(gbytes / gsec / 1e9 / peak, 4),
                             "peak_source": f"{src} HBM copy",
                             "what": "J = 8000 fibres of the contiguous mode (I = 2000, FP32), "
                                     "read + weighted write, CUDA events over 50 launches"}}


def run_serving(T, dev, seconds, rate=200.0, warmup_s=3.0, pool_size=128, seed=0,
                max_drain_s=60.0):
    """Continuous-batching server under a Poisson stream of decomposition requests: N in
    {3, 4, 5}, entries log-uniform in [1e5, 1e8], ranks ~ U{4..16} per mode, J = 10 max L,
    FP32 TR(N(0,1) cores) + 1e-2 noise, stop at fit change < 1e-4 (cap 30 sweeps), 150 GB
    admission budget. X is materialised in HBM before the stream starts: a pool of
    `pool_size` tensors with shapes from that distribution; request i uses pool entry
    i mod pool_size with its own seed. Latency = scheduled arrival -> result ready."""
    shapes = inputs.serving_requests(pool_size, seed)
    pool = []
    for i, sh in enumerate(shapes):
        X, _ = inputs.tr_plus_noise(sh["dims"], sh["ranks"], seed=10_000 + i, rel_noise=1e-2,
                                    device=dev)
        pool.append((X, sh))
    torch.cuda.synchronize()
    pool_bytes = sum(X.numel() * 4 for X, _ in pool)
    total_s = warmup_s + seconds
    arrivals = [a for a in inputs.poisson_arrivals(int(rate * total_s * 1.5) + 16, rate, seed)
                if a < total_s]
    srv = T.Server(device=dev.index or 0, hbm_budget_bytes=150 << 30, arena_bytes=16 << 30,
                   max_slots=1024, max_modes=5, max_dim=1024, max_rank=16, max_samples=2560,
                   max_sweeps=30, fit_tol=1e-4, X_dtype=T.TR_F32, prec=T.TR_PREC_MIXED)
    srv.start()
    subs = []
    t_start = time.monotonic_ns()
    for i, at in enumerate(arrivals):
        due = t_start + int(at * 1e9)
        now = time.monotonic_ns()
        if due > now:
            time.sleep((due - now) / 1e9)
        X, sh = pool[i % pool_size]
        cores = T.empty_cores(sh["dims"], sh["ranks"], device=dev)
        subs.append((srv.submit(X, sh["ranks"], sh["J"], 1 + i, cores), due, at, sh))
    t_arrivals_end = time.monotonic_ns()
    # Drain for at most max_drain_s after the last arrival; requests still unfinished then
    # are reported as such (an overloaded server would otherwise hold the bench for minutes).
    deadline = t_arrivals_end + int(max_drain_s * 1e9)
    results = []
    unfinished = 0
    for t, due, at, sh in subs:
        left_ms = max(1, (deadline - time.monotonic_ns()) // 1_000_000)
        try:
            res = srv.wait(t, timeout_ms=int(left_ms))
        except T.TrError as e:
            if e.status != T.TR_ERR_TIMEOUT:
                raise
            res = srv.poll(t)
        if res["done"]:
            srv.release(t)
        else:
            unfinished += 1
        results.append((res, due, at, sh))
    t_end = time.monotonic_ns()
    st = srv.stats()
    srv.stop()
    srv.close()
    meas = [(r, due, sh) for r, due, at, sh in results if at >= warmup_s and r["done"]]
    lat = sorted((r["t_done_ns"] - due) / 1e6 for r, due, sh in meas)
    queue = sorted((r["t_admit_ns"] - r["t_submit_ns"]) / 1e6 for r, due, sh in meas)
    # sustained rate: measured requests over the time from the first measured arrival to
    # the last measured completion (includes any backlog drained after the stream ends)
    t0m = t_start + int(warmup_s * 1e9)
    t1m = max((r["t_done_ns"] for r, _, _ in meas), default=t0m + 1)
    win_s = max(seconds, (t1m - t0m) / 1e9)
    in_window = sum(1 for r, _, _ in meas if r["t_done_ns"] <= t0m + int(seconds * 1e9))
    sweeps = [r["sweeps"] for r, _, _ in meas]
    n_upd = sum(r["sweeps"] * len(sh["dims"]) for r, _, sh in meas)
    conv = sum(1 for r, _, _ in meas if r["status"] == T.TR_OK)
    late = max(0.0, (t_arrivals_end - t_start) / 1e9 - total_s)
    return {
        "workload": "Poisson stream, mean 200 req/s, N ~ U{3,4,5}, entries log-uniform in "
                    "[1e5, 1e8], ranks ~ U{4..16}, J = 10 max_k L_k, FP32 TR + 1e-2 noise, "
                    "stop at |fit change| < 1e-4 (cap 30 sweeps), 150 GB HBM budget, mixed "
                    "precision, native worker thread",
        "offered_req_per_s": rate, "seconds": seconds, "warmup_s": warmup_s,
        "requests_measured": len(meas), "requests_total": len(results),
        "unfinished_at_drain_deadline": unfinished, "max_drain_s": max_drain_s,
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 2) if lat else None,
                       "p99": round(float(np.percentile(lat, 99)), 2) if lat else None,
                       "max": round(lat[-1], 2) if lat else None,
                       "what": "scheduled arrival -> end of the tick that finished it"},
        "admission_wait_ms": {"p50": round(float(np.percentile(queue, 50)), 3) if queue else None,
                              "p99": round(float(np.percentile(queue, 99)), 3) if queue else None},
        "throughput_req_per_s": round(len(meas) / win_s, 2),
        "throughput_window_s": round(win_s, 2),
        "completed_in_arrival_window": in_window,
        "sweeps_per_s": round(sum(sweeps) / win_s, 1),
        "updates_per_s": round(n_upd / win_s, 1),
        "sweeps_per_request": {"mean": round(float(np.mean(sweeps)), 2) if sweeps else None,
                               "p50": float(np.percentile(sweeps, 50)) if sweeps else None,
                               "max": max(sweeps) if sweeps else None},
        "converged_fraction": round(conv / max(1, len(meas)), 3),
        "median_fit": round(float(np.median([r["fit"] for r, _, _ in meas])), 5) if meas else None,
        "fit_by_modes": fit_by_modes(meas),
        "singular_updates": int(sum(r["singular_updates"] for r, _, _ in meas)),
        "fit_note": "fit = 1 - relative error after the last sweep; requests near fit 0 are "
                    "ALS stalls from the random N(0,1) start, which the FP64 oracle's stopped "
                    "driver shows on the same shapes (tests/test_gpu_serving_stalls.py)",
        "ticks": st["ticks"], "ms_per_tick": round(st["tick_ns"] / 1e6 / max(1, st["ticks"]), 3),
        "peak_active": st["peak_active"],
        "peak_charged_gb": round(st["peak_charged_bytes"] / 1e9, 3),
        "x_pool": {"tensors": pool_size, "gb": round(pool_bytes / 1e9, 2)},
        "drain_s": round((t_end - t_arrivals_end) / 1e9, 2),
        "arrival_lateness_s": round(late, 3),
    }


def fit_by_modes(meas):
    """Final fits of the measured served requests, grouped by their number of modes N: count,
    quartiles, the fraction at the noise floor (fit > 0.9) and the fraction stalled near
    relative error 1 (fit < 0.1)."""
    out = {}
    for N in (3, 4, 5):
        f = [r["fit"] for r, _, sh in meas if len(sh["dims"]) == N]
        if not f:
            continue
        q = np.percentile(f, [25, 50, 75])
        out[str(N)] = {"requests": len(f), "p25": round(float(q[0]), 4),
                       "p50": round(float(q[1]), 4), "p75": round(float(q[2]), 4),
                       "noise_floor_frac": round(sum(1 for v in f if v > 0.9) / len(f), 3),
                       "stalled_frac": round(sum(1 for v in f if v < 0.1) / len(f), 3)}
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = inputs.WORKLOADS[WORKLOAD]
    X, _ = inputs.tr_plus_noise(wl["dims"], wl["ranks"], seed=wl["seed"],
                                rel_noise=wl["rel_noise"], dtype=torch.float32)
    Xn = X.numpy()
    init = [c.numpy() for c in inputs.random_cores(wl["dims"], wl["ranks"], wl["init_seed"])]
    per_step = []
    total_sweeps = 0
    for k in range(args.warmup + args.steps):
        sw, dt, ncores = oracle_sample(Xn, init, wl, budget_s=4.0, max_sweeps=wl["sweeps"])
        if k >= args.warmup:
            per_step.append(dt)
            total_sweeps += sw
    T = sum(per_step)
    value = total_sweeps / T
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "sweeps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * T / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl),
        "cpu_baseline": {"value": round(value, 4), "unit": "sweeps/s", "cores": ncores,
                         "kind": "oracle",
                         "sample": f"each step: the NumPy FP64 oracle runs whole sweeps of the "
                                   f"same workload (up to {wl['sweeps']}, about 4 s of CPU work)"},
        "e2e": {"value": round(value, 4), "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------------------
# our path
# --------------------------------------------------------------------------------------
def run_ours(args):
    from paper_2010_08581_gb300 import plain_fp64
    from paper_2010_08581_gb300 import trals as T

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    wl = inputs.WORKLOADS[WORKLOAD]
    dims, ranks, J, sweeps = wl["dims"], wl["ranks"], wl["J"], wl["sweeps"]
    N = len(dims)

    # CPU oracle sample first (rank 0, N = 1 only), before any GPU work.
    cpu = None
    X_cpu = None
    init_paper = [c for c in inputs.random_cores(dims, ranks, wl["init_seed"])]
    if rank == 0 and world == 1 and not args.skip_cpu:
        X_cpu, _ = inputs.tr_plus_noise(dims, ranks, seed=wl["seed"], rel_noise=wl["rel_noise"],
                                        dtype=torch.float32)
        sw, dt, ncores = oracle_sample(X_cpu.numpy(), [c.numpy() for c in init_paper], wl,
                                       budget_s=args.cpu_seconds)
        cpu = {"value": round(sw / dt, 4), "unit": "sweeps/s", "cores": ncores, "kind": "oracle",
               "sample": f"{sw} whole sweeps of the same workload by the NumPy FP64 oracle "
                         f"(paper's QR solve), {dt:.1f} s on the host; cores = visible CPUs "
                         "(NumPy's BLAS default thread count)"}
        st = oracle_sample_single_thread(min(10.0, args.cpu_seconds))
        if st:
            cpu["single_thread"] = {
                "value": round(st["sweeps"] / st["seconds"], 4), "unit": "sweeps/s", "cores": 1,
                "sample": f"{st['sweeps']} whole sweeps by the same oracle in a child process "
                          f"with BLAS/OpenMP held to one thread, {st['seconds']:.1f} s"}

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=wl["seed"] + rank, rel_noise=wl["rel_noise"],
                                device=dev, dtype=torch.float32)
    init_dev = [inputs.slice_major(c).to(dev) for c in init_paper]
    ctx = T.Context(local)
    cores = T.empty_cores(dims, ranks, device=dev)
    stream = torch.cuda.current_stream()

    def step(i):
        T.tr_als_sampled(ctx, X, ranks, J, sweeps, wl["sample_seed"] + i, T.TR_PREC_MIXED, cores,
                         init_cores=init_dev)

    clocks = ClockSampler(local)
    clocks.start()
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i in range(args.steps):
        evs[i][0].record(stream)
        step(args.warmup + i)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value = weak_scaling_value(sweeps * args.steps, sum(step_ms) / 1e3, world)
    total_s = world * sweeps * args.steps / value
    fit = T.tr_rel_error(ctx, X, ranks, cores)

    # The same steps again with every kernel bracketed by CUDA events on its stream (the
    # events are nodes of the captured graph); this pass gives the per-kernel times and
    # the roofline, and is kept apart so that its event nodes do not slow the headline.
    T.tr_profile_begin(ctx)
    step(0)                      # re-capture the graph with the event nodes
    T.tr_profile_end(ctx)
    T.tr_profile_begin(ctx)
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pa.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    pb.record(stream)
    torch.cuda.synchronize()
    prof = T.tr_profile_end(ctx)
    profiled_value = sweeps * args.steps / (pa.elapsed_time(pb) / 1e3)

    # end to end through the host entry point: H2D of X and the initial cores, D2H of the
    # resulting cores, every step.
    Xh = X.cpu().pin_memory()
    init_h = [c.cpu().pin_memory() for c in init_dev]
    out_h = [torch.empty(c.shape, dtype=torch.float64).pin_memory() for c in cores]
    e2e_steps = max(1, min(args.steps, 5))
    T.tr_als_sampled_host(ctx, Xh, ranks, J, sweeps, 1, T.TR_PREC_MIXED, out_h, init_h)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for i in range(e2e_steps):
        T.tr_als_sampled_host(ctx, Xh, ranks, J, sweeps, 100 + i, T.TR_PREC_MIXED, out_h, init_h)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = allreduce_max(max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0), world)
    e2e_value = world * sweeps * e2e_steps / e2e_s
    h2d = Xh.numel() * 4 + sum(c.numel() * 8 for c in init_h[1:])
    d2h = sum(c.numel() * 8 for c in out_h)
    # the host link's rate for the same pinned buffer, one plain copy: the end-to-end rate
    # differs from the device rate by about h2d / this per step
    Xcopy = torch.empty_like(X)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        Xcopy.copy_(Xh, non_blocking=True)
        h0.record(stream)
        for _ in range(3):
            Xcopy.copy_(Xh, non_blocking=True)
        h1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = 3 * Xh.numel() * Xh.element_size() / (h0.elapsed_time(h1) / 1e3) / 1e9
    del Xcopy

    # plain FP64 GPU form at the same workload (comparator of the metric)
    fp64 = None
    if not args.skip_fp64:
        init_pl = [c.to(dev) for c in init_paper]
        plain_fp64.als_sampled(X, init_pl, J, 1, 0)       # warm-up
        torch.cuda.synchronize()
        reps = 2
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for r in range(reps):
            res = plain_fp64.als_sampled(X, init_pl, J, sweeps, 1 + r)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        fp64_fit = plain_fp64.rel_error(X, res)
        fp64 = {"value": round(sweeps * reps / sec, 3), "unit": "sweeps/s",
                "final_rel_err": fp64_fit,
                "speedup": round(value / world / (sweeps * reps / sec), 2),
                "equal_fit": abs(fit - fp64_fit) <= 0.01 * fp64_fit}

    # the same decomposition with both factorisations in FP64 (configuration 2 as stated:
    # "FP64 Cholesky plus one refinement step"), same inputs and seeds
    fp64fact = None
    if not args.skip_fp64 and world == 1:
        fp64fact = run_fp64_factorisations(T, X, ranks, J, sweeps, init_dev, wl, stream,
                                           max(1, min(args.steps, 5)), value, fit)

    # uniform sampling (Sec. 5 variant) on the same workload: at the same J and at 5 J (the
    # paper needs several times more uniform samples for the same error)
    uniform = None
    if not args.skip_uniform and world == 1:
        uniform = run_uniform(T, X, ranks, J, sweeps, init_dev, dims, stream,
                              max(1, min(args.steps, 5)))

    dense = None
    if not args.skip_dense and world == 1:
        dense = run_dense(T, X, ranks, sweeps, init_dev, dims, stream,
                          max(1, min(args.steps, 3)), value / world, fit)

    batched = None
    if not args.skip_batched and world == 1:
        batched = run_batched(T, plain_fp64, dev, max(1, min(args.steps, 5)), 1, stream)

    peaks = measured_peaks()
    config1 = config3 = None
    if not args.skip_configs and world == 1:
        config1 = run_config1(T, plain_fp64, dev, stream)
        config3 = run_config3(T, dev, stream, peaks)

    protocol = None
    if args.paper_protocol and world == 1:
        protocol = run_paper_protocol(T, dev)

    serving = None
    if not args.skip_serving and world == 1 and args.serve_seconds > 0:
        serving = run_serving(T, dev, args.serve_seconds)

    roof = roofline(prof, wl, peaks)
    roof_top = rooflines(prof, wl, peaks, 6)
    launches = int(sum(v[1] for v in prof.values()))
    lat = sorted(step_ms)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "sweeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_s * 1e3 / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(wl),
            "final_rel_err": fit,
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                           "p99": round(float(np.percentile(lat, 99)), 4),
                           "what": "one whole decomposition (10 sweeps) per step"},
            "e2e": {"value": round(e2e_value, 3), "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "h2d_gbs": round(h2d_gbs, 1),
                    "h2d_what": "pinned host -> device copy of X alone, CUDA events, 3 copies"},
            "gpu_launches": launches,
            "gpu_launches_note": "kernels of this library launched in the profiled repeat of "
                                 "the timed steps (same work as the timed region)",
            "roofline": roof,
            "rooflines_top": roof_top,
            "profiled_pass": {"value": round(profiled_value, 3), "unit": "sweeps/s",
                              "what": "the timed steps repeated with CUDA events around every "
                                      "kernel; source of kernels_ms and roofline"},
            "kernels_ms": {k: [round(v[0], 4), v[1]] for k, v in
                           sorted(prof.items(), key=lambda kv: -kv[1][0])},
            "fp64_gpu_form": fp64,
            "fp64_factorisations": fp64fact,
            "uniform_sampling": uniform,
            "dense_tr_als": dense,
            "batched_512": batched,
            "config1_fp64_100": config1,
            "config3_cosine_4way": config3,
            "serving": serving,
            "paper_protocol": protocol,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-uniform", action="store_true")
    ap.add_argument("--skip-dense", action="store_true")
    ap.add_argument("--paper-protocol", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-configs", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
