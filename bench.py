"""Benchmark: Gaussian-process log-likelihood + score evaluations per second.

Workload (one "step" = one evaluation of Algorithm 1): n = 262,144 points from
the uniform + 4-cluster mixture (seed 3), Matern 3/2 with
theta = (l 0.05, s2 2, nugget 1e-2), eps_fact 1e-9, eps_peel 1e-6: quadtree,
RSF of Sigma and of dSigma/dl, the solve for the log-likelihood, two peeled
traces and the score.  theta's length scale is perturbed every step
(l * (1 + 1e-3 (i mod 7))) so nothing carries over between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                      [--precision mixed|fp64] [--workload NAME]
Under torchrun each rank runs its own evaluations (independent theta values;
replicas, weak scaling) and rank 0 prints one JSON line.

GPU arm, in order: W warm-up evaluations; K timed evaluations (library
timers off, CUDA events on the launching stream around the whole loop);
one profiled evaluation (the library's per-launch CUDA-event timers on) for
the kernel shares and the roofline; end-to-end evaluations through the
public call with points and z copied from pinned host memory each step (the
same theta sequence, as many of the K as the wall-clock budget allows); one
evaluation of the other precision form at the last timed theta (its time and
the relative differences of loglik, quadratic form and score); the CPU
oracle on small subsamples.

``--impl reference`` times the CPU oracle (the plain fp64 NumPy/SciPy
implementation of the same algorithm) on the host cores: each step is one
evaluation on a bounded sample of the workload (a 2,048-point subsample),
scaled to n = 262,144 with the n^1.5 cost law (Thm. 1; the paper observes
n^1.5 to n^1.6).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1603_08057_gb300 import workloads as WL  # noqa: E402

WORKLOAD = "matern32_mixture_n262144"
METRIC = "loglik+score evals/s at n=262k: plain FP64 vs batched mixed form at 1e-6 rel err"
UNIT = "evals/s"
FORMS = {"mixed": "mixed precision: fp64 IDs, Cholesky/QR factors, log-determinant and rank decisions; "
                  "df64 (fp32-pair) solve and peeling operands multiplied on the tcgen05 tensor cores "
                  "(exact bf16 slices, fp32 accumulation)",
         "mixed_df64": "mixed precision with the solve and peeling products in df64 arithmetic on the CUDA cores",
         "fp64": "plain fp64 RSF + weak peeling"}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
# df64 multiply-add = 12 fp32-pipe instructions (1 mul, 3 fma for the exact
# product, 6 for TwoSum, 2 for the error accumulation); 128 fp32 lanes per SM
DF64_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12
CPU_SIZES = (1024, 2048)        # oracle subsample sizes timed by the CPU leg
CPU_EXPONENT = 1.5              # cost law used to scale them to n (Thm. 1)
WALL_BUDGET_S = 1500.0          # the e2e loop shrinks to keep the run inside this


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(WL.WORKLOADS))
    p.add_argument("--n", type=int, default=None, help="override the point count (testing)")
    p.add_argument("--tol-peel", type=float, default=None, help="override the workload's eps_peel")
    p.add_argument("--mle", action="store_true",
                   help="instead of the benchmark: the full-MLE workload's L-BFGS fit (Matern nu=1, mixture points, "
                        "data drawn at theta (0.05, 1, 1e-2), started from (0.2, 0.5, 0.1)) at --n points "
                        "(default 65,536) for --mle-iters iterations")
    p.add_argument("--mle-iters", type=int, default=30)
    p.add_argument("--mle-staged", action="store_true",
                   help="with --mle: tighten the tolerances over three stages (mle.fit_staged) instead of "
                        "running all iterations at eps_fact 1e-9, eps_peel 1e-6")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-other-form", action="store_true",
                   help="skip the evaluation in the other precision form")
    p.add_argument("--budget-s", type=float, default=WALL_BUDGET_S,
                   help="wall-clock budget of the whole run; the e2e loop runs as many of the K steps as fit")
    p.add_argument("--precision", default="mixed", choices=["mixed", "mixed_df64", "fp64"],
                   help="mixed (default): fp64 IDs, Cholesky/QR factors and log-determinant, solve and "
                        "peeling products on the tensor cores; mixed_df64: those products in df64 on the "
                        "CUDA cores; fp64: every step in fp64 (the plain form)")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(ms_local: float, steps: int, device=None) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: every rank ran `steps`
    evaluations in `ms_local` ms; the job time is the max over ranks (needs an
    initialised process group when WORLD_SIZE > 1).  Returns (evals/s, max ms)."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ws * steps / (ms_max / 1e3), ms_max


FAMILY_NAMES = {WL.MATERN12: "matern12 nu=1/2", WL.MATERN32: "matern32 nu=3/2", WL.MATERN52: "matern52 nu=5/2",
                WL.RQ: "rational quadratic"}


def workload_config(name, n=None):
    wl = dict(WL.WORKLOADS[name])
    n = n or wl["n"]
    pts = {"mixture": "uniform+4 clusters (sigma 0.03)", "uniform": "uniform in [0,1]^2",
           "grid": "sqrt(n) x sqrt(n) grid of [0,100]^2, anisotropic theta = (l1, s2, nug, l2)"}[wl["points"]]
    fam = FAMILY_NAMES[wl["family"]] + (f" alpha={wl['alpha']:g}" if wl["family"] == WL.RQ else "")
    return wl, {"workload": f"{fam} {wl['points']} n={n}", "n": n, "points": pts,
                "theta": list(wl["theta"]), "tol_fact": wl["tol_fact"], "tol_peel": wl["tol_peel"],
                "n_occ": 64, "n_prox": 256, "l2": "inputs and factors exceed the 126 MB L2 (no flush needed)"}


def theta_at(th0, i):
    return (th0[0] * (1 + 1e-3 * (i % 7)),) + tuple(th0[1:])


# --------------------------------------------------------------- CPU oracle
def cpu_oracle_eval(x, z, theta, wl):
    from oracle import mle
    t0 = time.perf_counter()
    mle.loglik_and_score(x, z, wl["family"], theta, wl["tol_fact"], wl["tol_peel"], wl["alpha"])
    return time.perf_counter() - t0


def cpu_sample(wl, m, seed=4):
    from oracle import dense
    x_full = WL.make_points(wl["points"], wl["n"], wl["seed_points"])
    xs, _ = WL.subsample(x_full, m, seed)
    z = dense.sample_z_dense(xs, wl["family"], wl["theta"], WL.standard_normal(m, wl["seed_z"]), wl["alpha"])
    return xs, z


def cpu_leg(wl, n):
    """The oracle timed on subsamples of CPU_SIZES points: evals/s scaled to n
    with the n^1.5 law, plus the exponent fitted between the two sizes."""
    times = []
    for m in CPU_SIZES:
        xs, zs = cpu_sample(wl, m)
        times.append(cpu_oracle_eval(xs, zs, wl["theta"], wl))
    m1, m2 = CPU_SIZES
    t1, t2 = times
    p_fit = float(np.log(t2 / t1) / np.log(m2 / m1))
    value = 1.0 / (t2 * (n / m2) ** CPU_EXPONENT)
    sample = (f"oracle Algorithm 1 (NumPy/SciPy fp64) timed on {m1}- and {m2}-point subsamples "
              f"({t1:.1f} s, {t2:.1f} s; local exponent {p_fit:.2f}); the {m2}-point time scaled to "
              f"n={n} by (n/{m2})^{CPU_EXPONENT} (Thm. 1; the paper observes n^1.5-1.6)")
    return {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
            "largest_n_timed": m2, "seconds": dict(zip([str(m) for m in CPU_SIZES], times)),
            "fitted_exponent": p_fit, "scaling_exponent": CPU_EXPONENT}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl, cfg = workload_config(args.workload, args.n)
    m = CPU_SIZES[-1]
    xs, z = cpu_sample(wl, m)
    th0 = wl["theta"]
    for i in range(args.warmup):
        cpu_oracle_eval(xs, z, theta_at(th0, i), wl)
    ts = []
    for i in range(args.steps):
        ts.append(cpu_oracle_eval(xs, z, theta_at(th0, i), wl))
    t = statistics.median(ts)
    v = 1.0 / (t * (cfg["n"] / m) ** CPU_EXPONENT)
    cores = os.cpu_count()
    sample = (f"oracle Algorithm 1 on a {m}-point subsample (median {t:.1f} s per step), "
              f"scaled by (n/{m})^{CPU_EXPONENT}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, parallelism=f"host cores x{cores} (rank 0)",
                           form="CPU oracle: plain fp64 NumPy/SciPy RSF + weak peeling"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
TC_SLICES = 7
TC_PRODUCTS = TC_SLICES * (TC_SLICES + 1) // 2   # slice products with s + t < 7


def measured_peaks():
    """MEASURED_PEAKS.json (driver-written, the GB300s) or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def bf16_peak_tflops():
    """Dense bf16 tensor peak (sustained, for a kernel timed inside a long
    step) and where it comes from."""
    mp = measured_peaks()
    if mp:
        for key in ("bf16_tflops_sustained", "bf16_tflops"):
            if isinstance(mp.get(key), (int, float)) and mp[key] > 0:
                return float(mp[key]), f"MEASURED_PEAKS.json {key} (of measured)"
    return 1700.0, "profiling recipe fallback: 1.7 PFLOP/s bf16 sustained (of fallback)"


def roofline_of(B, prof, ms_prof):
    """Roofline of the GEMM engine that took the most time in the profiled
    evaluation: achieved = its algorithmic (fp64-equivalent, 2 M N K per
    descriptor) flops / its summed CUDA-event time."""
    cands = [(prof[B.PROF_GEMM_TC], "tc"), (prof[B.PROF_GEMM_DF], "df"), (prof[B.PROF_GEMM], "fp64")]
    g, kind = max(cands, key=lambda c: c[0]["ms"])
    achieved = g["flops"] / (g["ms"] / 1e3) / 1e12 if g["ms"] > 0 else None
    extra = {}
    if kind == "tc":
        bf16, src = bf16_peak_tflops()
        kname = "tc_slice_kernel + tc_gemm_pre_kernel (batched ragged GEMM on tcgen05, df64 operands pre-sliced into exact bf16 slices)"
        bound, peak = "tensor", bf16 / TC_PRODUCTS
        psrc = (f"dense bf16 tensor peak {bf16:.0f} TFLOP/s from {src}, divided by the {TC_PRODUCTS} bf16 slice "
                f"multiply-adds ({TC_SLICES} slices per operand, products with s + t < {TC_SLICES}) that make one "
                "fp64-class multiply-add")
        extra = {"bf16_peak": bf16, "bf16_slice_flops_per_fp64_flop": TC_PRODUCTS}
    elif kind == "df":
        kname = "gemm_kernel<true> (batched ragged GEMM, df64 arithmetic)"
        bound, peak = "alu", DF64_PEAK_TFLOPS
        psrc = ("df64 on the fp32 pipe: 152 SMs x 128 lanes x 2.07 GHz / 12 instructions per multiply-add "
                "x 2 flop (recipe unit counts and clock)")
    else:
        kname = "gemm_kernel<false> (batched ragged GEMM, fp64)"
        bound, peak = "alu", FP64_PEAK_TFLOPS
        psrc = "fp64 ALU: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (recipe unit counts and clock)"
    r = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
         "frac": (achieved / peak) if achieved else None, "traffic": None, "peak_source": psrc,
         "flops_counted": "2 per multiply-add of each GEMM descriptor (M N K, triangular operands and "
                          "lower-triangle outputs counted exactly), fp64-equivalent",
         "measured_on": "one profiled evaluation after the timed loop (per-launch CUDA events on the "
                        "launching stream)",
         "launches": g["launches"], "kernel_ms": g["ms"], "profiled_eval_ms": ms_prof,
         "share_of_step": g["ms"] / ms_prof if ms_prof > 0 else None,
         "phases_ms": {B.PROF_NAMES[c]: prof[c]["ms"] for c in prof if prof[c]["launches"] > 0}}
    r.update(extra)
    r["engines"] = engine_rooflines(B, prof)
    return r


def engine_rooflines(B, prof):
    """Every GEMM engine that ran in the profiled evaluation against its own
    bound (the tensor-core engine against the bf16 peak / 28, the CUDA-core
    engines against their derived ALU peaks), and the flop-weighted total of
    the three: their summed algorithmic flops over their summed time."""
    bf16, _ = bf16_peak_tflops()
    rows = []
    tot_fl = tot_ms = 0.0
    for cat, name, peak in ((B.PROF_GEMM_TC, "tensor-core GEMM (slicing + products)", bf16 / TC_PRODUCTS),
                            (B.PROF_GEMM_DF, "df64 CUDA-core GEMM", DF64_PEAK_TFLOPS),
                            (B.PROF_GEMM, "fp64 GEMM", FP64_PEAK_TFLOPS)):
        g = prof.get(cat)
        if not g or g["launches"] <= 0 or g["ms"] <= 0:
            continue
        tf = g["flops"] / (g["ms"] / 1e3) / 1e12
        rows.append({"engine": name, "launches": g["launches"], "ms": g["ms"], "achieved_tflops": tf,
                     "peak_tflops": peak, "frac": tf / peak})
        tot_fl += g["flops"]
        tot_ms += g["ms"]
    total = {"achieved_tflops": tot_fl / (tot_ms / 1e3) / 1e12, "ms": tot_ms} if tot_ms > 0 else None
    return {"per_engine": rows, "flop_weighted_total": total}


def rel(a, b):
    return float(abs(a - b) / max(abs(b), 1e-300))


def run_gpu(args):
    import torch
    t_start = time.perf_counter()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1603_08057_gb300 import build
    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    from paper_1603_08057_gb300 import binding as B

    wl, cfg = workload_config(args.workload, args.n)
    if args.tol_peel:
        wl["tol_peel"] = cfg["tol_peel"] = args.tol_peel
    n = cfg["n"]
    fam, alpha = wl["family"], wl["alpha"]
    x = WL.make_points(wl["points"], n, wl["seed_points"])
    th0 = wl["theta"]
    pts = torch.tensor(x, dtype=torch.float64, device="cuda")
    # z ~ N(0, Sigma) through F^1/2 (Sec. 2.3.2) of a tight fp64 factorization
    F = B.Factorization(pts, fam, th0, B.SIGMA, 1e-12, alpha, B.opts(precision=B.PREC_FP64))
    w = torch.tensor(WL.standard_normal(n, wl["seed_z"]), dtype=torch.float64, device="cuda")
    z = F.solve(w, B.OP_SQRT)
    del F
    torch.cuda.synchronize()

    forms = {"mixed": B.PREC_MIXED, "mixed_df64": B.PREC_MIXED_DF64, "fp64": B.PREC_FP64}
    o = B.opts(precision=forms[args.precision])

    def step(i, opts=o, p=pts, zz=z):
        return B.loglik_and_score(p, zz, fam, theta_at(th0, i), wl["tol_fact"], wl["tol_peel"], alpha, opts)

    for i in range(args.warmup):
        step(i)
    stream = torch.cuda.current_stream()
    B.profile(False)
    B.launch_count(reset=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    t_timed0 = time.perf_counter()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for i in range(args.steps):
            results.append(step(i))
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    t_step_wall = (time.perf_counter() - t_timed0) / max(1, args.steps)
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = B.launch_count(reset=True)
    value, ms_max = replica_throughput(ms, args.steps, device="cuda")

    # one profiled evaluation: per-launch CUDA events of the library's GEMM
    # and QR launches and of its phases, for the kernel shares and roofline
    B.profile(True)
    for c in range(len(B.PROF_NAMES)):
        B.profile_read(c, reset=True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    step(args.steps - 1)
    pe1.record(stream)
    torch.cuda.synchronize()
    ms_prof = pe0.elapsed_time(pe1)
    prof = {c: B.profile_read(c, reset=True) for c in range(len(B.PROF_NAMES))}
    B.profile(False)

    # the other precision form at the last timed theta: its time and the
    # relative differences of loglik, quadratic form and score components
    other = None
    if not args.no_other_form:
        oname = "fp64" if args.precision != "fp64" else "mixed"
        oo = B.opts(precision=forms[oname])
        torch.cuda.synchronize()
        oe0, oe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        oe0.record(stream)
        ll_o, g_o, t_o = step(args.steps - 1, oo)
        oe1.record(stream)
        torch.cuda.synchronize()
        ms_o = oe0.elapsed_time(oe1)
        ll_m, g_m, t_m = results[-1]
        ref = (ll_o, g_o.numpy(), t_o.numpy()) if oname == "fp64" else (ll_m, g_m.numpy(), t_m.numpy())
        cmp_ = (ll_m, g_m.numpy(), t_m.numpy()) if oname == "fp64" else (ll_o, g_o.numpy(), t_o.numpy())
        p = len(th0)
        scale = 0.5 * np.abs(ref[2][:p]) + 0.5 * np.abs(ref[2][p:])
        g_rel = [rel(a, b) for a, b in zip(cmp_[1], ref[1])]
        g_scl = [float(abs(a - b) / s) for a, b, s in zip(cmp_[1], ref[1], scale)]
        other = {"form": oname, "steps": 1, "value": 1e3 / ms_o, "unit": UNIT, "ms_per_step": ms_o,
                 "theta": list(theta_at(th0, args.steps - 1)),
                 "mixed_vs_fp64": {"loglik_rel": rel(cmp_[0], ref[0]),
                                   "score_rel": g_rel, "score_rel_term_scale": g_scl,
                                   "quad_terms_rel": [rel(a, b) for a, b in zip(cmp_[2][:p], ref[2][:p])],
                                   "trace_terms_rel": [rel(a, b) for a, b in zip(cmp_[2][p:], ref[2][p:])],
                                   "gates": {"loglik_1e-6": rel(cmp_[0], ref[0]) <= 1e-6,
                                             "score_1e-3": all(e <= 1e-3 for e in g_rel)}}}

    # end to end through the public API with host buffers: H2D of points and
    # z every step, the call, D2H of the log-likelihood and score
    e2e = None
    if not args.no_e2e:
        hp = torch.tensor(x, dtype=torch.float64).pin_memory()
        hz = z.cpu().pin_memory()
        dp = torch.empty_like(pts)
        dz = torch.empty_like(z)
        reserve = 30.0 if args.no_cpu else 60.0
        left = args.budget_s - (time.perf_counter() - t_start) - reserve
        k_e2e = max(1, min(args.steps, int(left / max(t_step_wall, 1e-3))))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(k_e2e):
            dp.copy_(hp, non_blocking=True)
            dz.copy_(hz, non_blocking=True)
            step(i, o, dp, dz)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": k_e2e / te, "unit": UNIT, "h2d_bytes_per_step": int(hp.numel() * 8 + hz.numel() * 8),
               "d2h_bytes_per_step": (1 + 3 * len(th0)) * 8, "steps": k_e2e,
               "theta": "the first %d of the timed steps' theta values" % k_e2e}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    roofline = roofline_of(B, prof, ms_prof)
    cpu = None if args.no_cpu else cpu_leg(wl, n)
    ll, gsc, terms = results[-1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+df64",
            "data": "synthetic",
            "config": dict(cfg, parallelism=f"replicas x{ws}", form=FORMS[args.precision],
                           library_timers="off in the timed loop"),
            "clocks": clk.summary(), "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "other_form": other,
            "last_eval": {"loglik": ll, "score": gsc.tolist(), "terms": terms.tolist()},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_mle(args):
    """The MLE loop of the full-MLE workload on one GPU: one JSON line with the
    wall time per L-BFGS iteration and the error of the fitted theta."""
    import torch
    from paper_1603_08057_gb300 import build
    build.build()
    from paper_1603_08057_gb300 import binding as B
    from paper_1603_08057_gb300 import mle
    n = args.n or 65536
    th_true, th0 = (0.05, 1.0, 1e-2), (0.2, 0.5, 0.1)
    pts = torch.tensor(WL.mixture(n, 9), dtype=torch.float64, device="cuda")
    F = B.Factorization(pts, B.MATERN1, th_true, B.SIGMA, 1e-12, 0.0, B.opts(precision=B.PREC_FP64))
    z = F.solve(torch.tensor(WL.standard_normal(n, 10), dtype=torch.float64, device="cuda"), B.OP_SQRT)
    del F
    torch.cuda.synchronize()
    if args.mle_staged:
        th, info = mle.fit_staged(pts, z, B.MATERN1, th0)
        info["trace"] = [t for st in info["stages"] for t in st["trace"]]
    else:
        th, info = mle.fit(pts, z, B.MATERN1, th0, max_iter=args.mle_iters)
    iters = len({tuple(t[0]) for t in info["trace"]})
    line = {"mode": "mle", "workload": f"matern nu=1 mixture n={n}", "n": n, "theta_true": list(th_true),
            "theta0": list(th0), "theta_hat": th, "theta_rel_err": [abs(a - b) / b for a, b in zip(th, th_true)],
            "lbfgs_max_iter": args.mle_iters, "evaluations": info["evals"], "seconds": info["seconds"],
            "s_per_evaluation": info["seconds"] / max(1, info["evals"]), "distinct_thetas": iters,
            "final_loglik": info["loglik"], "final_score": info["trace"][-1][2] if info["trace"] else None,
            "tolerance_stages": ([(st["tol_fact"], st["tol_peel"], st["evals"]) for st in info["stages"]]
                                 if args.mle_staged else None)}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.mle:
        return run_mle(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
