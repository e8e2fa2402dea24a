"""Benchmark: Gaussian-process log-likelihood + score evaluations per second.

Workload (one "step" = one evaluation of Algorithm 1): n = 262,144 points from
the uniform + 4-cluster mixture (seed 3), Matern 3/2 with
theta = (l 0.05, s2 2, nugget 1e-2), eps_fact 1e-9, eps_peel 1e-6: quadtree,
RSF of Sigma and of dSigma/dl, the solve for the log-likelihood, two peeled
traces and the score.  theta's length scale is perturbed every step
(l * (1 + 1e-3 i)) so nothing carries over between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                      [--precision mixed|fp64]
Under torchrun each rank runs its own evaluations (independent theta values;
replicas, weak scaling) and rank 0 prints one JSON line.

``--impl reference`` times the CPU oracle (the plain fp64 NumPy/SciPy
implementation of the same algorithm) on the host cores: each step is one
evaluation on a bounded sample of the workload (a 2,048-point subsample),
scaled to n = 262,144 with the O(n^1.5) cost law of Sec. 2.3.3 / Thm. 1.
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
                  "df64 (fp32-pair) multi-RHS solves and peeling GEMMs",
         "fp64": "plain fp64 RSF + weak peeling"}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
# df64 multiply-add = 12 fp32-pipe instructions (1 mul, 3 fma for the exact
# product, 6 for TwoSum, 2 for the error accumulation); 128 fp32 lanes per SM
DF64_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12
CPU_SAMPLE_N = 2048


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=None, help="override the point count (testing)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                   help="mixed (default): fp64 IDs, Cholesky/QR factors and log-determinant, df64 "
                        "solves and peeling GEMMs; fp64: every step in fp64 (the plain form)")
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


def workload_config(n):
    wl = WL.WORKLOADS[WORKLOAD]
    return wl, {"workload": f"matern32 nu=3/2 mixture n={n}", "n": n, "points": "uniform+4 clusters (sigma 0.03)",
                "theta": list(wl["theta"]), "tol_fact": wl["tol_fact"], "tol_peel": wl["tol_peel"],
                "n_occ": 64, "n_prox": 256, "l2": "inputs and factors exceed the 126 MB L2 (no flush needed)"}


# --------------------------------------------------------------- CPU oracle
def cpu_oracle_eval(x, z, theta, wl):
    from oracle import mle
    t0 = time.perf_counter()
    mle.loglik_and_score(x, z, 1, theta, wl["tol_fact"], wl["tol_peel"])
    return time.perf_counter() - t0


def cpu_sample(wl, seed=4):
    from oracle import dense
    x_full = WL.mixture(wl["n"], wl["seed_points"])
    xs, _ = WL.subsample(x_full, CPU_SAMPLE_N, seed)
    z = dense.sample_z_dense(xs, 1, wl["theta"], WL.standard_normal(CPU_SAMPLE_N, wl["seed_z"]))
    return xs, z


def cpu_scale(t_sample, n):
    """evals/s at n from one sample evaluation at CPU_SAMPLE_N, O(n^1.5)."""
    return 1.0 / (t_sample * (n / CPU_SAMPLE_N) ** 1.5)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl, cfg = workload_config(args.n or WL.WORKLOADS[WORKLOAD]["n"])
    xs, z = cpu_sample(wl)
    th0 = wl["theta"]
    for i in range(args.warmup):
        cpu_oracle_eval(xs, z, (th0[0] * (1 + 1e-3 * i), th0[1], th0[2]), wl)
    ts = []
    for i in range(args.steps):
        ts.append(cpu_oracle_eval(xs, z, (th0[0] * (1 + 1e-3 * i), th0[1], th0[2]), wl))
    t = statistics.median(ts)
    v = cpu_scale(t, cfg["n"])
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, parallelism=f"host cores x{cores} (rank 0)",
                           form="CPU oracle: plain fp64 NumPy/SciPy RSF + weak peeling"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"oracle Algorithm 1 on a {CPU_SAMPLE_N}-point subsample, scaled by (n/{CPU_SAMPLE_N})^1.5"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
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

    wl, cfg = workload_config(args.n or WL.WORKLOADS[WORKLOAD]["n"])
    n = cfg["n"]
    x = WL.mixture(n, wl["seed_points"])
    th0 = wl["theta"]
    pts = torch.tensor(x, dtype=torch.float64, device="cuda")
    # z ~ N(0, Sigma) through F^1/2 (Sec. 2.3.2) of a tight factorization
    F = B.Factorization(pts, B.MATERN32, th0, B.SIGMA, 1e-12)
    w = torch.tensor(WL.standard_normal(n, wl["seed_z"]), dtype=torch.float64, device="cuda")
    z = F.solve(w, B.OP_SQRT)
    del F
    torch.cuda.synchronize()

    def theta(i):
        return (th0[0] * (1 + 1e-3 * (i % 7)), th0[1], th0[2])

    o = B.opts(precision=B.PREC_MIXED if args.precision == "mixed" else B.PREC_FP64)

    def step(i):
        return B.loglik_and_score(pts, z, B.MATERN32, theta(i), wl["tol_fact"], wl["tol_peel"], 0.0, o)

    for i in range(args.warmup):
        step(i)
    stream = torch.cuda.current_stream()
    B.profile(True)
    for c in range(len(B.PROF_NAMES)):
        B.profile_read(c, reset=True)
    B.launch_count(reset=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for i in range(args.steps):
            results.append(step(i))
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = B.launch_count(reset=True)
    prof = {c: B.profile_read(c, reset=True) for c in range(len(B.PROF_NAMES))}
    B.profile(False)
    value, ms_max = replica_throughput(ms, args.steps, device="cuda")

    # end to end through the public API with host buffers: H2D of points and
    # z every step, the call, D2H of the log-likelihood and score
    e2e = None
    if not args.no_e2e:
        hp = torch.tensor(x, dtype=torch.float64).pin_memory()
        hz = z.cpu().pin_memory()
        dp = torch.empty_like(pts)
        dz = torch.empty_like(z)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(max(1, min(args.steps, 1))):
            dp.copy_(hp, non_blocking=True)
            dz.copy_(hz, non_blocking=True)
            B.loglik_and_score(dp, dz, B.MATERN32, theta(i), wl["tol_fact"], wl["tol_peel"], 0.0, o)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": max(1, min(args.steps, 1)) / te, "unit": UNIT, "h2d_bytes_per_step": int(hp.numel() * 8 + hz.numel() * 8),
               "d2h_bytes_per_step": 4 * 8}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    gdf, g64 = prof[B.PROF_GEMM_DF], prof[B.PROF_GEMM]
    if gdf["ms"] >= g64["ms"]:
        g, kname, peak = gdf, "gemm_kernel<true> (batched ragged GEMM, df64 arithmetic)", DF64_PEAK_TFLOPS
        psrc = ("df64 on the fp32 pipe: 152 SMs x 128 lanes x 2.07 GHz / 12 instructions per multiply-add "
                "x 2 flop (recipe unit counts and clock)")
    else:
        g, kname, peak = g64, "gemm_kernel<false> (batched ragged GEMM, fp64)", FP64_PEAK_TFLOPS
        psrc = "fp64 ALU: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (recipe unit counts and clock)"
    achieved = g["flops"] / (g["ms"] / 1e3) / 1e12 if g["ms"] > 0 else None
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None, "peak_source": psrc,
                "flops_counted": "2 per multiply-add of each GEMM descriptor (M N K, triangular operands and "
                                 "lower-triangle outputs counted exactly), fp64-equivalent",
                "launches": g["launches"], "kernel_ms_per_step": g["ms"] / args.steps,
                "share_of_step": g["ms"] / ms if ms > 0 else None,
                "phases_ms_per_step": {B.PROF_NAMES[c]: prof[c]["ms"] / args.steps for c in prof
                                       if prof[c]["launches"] > 0}}
    cpu = None
    if not args.no_cpu:
        xs, zs = cpu_sample(wl)
        ts = cpu_oracle_eval(xs, zs, th0, wl)
        vcpu = cpu_scale(ts, n)
        cpu = {"value": vcpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle Algorithm 1 on a {CPU_SAMPLE_N}-point subsample ({ts:.1f} s), scaled by (n/{CPU_SAMPLE_N})^1.5"}
    ll, gsc, terms = results[-1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+df64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": dict(cfg, parallelism=f"replicas x{ws}", form=FORMS[args.precision]),
            "clocks": clk.summary(), "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "last_eval": {"loglik": ll, "score": gsc.tolist(), "terms": terms.tolist()}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
