#!/usr/bin/env python
"""Benchmark: TFLOP/s of mixed-precision LU and Cholesky solves refined to
1e-14 backward error at N = 32768 on one GB300, next to this project's FP64
path and the CPU oracle.

One step = cf_gesv_mixed (LU with tournament pivoting at v = 64, leaves of
512 rows, arity 8; FP16 tensor-core Schur updates with FP32 accumulation;
FP64-accurate refinement with residuals on the tensor cores; A = U[-1,1] +
2 sqrt(N) I, 16 right-hand sides) + cf_posv_mixed (Cholesky, FP16 updates,
the same refinement; A = G G^T / N + alpha I with kappa ~ 1e2, 8 right-hand
sides).  Each system takes the update precision with which it is solved
fastest (measured: FP16 for both; BF16 needs more refinement steps, split
BF16 (hi + lo operands, three products) costs more to factor than the steps
it saves now that a refinement step is cheap; the others run as variants).
value = (2N^3/3 + N^3/3) / step time.  A step counts only if every
right-hand side reaches eta <= 1e-14 (checked here with an FP64 residual).
--prec / --chol-prec choose the precisions; by default the other BF16, FP16
and split-BF16 solves, the unshifted LU (s = 0) and the N = 65536 Cholesky
with FP8 updates run once after the timed step ("variants").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cf|reference]

For N > 1 (torchrun) every rank solves its own replica (the factorization
of one matrix does not shard): value = flops of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TFLOP/s for LU/Cholesky at N=32768, mixed+refine vs FP64, at 1e-14 backward err"
UNIT = "TFLOP/s"
TOL = 1e-14
SOLVER_TOL = 0.9e-14   # asked of the solver: a 10% margin for the independent FP64 check at TOL
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal; ~2 DFMA/clk/SM x 152 SMs x 2.07 GHz)
RESID_TRAFFIC_8192 = 542.2e6   # k_residual_f64 DRAM bytes per launch at N = 8192 (ncu)
# FP32 tournament DRAM bytes per launch, averaged over an LU's panels, keyed
# by (N, v, leaf_h, arity), from ncu captures under profiles/
# (profiles/k_tourn32w_n32768.md: the launch reads exactly its panel, m x 64 x 4 bytes)
TOURN_TRAFFIC = {(32768, 64, 512, 8): sum(4.0 * 64 * (32768 - 64 * i) for i in range(512)) / 512}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cf", "reference"], default="cf")
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--chol-prec", default="f16", choices=["bf16", "f16", "bf16x3"],
                    help="update precision of the timed Cholesky solve")
    ap.add_argument("--prec", default="f16", choices=["bf16", "f16", "bf16x3"],
                    help="update precision of the timed step (the other 16-bit one runs once as a variant)")
    ap.add_argument("--v", type=int, default=64, help="block size of the mixed LU's steps")
    ap.add_argument("--leaf-h", type=int, default=512, help="tournament leaf height of the mixed LU")
    ap.add_argument("--arity", type=int, default=8, help="children per playoff node of the mixed LU's tournament")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    ap.add_argument("--fp64-sizes", default="8192,16384,32768",
                    help="sizes of the FP64 path at paper-like sizes (config 2); empty to skip")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the once-run legs (FP16, s = 0 LU, FP8 Cholesky at N = 65536)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                     "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5).stdout
                parts = [p.strip() for p in out.strip().split(",")]
                if len(parts) >= 8:
                    self.samples.append(parts)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for nm, v in zip(names, s[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ------------------------------------------------------------------ ranks
def _reduce_over_ranks(x: float, world: int, device, op: str = "max") -> float:
    """Max (or min) of a host scalar over the ranks of the default process
    group (NCCL on GPUs, gloo on the CPU); x itself for a single rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.MIN)
    return float(t.item())


# two-sided 95% Student t quantiles for 1..10 degrees of freedom (1.96 beyond)
_T95 = (12.706, 4.303, 3.182, 2.776, 2.571, 2.447, 2.365, 2.306, 2.262, 2.228)


def _step_stats(ms):
    """Median, min, max and mean of the per-step times with the 95%
    confidence half-width of the mean (Student t; None for one step)."""
    k = len(ms)
    mean = statistics.fmean(ms)
    ci = None
    if k > 1:
        t = _T95[k - 2] if k - 1 <= len(_T95) else 1.96
        ci = t * statistics.stdev(ms) / math.sqrt(k)
    return {"median_ms": statistics.median(ms), "min_ms": min(ms), "max_ms": max(ms), "mean_ms": mean,
            "ci95_mean_ms": ci, "steps": k}


def _lpt_shards(costs, world: int):
    """Longest-processing-time partition of independent jobs over `world`
    ranks: jobs in decreasing cost, each to the least-loaded rank (ties to the
    lowest rank).  Returns one list of job indices per rank."""
    import heapq
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return shards


def _job_tflops(world: int, flops_per_rank: float, ms_per_step: float) -> float:
    """Whole-job rate of `world` replicas, each doing flops_per_rank per step,
    timed by the slowest rank's ms_per_step."""
    return world * flops_per_rank / (ms_per_step * 1e-3) / 1e12


# ------------------------------------------------------------------ oracle
def _host_cpu(cpuinfo: str = "/proc/cpuinfo") -> str:
    """The host CPU as /proc/cpuinfo names it (x86 'model name'; on Arm the
    implementer / part codes), with the logical CPU count."""
    import platform
    name = None
    try:
        fields = {}
        for line in open(cpuinfo):
            if ":" in line:
                k, v = (x.strip() for x in line.split(":", 1))
                fields.setdefault(k, v)
        name = fields.get("model name") or fields.get("Model") or (
            "Arm implementer %s part %s" % (fields["CPU implementer"], fields["CPU part"])
            if "CPU implementer" in fields and "CPU part" in fields else None)
    except OSError:
        pass
    return "%s, %d logical CPUs" % (name or platform.machine(), os.cpu_count() or 1)


def _oracle_sample(n_sample: int, v: int = 64, h: int = 512, arity: int = 8):
    """The FP64 oracle as it stands on this host's cores: LU (the mixed LU's
    tournament shape: v = 64, leaves of 512 rows, arity 8) and Cholesky at
    n_sample with the same generators.  Returns (TFLOP/s, seconds, threads)."""
    import oracle
    from paper_2108_09337_gb300 import inputs
    A = inputs.uniform_pm1(n_sample, seed=0, shift=2 * math.sqrt(n_sample))
    S = inputs.spd_gram(n_sample, seed=1)
    t0 = time.perf_counter()
    oracle.getrf(A, v=v, h=h, arity=arity)
    oracle.potrf(S)
    dt = time.perf_counter() - t0
    fl = oracle.lu_flops(n_sample) + oracle.chol_flops(n_sample)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return fl / dt / 1e12, dt, threads


def run_reference(args, rank: int):
    """--impl reference: the oracle, timed on the host cores, each step a
    bounded sample (N = 2048 LU + Cholesky) of the benchmark workload."""
    if rank != 0:
        return
    n_s = 2048
    for _ in range(args.warmup):
        _oracle_sample(n_s, args.v, args.leaf_h, args.arity)
    times, rates = [], []
    for _ in range(args.steps):
        r, dt, threads = _oracle_sample(n_s, args.v, args.leaf_h, args.arity)
        times.append(dt)
        rates.append(r)
    value = statistics.median(rates)
    sample = ("oracle LU (tournament, v=%d, h=%d, arity %d) + Cholesky at N=%d per step, same generators"
              % (args.v, args.leaf_h, args.arity, n_s))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "CPU oracle sample of the N=32768 LU/Cholesky workload", "n_sample": n_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "host": _host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def _tourn_kw(args):
    """Block size and tournament shape of the mixed LU (v, leaf height, arity)."""
    return {"v": args.v, "leaf_h": args.leaf_h, "arity": args.arity}


def _gen_inputs(n, device):
    from paper_2108_09337_gb300 import inputs
    A_lu = inputs.uniform_pm1_torch(n, seed=0, shift=2.0 * math.sqrt(n), device=device)
    B_lu = inputs.rhs_normal_torch(n, 16, seed=3, device=device)
    A_ch = inputs.spd_gram_torch(n, seed=1, alpha=0.0, device=device)
    # alpha = lambda_max / (kappa - 1), kappa = 1e2; lambda_max by power iteration
    alpha, lam = inputs.shift_to_kappa_torch(A_ch, 1e2)
    B_ch = inputs.rhs_normal_torch(n, 8, seed=4, device=device)
    return A_lu, B_lu, A_ch, B_ch, {"lambda_max_est": lam, "alpha": alpha}


def _timed(fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def _run_variants(args, n, dev, A_lu, B_lu, A_ch, B_ch, rank=0, world=1):
    """One timed run each of the configurations the headline does not cover:
    the other 16-bit and the split-BF16 updates at N = 32768 (LU and
    Cholesky); the unshifted
    LU (s = 0) with split BF16, BF16 and FP16 updates (GMRES-IR; BF16 / FP16
    escalate to split BF16); Cholesky at N = 65536 with FP8 e4m3 updates and
    per-tile scales, kappa = 1e2 and 1e4; the 20,000-matrix batched
    configuration.  Every result is checked with an independent FP64
    residual (the batched one by the solver's own per-matrix FP64 eta)."""
    import torch
    from paper_2108_09337_gb300 import cf, inputs
    out = {}

    def rec(name, fn, A, B, fl):
        (X, info, S, st), ms = _timed(fn)
        d = S.as_dict()
        out[name] = {"ms": ms, "tflops": fl / (ms * 1e-3) / 1e12, "status": int(st),
                     "eta": _eta(A, X, B), "iterations": d["iterations"], "solver": d["solver"],
                     "gmres_iterations": d["gmres_iterations"], "shift": d["shift"], "escalated": d["escalated"],
                     "factor_ms": d["factor_ms"], "refine_ms": d["refine_ms"]}
        del X

    lu_fl, ch_fl = 2.0 * n ** 3 / 3.0, n ** 3 / 3.0
    for p in ("bf16", "f16", "bf16x3"):
        if p != args.prec:
            rec("lu_%s_n%d" % (p, n), lambda: cf.gesv_mixed(A_lu, B_lu, prec=p, **_tourn_kw(args)), A_lu, B_lu,
                lu_fl)
        if p != args.chol_prec:
            rec("chol_%s_n%d" % (p, n), lambda: cf.posv_mixed(A_ch, B_ch, prec=p), A_ch, B_ch, ch_fl)
    A0 = inputs.uniform_pm1_torch(n, seed=0, shift=0.0, device=dev)
    for p in ("bf16x3", "bf16", "f16"):
        rec("lu_s0_%s_n%d" % (p, n), lambda: cf.gesv_mixed(A0, B_lu, prec=p, **_tourn_kw(args)), A0, B_lu, lu_fl)
    del A0
    torch.cuda.empty_cache()
    if n == 32768:
        # the N = 65536 Cholesky configuration: A = G G^T / N + alpha I
        n2 = 65536
        A2 = inputs.spd_gram_torch(n2, seed=1, alpha=0.0, device=dev)
        g = torch.Generator(device=dev)
        g.manual_seed(5)
        x = torch.randn(n2, 1, generator=g, device=dev, dtype=torch.float64)
        lam = 0.0
        for _ in range(30):
            y = A2 @ x
            lam = float(torch.linalg.vector_norm(y) / torch.linalg.vector_norm(x))
            x = y / torch.linalg.vector_norm(y)
        B2 = inputs.rhs_normal_torch(n2, 8, seed=4, device=dev)
        alpha_prev = 0.0
        for kappa in (1e2, 1e4):
            alpha = lam / (kappa - 1.0)
            A2.diagonal().add_(alpha - alpha_prev)
            alpha_prev = alpha
            rec("chol_fp8_n%d_kappa%.0e" % (n2, kappa), lambda: cf.posv_mixed(A2, B2, prec="fp8"), A2, B2,
                n2 ** 3 / 3.0)
            out["chol_fp8_n%d_kappa%.0e" % (n2, kappa)]["alpha"] = alpha
        out["lambda_max_est_n%d" % n2] = lam
        del A2, B2
        torch.cuda.empty_cache()
        out["batched_20000"] = _run_batched(dev, rank, world)
    return out


def _run_batched(dev, rank=0, world=1):
    """The batched configuration: 20,000 matrices, n ~ U{16..512} (numpy
    default_rng(7)), odd index LU of U[-1,1], even index Cholesky of
    G G^T / n + I (formed on the device; torch Philox seed 7); launch
    configuration from the autotuner; each call captured in a CUDA graph and
    timed as a graph replay (FP64 factorization; FP32 factors + FP64
    refinement with one N(0,1) right-hand side per matrix).  With several
    ranks the matrices are split by LPT on their flops (no exchange; each
    rank draws its share's values with seed 7 + 1000 rank) and the time is
    the slowest rank's."""
    import numpy as np
    import torch
    from paper_2108_09337_gb300 import cf
    sizes_all = np.random.default_rng(7).integers(16, 513, 20000).tolist()
    kinds_all = [0 if i % 2 else 1 for i in range(len(sizes_all))]
    fl_all = sum((2.0 if k == 0 else 1.0) * n ** 3 / 3.0 for n, k in zip(sizes_all, kinds_all))
    if world > 1:
        costs = [(2.0 if k == 0 else 1.0) * n ** 3 for n, k in zip(sizes_all, kinds_all)]
        shard = sorted(_lpt_shards(costs, world)[rank])
        sizes, kinds = [sizes_all[i] for i in shard], [kinds_all[i] for i in shard]
    else:
        sizes, kinds = sizes_all, kinds_all
    b = cf.Batch(sizes, kinds=kinds, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(7 + 1000 * rank)
    b.data.uniform_(-1.0, 1.0, generator=g)
    for i in range(len(sizes)):
        if kinds[i] == 1:
            M = b.matrix(i)
            M.copy_((M @ M.t()) / sizes[i] + torch.eye(sizes[i], device=dev, dtype=torch.float64))
    A0 = b.data.clone()
    fl = fl_all
    res = {"matrices": len(sizes_all), "flops": fl}
    if world > 1:
        res["matrices_this_rank"] = len(sizes)
    opt_f, ms_tf = cf.batched_autotune(b, mixed=False)
    opt_m, ms_tm = cf.batched_autotune(b, mixed=True)
    res["tuned_factor"] = {"v": opt_f.v, "ctas_per_sm": opt_f.batch_cps, "sample_ms": ms_tf}
    res["tuned_mixed"] = {"v": opt_m.v, "ctas_per_sm": opt_m.batch_cps, "sample_ms": ms_tm}
    pf = cf.BatchedPlan(b, "factor", opt=opt_f)
    pf.capture()
    b.data.copy_(A0)
    pf.replay()                                     # warm-up
    b.data.copy_(A0)
    _, ms = _timed(pf.replay)
    ms = _reduce_over_ranks(ms, world, dev, "max")
    res["fp64_factor_ms"] = ms
    res["fp64_factor_tflops"] = fl / (ms * 1e-3) / 1e12
    res["fp64_info_nonzero"] = int((pf.info != 0).sum().item())
    del pf
    b.data.copy_(A0)
    pm = cf.BatchedPlan(b, "mixed", opt=opt_m)
    pm.B.normal_(generator=g)
    pm.capture()
    pm.replay()
    _, ms = _timed(pm.replay)
    ms = _reduce_over_ranks(ms, world, dev, "max")
    eta = pm.eta.cpu().numpy()
    res["mixed_solve_ms"] = ms
    res["mixed_solve_tflops"] = fl / (ms * 1e-3) / 1e12
    res["mixed_max_eta"] = float(eta.max())
    res["mixed_mean_iterations"] = float(pm.iters.float().mean().item())
    res["mixed_fp64_fallbacks"] = int((pm.solver == 64).sum().item())
    del pm, b, A0
    torch.cuda.empty_cache()
    return res


def _perm_from_ipiv(ipiv):
    """Row order p with (P A)[i] = A[p[i]] from 1-based LAPACK interchanges."""
    import numpy as np
    ip = ipiv.cpu().numpy().astype(np.int64) - 1
    p = np.arange(ip.size)
    for i, j in enumerate(ip):
        if j != i:
            p[i], p[j] = p[j], p[i]
    return p


def _projection_residual(apply_pa, apply_l, apply_u, n, fro, dev, nvec=4, seed=0):
    """max over nvec N(0,1) vectors z of ||P A z - L (U z)||_2 / (||A||_F ||z||_2),
    the O(n^2) probabilistic form of the factorization residual, in torch FP64
    (an independent check: torch's own products, not this library's)."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    Z = torch.randn((n, nvec), generator=g, device=dev, dtype=torch.float64)
    R = apply_pa(Z) - apply_l(apply_u(Z))
    return float((torch.linalg.vector_norm(R, dim=0) / (fro * torch.linalg.vector_norm(Z, dim=0))).max())


def _run_fp64_config2(dev, sizes):
    """The FP64 path at paper-like sizes, look-ahead on: LU of U[-1,1]
    (seed 0) and Cholesky of G G^T / N + I (seed 1), one N(0,1) right-hand
    side (seed 2).  Each factorization is timed alone with CUDA events, then
    solved (cf_getrs / cf_potrs, untimed) and checked in torch FP64: eta of
    the solution and the probabilistic factorization residual over 4 random
    z, each also divided by n u (the bound the FP64 path is held to is 20 n u)."""
    import torch
    from paper_2108_09337_gb300 import cf, inputs
    u = 2.0 ** -53
    out = {}
    for n in sizes:
        rec = {}
        A = inputs.uniform_pm1_torch(n, seed=0, device=dev)
        b = inputs.rhs_normal_torch(n, 1, seed=2, device=dev)
        LU = A.t().clone().t()
        (res, ms) = _timed(lambda: cf.getrf(LU, lookahead=1))
        ipiv, info = res
        x = b.t().clone().t()
        cf.getrs(LU, ipiv, x)
        p = torch.from_numpy(_perm_from_ipiv(ipiv)).to(dev)
        Ls = torch.tril(LU, -1)
        U = torch.triu(LU)
        proj = _projection_residual(lambda Z: A[p] @ Z, lambda Z: Ls @ Z + Z, lambda Z: U @ Z, n,
                                    float(torch.linalg.matrix_norm(A)), dev)
        del Ls, U
        eta = _eta(A, x, b)
        rec["lu"] = {"ms": ms, "tflops": 2.0 * n ** 3 / 3.0 / (ms * 1e-3) / 1e12, "info": int(info.item()),
                     "eta": eta, "eta_over_nu": eta / (n * u), "proj_residual": proj,
                     "proj_residual_over_nu": proj / (n * u)}
        del A, LU, x, p
        torch.cuda.empty_cache()
        S = inputs.spd_gram_torch(n, seed=1, alpha=1.0, device=dev)
        L = S.t().clone().t()
        (info, ms) = _timed(lambda: cf.potrf(L, lookahead=1))
        x = b.t().clone().t()
        cf.potrs(L, x)
        Lt = torch.tril(L)
        proj = _projection_residual(lambda Z: S @ Z, lambda Z: Lt @ Z, lambda Z: Lt.t() @ Z, n,
                                    float(torch.linalg.matrix_norm(S)), dev)
        eta = _eta(S, x, b)
        rec["chol"] = {"ms": ms, "tflops": n ** 3 / 3.0 / (ms * 1e-3) / 1e12, "info": int(info.item()),
                       "eta": eta, "eta_over_nu": eta / (n * u), "proj_residual": proj,
                       "proj_residual_over_nu": proj / (n * u)}
        rec["within_20nu"] = all(rec[k]["info"] == 0 and rec[k]["eta_over_nu"] <= 20 and
                                 rec[k]["proj_residual_over_nu"] <= 20 for k in ("lu", "chol"))
        del S, L, Lt, x, b
        torch.cuda.empty_cache()
        out["n%d" % n] = rec
    return out


def _eta(A, X, B):
    import torch
    R = B - A @ X
    an = torch.linalg.matrix_norm(A, ord=float("inf"))
    num = R.abs().amax(dim=0)
    den = an * X.abs().amax(dim=0) + B.abs().amax(dim=0)
    return float((num / den).max())


def _fwd_err(X, Xref):
    """max_j ||x_j - xref_j||_inf / ||xref_j||_inf."""
    return float(((X - Xref).abs().amax(dim=0) / Xref.abs().amax(dim=0)).max())


def _unshifted_summary(variants, n):
    """The other half of the mixed-LU configuration (s = 0, the same uniform
    matrix without the diagonal shift), next to the headline: each update
    precision's once-run result (GMRES-IR; BF16 and FP16 escalate to split
    BF16) and the fastest of them."""
    if not variants:
        return None
    runs = {p: variants.get("lu_s0_%s_n%d" % (p, n)) for p in ("bf16x3", "bf16", "f16")}
    runs = {p: r for p, r in runs.items() if r}
    if not runs:
        return None
    ok = {p: r for p, r in runs.items() if r["status"] == 0 and r["eta"] <= TOL}
    best = min(ok, key=lambda p: ok[p]["ms"]) if ok else None
    return {"n": n, "shift": 0.0, "best_prec": best, "tflops": ok[best]["tflops"] if best else 0.0,
            "ms": ok[best]["ms"] if best else None,
            "runs": {p: {k: r[k] for k in ("ms", "tflops", "eta", "iterations", "gmres_iterations", "escalated")}
                     for p, r in runs.items()}}


def run_gpu(args, rank: int, world: int, local_rank: int):
    import numpy as np  # noqa: F401
    import torch
    import torch.distributed as dist
    from paper_2108_09337_gb300 import cf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n
    prec = args.prec
    lu_fl = 2.0 * n ** 3 / 3.0
    ch_fl = n ** 3 / 3.0

    A_lu, B_lu, A_ch, B_ch, gen_info = _gen_inputs(n, dev)
    ws_lu = torch.empty(cf.gesv_mixed_workspace_size(n, 16, prec, **_tourn_kw(args)), dtype=torch.uint8, device=dev)
    cprec = args.chol_prec
    ws_ch = torch.empty(cf.posv_mixed_workspace_size(n, 8, cprec), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step():
        X1, info1, st1, s1 = cf.gesv_mixed(A_lu, B_lu, prec=prec, work=ws_lu, **_tourn_kw(args), tol=SOLVER_TOL)
        X2, info2, st2, s2 = cf.posv_mixed(A_ch, B_ch, prec=cprec, work=ws_ch, tol=SOLVER_TOL)
        return (X1, st1, s1), (X2, st2, s2)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_step = []
    stats_lu, stats_ch = [], []
    launches0 = cf.kernel_launches()
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            (X1, S1, st1), (X2, S2, st2) = step()
            s1.record(stream)
            per_step.append((s0, s1))
            stats_lu.append(S1.as_dict())
            stats_ch.append(S2.as_dict())
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = cf.kernel_launches() - launches0
    step_stats = _step_stats([a.elapsed_time(b) for a, b in per_step])
    total_ms = _reduce_over_ranks(e0.elapsed_time(e1), world, dev, "max")
    ms_step = total_ms / args.steps
    value = _job_tflops(world, lu_fl + ch_fl, ms_step)

    # verify the last step's solutions independently (FP64 residual in torch)
    eta_lu = _eta(A_lu, X1, B_lu)
    eta_ch = _eta(A_ch, X2, B_ch)
    ok = (eta_lu <= TOL) and (eta_ch <= TOL) and st1 == cf.CF_OK and st2 == cf.CF_OK
    ok = _reduce_over_ranks(1.0 if ok else 0.0, world, dev, "min") > 0.5   # every replica converged

    # ---- per-kernel device time inside the timed steps (CUDA events on the
    # solver's stream around every launch of these kernels), and the roofline
    # of the one that takes the most time
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_mhz = float(peaks.get("sm_max_mhz") or 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = 2.0 * 128 * n_sm * sm_mhz * 1e6 / 1e12          # FFMA: 128 lanes/clk/SM
    allst = [(s, 16) for s in stats_lu] + [(s, 8) for s in stats_ch]

    def kern(ms_key, n_key, flops):
        ms = sum(s[ms_key] for s, _ in allst)
        cnt = sum(s[n_key] for s, _ in allst)
        return ms, cnt, flops
    res = kern("residual_ms", "residual_launches",
               sum(2.0 * n * n * k * s["residual_launches"] for s, k in allst))
    pair = kern("pair_ms", "pair_launches", sum(2.0 * n * n * k * s["pair_launches"] for s, k in allst))
    upd = kern("update_ms", "update_launches", sum(s["update_flops"] for s, _ in allst))
    tourn = kern("tourn_ms", "tourn_launches", sum(s["tourn_flops"] for s, _ in allst))
    # tensor-core residuals: algorithmic bytes = the eight BF16 slices of A
    # read per product, 16 N^2; cutting A into its slices (once per solve):
    # A read in FP64 and the slices written, 24 N^2
    rtc = kern("tc_ms", "tc_launches", sum(16.0 * n * n * s["tc_launches"] for s, _ in allst))
    prep_ms = sum(s["tc_prep_ms"] for s, _ in allst)
    prep_cnt = sum(1 for s, _ in allst if s["tc_prep_ms"] > 0)
    prep = (prep_ms, prep_cnt, 24.0 * n * n * prep_cnt)
    bf16_pk = peaks.get("bf16_tflops_sustained") or 1700.0
    hbm_pk = (peaks.get("hbm_gbs") or 6800.0) / 1e3        # TB/s, so that bytes / ms / 1e9 compare
    cand = {
        "tourn32": (tourn, ("k_tourn32w (LU-1, FP32 tournament pivoting, v=%d, leaves of %d rows, arity %d; "
                            "latency-bound: one barrier per column per tree level)" % (args.v, args.leaf_h, args.arity)
                            if args.v <= 64 else
                            "k_tourn32 (LU-1, FP32 tournament pivoting; latency-bound: one barrier per column "
                            "per tree level)"), "alu", fp32_peak,
                    "FP32 FMA nominal: 128 lanes/clk/SM x %d SMs x %.0f MHz x 2 flops" % (n_sm, sm_mhz),
                    TOURN_TRAFFIC.get((n, args.v, args.leaf_h, args.arity))),
        "residual_f64": (res, "k_residual_f64 (R-1, FP64 r = b - A x)", "alu", FP64_PEAK_TFLOPS,
                         "GB300 FP64 nominal 1.25 TFLOP/s (~2 DFMA/clk/SM x 152 SMs x 2.07 GHz)",
                         RESID_TRAFFIC_8192 * (n / 8192.0) ** 2),
        "residual_pair": (pair, "k_residual_pair (R-1 in FP32 pair arithmetic)", "alu", fp32_peak / 12.0,
                          "FP32 nominal / 12 (12 FP32 operations per term and right-hand side, 2 flops)",
                          None),
        "residual_tc": (rtc, "k_resid_tc (R-1 on the tensor cores: digit slices of A, exact FP32 chunk sums)",
                        "hbm", hbm_pk, "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks
                        else "fallback 6.8 TB/s", None),
        "slice_a": (prep, "k_slice_a (A cut into eight BF16 digit slices for the tensor-core residuals)", "hbm",
                    hbm_pk, "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s", None),
        "schur_tc_KV": (upd, "k_schur_tc (LU-5/CH-3, K=V tcgen05 update)", "tensor", bf16_pk,
                        "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)" if peaks
                        else "fallback 1.7 PFLOP/s sustained", None),
    }
    kernels = {}
    for name, ((ms, cnt, fl), _, bound, pk, _, _) in cand.items():
        t = (fl / (ms * 1e-3) / 1e12) if ms else None      # TFLOP/s, or TB/s for an HBM-bound kernel
        kernels[name] = {"ms_per_step": ms / args.steps, "launches_per_step": cnt / args.steps,
                         ("tb_per_s" if bound == "hbm" else "tflops"): t, "frac_of_peak": (t / pk) if t else None}
    # the K = V updates of each solve: algorithmic rate, and the tensor-pipe
    # rate (split BF16 runs three products per algorithmic flop)
    for name, sts, pr in (("schur_tc_KV_lu", stats_lu, prec), ("schur_tc_KV_chol", stats_ch, cprec)):
        ms = sum(x["update_ms"] for x in sts)
        fl = sum(x["update_flops"] for x in sts)
        t = (fl / (ms * 1e-3) / 1e12) if ms else None
        tt = t * (3.0 if pr == "bf16x3" else 1.0) if t else None
        kernels[name] = {"ms_per_step": ms / args.steps, "tflops": t, "tensor_tflops": tt,
                         "tensor_frac_of_sustained_bf16": (tt / bf16_pk) if tt else None, "prec": pr}
    top = max(cand, key=lambda k: cand[k][0][0])
    (ms, cnt, fl), label, bound, pk, src, traffic = cand[top]
    ach = (fl / max(cnt, 1)) / (ms / max(cnt, 1) * 1e-3) / 1e12 if cnt else 0.0
    if bound == "hbm":            # report GB/s against the measured copy bandwidth
        ach, pk = ach * 1e3, pk * 1e3
    roof = {"kernel": label, "bound": bound, "achieved": ach, "peak": pk,
            "unit": "GB/s" if bound == "hbm" else "TFLOP/s", "frac": ach / pk,
            "traffic": traffic, "peak_source": src, "launches": cnt, "avg_ms": ms / max(cnt, 1)}
    if top == "residual_f64":
        roof["traffic_note"] = "bytes per launch, ncu capture at N=8192 scaled by N^2"
    elif top == "tourn32":
        roof["traffic_note"] = ("DRAM bytes per launch averaged over the LU's panels, from ncu captures (the panel "
                                "is read once); null when no capture of this kernel and shape exists")
    parts = {
        "lu": {"factor_ms": statistics.median(s["factor_ms"] for s in stats_lu),
               "refine_ms": statistics.median(s["refine_ms"] for s in stats_lu),
               "iterations": stats_lu[-1]["iterations"], "eta": eta_lu, "eta0": stats_lu[-1]["eta0"]},
        "chol": {"factor_ms": statistics.median(s["factor_ms"] for s in stats_ch),
                 "refine_ms": statistics.median(s["refine_ms"] for s in stats_ch),
                 "iterations": stats_ch[-1]["iterations"], "eta": eta_ch, "eta0": stats_ch[-1]["eta0"],
                 "shift": stats_ch[-1]["shift"]},
    }
    for k in parts:
        p = parts[k]
        fl = lu_fl if k == "lu" else ch_fl
        p["tflops"] = fl / ((p["factor_ms"] + p["refine_ms"]) * 1e-3) / 1e12

    # ---- e2e: same step through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        hA_lu = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hA_lu.copy_(A_lu)
        hB_lu = torch.empty((16, n), dtype=torch.float64, pin_memory=True).t()
        hB_lu.copy_(B_lu)
        hA_ch = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hA_ch.copy_(A_ch)
        hB_ch = torch.empty((8, n), dtype=torch.float64, pin_memory=True).t()
        hB_ch.copy_(B_ch)
        hX1 = torch.empty((16, n), dtype=torch.float64, pin_memory=True).t()
        hX2 = torch.empty((8, n), dtype=torch.float64, pin_memory=True).t()
        # Inputs are staged on a side stream while the solves run: at the
        # start of step k, step k's Cholesky system and then step k+1's LU
        # system (double-buffered).  Every step
        # copies all of its inputs inside the timed region, the first step's
        # LU system included; a copy waits for the solve that last read its
        # destination.
        dA1 = [torch.empty_like(A_lu), torch.empty_like(A_lu)]
        dB1 = [torch.empty_like(B_lu), torch.empty_like(B_lu)]
        dA2, dB2 = torch.empty_like(A_ch), torch.empty_like(B_ch)
        del A_lu, A_ch
        torch.cuda.empty_cache()
        side = torch.cuda.Stream(device=dev)
        lu_in = [torch.cuda.Event(), torch.cuda.Event()]
        lu_free = [torch.cuda.Event(), torch.cuda.Event()]
        ch_in, ch_free = torch.cuda.Event(), torch.cuda.Event()

        def copy_lu(slot):
            side.wait_event(lu_free[slot])
            with torch.cuda.stream(side):
                dA1[slot].copy_(hA_lu, non_blocking=True)
                dB1[slot].copy_(hB_lu, non_blocking=True)
                lu_in[slot].record(side)

        def e2e_run(k):
            for ev in lu_free + [ch_free]:
                ev.record(stream)
            copy_lu(0)
            for i in range(k):
                slot = i & 1
                side.wait_event(ch_free)
                with torch.cuda.stream(side):
                    dA2.copy_(hA_ch, non_blocking=True)
                    dB2.copy_(hB_ch, non_blocking=True)
                    ch_in.record(side)
                if i + 1 < k:
                    copy_lu(1 - slot)       # its buffer's last reader was step i-1
                stream.wait_event(lu_in[slot])
                X1_, _, _, _ = cf.gesv_mixed(dA1[slot], dB1[slot], prec=prec, work=ws_lu, **_tourn_kw(args),
                                             tol=SOLVER_TOL)
                lu_free[slot].record(stream)
                hX1.copy_(X1_, non_blocking=True)
                stream.wait_event(ch_in)
                X2_, _, _, _ = cf.posv_mixed(dA2, dB2, prec=cprec, work=ws_ch, tol=SOLVER_TOL)
                ch_free.record(stream)
                hX2.copy_(X2_, non_blocking=True)
            stream.wait_stream(side)

        e2e_run(1)
        torch.cuda.synchronize()
        k2 = max(1, args.steps)
        barrier()
        e0.record(stream)
        e2e_run(k2)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms2 = _reduce_over_ranks(e0.elapsed_time(e1) / k2, world, dev, "max")
        h2d = 2 * n * n * 8 + (16 + 8) * n * 8
        d2h = (16 + 8) * n * 8
        e2e = {"value": _job_tflops(world, lu_fl + ch_fl, ms2), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms2}
        del hA_lu, hA_ch, dA1, dA2, dB1, dB2
        torch.cuda.empty_cache()

    # ---- this project's FP64 path on the same matrices (one run each)
    fp64 = None
    if not args.no_fp64:
        from paper_2108_09337_gb300 import inputs
        A64 = inputs.uniform_pm1_torch(n, seed=0, shift=2.0 * math.sqrt(n), device=dev)
        A64 = A64.t().contiguous().t() if A64.stride(0) != 1 else A64
        torch.cuda.synchronize()
        e0.record(stream)
        ipiv, info = cf.getrf(A64)
        e1.record(stream)
        torch.cuda.synchronize()
        lu_ms = e0.elapsed_time(e1)
        # forward error of the timed step's mixed solutions against this
        # FP64 path's solutions of the same systems (untimed)
        fwd = {}
        X64 = B_lu.t().clone().t()
        cf.getrs(A64, ipiv, X64)
        fwd["lu"] = _fwd_err(X1, X64)
        del A64, ipiv, X64
        S64 = inputs.spd_gram_torch(n, seed=1, alpha=gen_info["alpha"], device=dev)
        torch.cuda.synchronize()
        e0.record(stream)
        cf.potrf(S64)
        e1.record(stream)
        torch.cuda.synchronize()
        ch_ms = e0.elapsed_time(e1)
        X64 = B_ch.t().clone().t()
        cf.potrs(S64, X64)
        fwd["chol"] = _fwd_err(X2, X64)
        del S64, X64
        fp64 = {"lu_ms": lu_ms, "chol_ms": ch_ms, "lu_tflops": lu_fl / (lu_ms * 1e-3) / 1e12,
                "chol_tflops": ch_fl / (ch_ms * 1e-3) / 1e12,
                "tflops": (lu_fl + ch_fl) / ((lu_ms + ch_ms) * 1e-3) / 1e12,
                "mixed_forward_error_vs_fp64": fwd,
                "note": "factorization only (FP64 path; its solve adds O(N^2))"}
        torch.cuda.empty_cache()
        sizes = [int(x) for x in args.fp64_sizes.split(",") if x.strip()]
        if sizes:
            fp64["config2"] = _run_fp64_config2(dev, sizes)

    # ---- once-run legs of the other configurations (not part of value),
    # after the timed legs so that their allocations cannot disturb them
    variants = None
    if not args.no_variants:
        A_lu, B_lu, A_ch, B_ch, _ = _gen_inputs(n, dev)
        variants = _run_variants(args, n, dev, A_lu, B_lu, A_ch, B_ch, rank, world)
        del A_lu, A_ch
        torch.cuda.empty_cache()

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        r, dt, threads = _oracle_sample(4096, args.v, args.leaf_h, args.arity)
        cpu = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle", "host": _host_cpu(),
               "sample": "FP64 oracle LU (tournament, v=%d, h=%d, arity %d) + Cholesky at N=4096, same "
                         "generators, %.1f s on this host" % (args.v, args.leaf_h, args.arity, dt)}
    line = {
        "metric": METRIC, "value": value if ok else 0.0, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec if prec == cprec else "%s (LU) + %s (Cholesky)" % (prec, cprec),
        "data": "synthetic",
        "config": {"workload": "mixed LU solve (N=32768, 16 RHS, A=U[-1,1]+2sqrt(N)I, %s tensor-core updates) + "
                               "mixed Cholesky solve (N=32768, 8 RHS, A=GG^T/N+alpha I, kappa~1e2, %s tensor-core "
                               "updates), FP32 accumulation, FP64 refinement to 1e-14" % (prec, cprec),
                   "n": n, "v": {"lu": args.v, "chol": 128}, "leaf_h": args.leaf_h, "arity": args.arity,
                   "outer_V": {"lu": 2048, "chol": 2048},
                   "factor_prec": prec,
                   "chol_factor_prec": cprec,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (A is 8.6 GB per matrix)", "inputs": gen_info},
        "converged": ok, "eta": {"lu": eta_lu, "chol": eta_ch},
        "step_stats": step_stats, "parts": parts, "kernels": kernels,
        "clocks": clk.summary(),
        "e2e": e2e, "gpu_launches": launches,
        "roofline": roof, "cpu_baseline": cpu, "fp64_path": fp64, "variants": variants,
        "speedup_vs_fp64": (value / fp64["tflops"]) if (fp64 and ok) else None,
        "lu_unshifted": _unshifted_summary(variants, n),
    }
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
