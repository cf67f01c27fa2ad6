#!/usr/bin/env python
"""Benchmark: GW self-energy evaluations per second on one GB300.

One step is one self-energy evaluation -- P0(tau) (Eq. tilde_P0_tau), the
tau -> i Omega transform, the auxiliary Dyson equation (Eq. tilde_P_omega),
the transform back, and Sigma(tau) (Eqs. sigma_gw, tilde_W_DF2) -- over every
k and tau of the 4x4x4 solid (nk=64, nao=52, naux=400, ntau=120, beta=200;
4295 TFLOP per evaluation), with V, G and all workspaces resident in HBM.
The Si-like 3x3x3 solid (nk=27, nao=26, naux=200) runs with
--workload solid_3x3x3_nao26.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x4|fp64]
    python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample
    python bench.py --serving [--serving-jobs N] [--precision P]   # scGW job stream alone
    python bench.py --batched [--precision P] [--steps K]          # 48 molecules: every batch mode

Under torchrun (N > 1) every rank evaluates its own seeded system (weak
scaling, no collective on the data path); the time is the maximum over ranks.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("GW Σ evals/s & TFLOP/s vs peak, mixed vs FP64 at max|ΔΣ|≤1e-6 Ha; p50/p99")
UNIT = "sigma_evals/s"
WORKLOAD = "solid_4x4x4_nao52"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 nominal FP64, used only if the live measurement fails
# a full FP64 evaluation is compared only up to this many algorithmic TFLOP (about 2 minutes of
# FP64 work); above it the FP64 comparison runs on a sample of momentum transfers q
FP64_FULL_MAX_TFLOP = 100.0


def canonical_fraction(nk3, n):
    """Share of (q, index) pairs computed when X^q(n-1-i) = X^{-q}(i)^T is used: the q with
    -q = q (mod the Gamma-centred mesh) keep (n+1)/2 of n indices, the other q half of theirs."""
    sc = 1
    for m in nk3:
        sc *= 2 if m % 2 == 0 else 1
    nk = int(np.prod(nk3))
    return (sc * ((n + 1) // 2) + (nk - sc) * n / 2.0) / (nk * n)


def algorithmic_flops(nk3, nao, naux, ntau, nwb):
    """Real flops of one evaluation as computed, 8 per complex multiply-add (Eqs. tilde_P0_tau ...
    sigma_gw): P0 and the aux Dyson solves only at canonical (q, tau) and (q, n); Sigma in full."""
    nk = int(np.prod(nk3))
    contraction = 8.0 * nk * nk * ntau * (2.0 * naux * nao ** 3 + naux ** 2 * nao ** 2)   # each of P0, Sigma
    transforms = 2 * 8.0 * nk * nwb * ntau * naux ** 2
    dyson = (8.0 * nk * nwb * naux ** 3 + 2.0 * nk * nwb * naux ** 2) * canonical_fraction(nk3, nwb)
    return contraction * canonical_fraction(nk3, ntau) + contraction + transforms + dyson


def stage_flops(nk3, nao, naux, ntau):
    """Algorithmic flops (8 per complex multiply-add) of one evaluation per tensor-core GEMM class,
    as computed: P0 and its V.G products at canonical (q, tau), the Sigma side at every (q, tau)."""
    nk = int(np.prod(nk3))
    cf = canonical_fraction(nk3, ntau)
    per = 8.0 * nk * nk * ntau
    return {"vg_gemm_tc": per * (2.0 * naux * nao ** 3 * cf + naux * nao ** 3),
            "p0_gemm_tc": per * cf * naux ** 2 * nao ** 2,
            "r_gemm_tc": per * naux ** 2 * nao ** 2,
            "sigma_gemm_tc": per * naux * nao ** 3}


def fp64_peak_tflops():
    """Measured FP64 rate of this GPU: torch complex128 matmul (cuBLAS ZGEMM) of 4096^3, best
    of 5, 8 real flops per complex multiply-add. cuBLAS serves only as the yardstick here."""
    import torch
    try:
        a = torch.randn(4096, 4096, dtype=torch.complex128, device="cuda")
        b = torch.randn_like(a)
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        return 8.0 * 4096 ** 3 / (best * 1e-3) / 1e12, "complex128 matmul 4096^3 on this GPU (measured)"
    except Exception as e:  # noqa: BLE001 - the nominal figure stands in, labelled as such
        return FP64_NOMINAL_TFLOPS, f"GB300 nominal (measurement failed: {e})"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9 and p[1].replace(".", "").isdigit():
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def oracle_sample(w, h, v, g, budget_s=15.0):
    """Time the FP64 CPU oracle on whole units of each stage and extrapolate one evaluation.

    Units: P0 for one (q, tau); Sigma for one (k, tau); one aux Dyson solve (q, Omega);
    the transforms for one q. The loop repeats units until budget_s is spent.
    """
    from oracle import grids, gw as O
    nk, ntau = w.nk, w.ntau
    m, F, B = grids.transform_matrices(ntau, w.beta, 0)
    nwb = len(m)
    rng = np.random.default_rng(0)
    t_p0 = t_sig = t_dys = t_tr = 0.0
    n_p0 = n_sig = n_dys = n_tr = 0
    start = time.perf_counter()
    pt_fake = None
    while True:
        t0 = time.perf_counter()
        q, t = int(rng.integers(nk)), int(rng.integers(ntau))
        p0 = O.polarization(v, g, w.nk3, 2.0, q_list=[q], t_list=[t])
        t_p0 += time.perf_counter() - t0
        n_p0 += 1
        if pt_fake is None:
            pt_fake = np.broadcast_to(p0[0, 0], (nk, ntau) + p0.shape[2:]).copy()
        t0 = time.perf_counter()
        O.self_energy(v, g, pt_fake, w.nk3, k_list=[int(rng.integers(nk))], t_list=[t])
        t_sig += time.perf_counter() - t0
        n_sig += 1
        t0 = time.perf_counter()
        O.aux_dyson(pt_fake[:1, :1])
        t_dys += time.perf_counter() - t0
        n_dys += 1
        if n_tr == 0 or time.perf_counter() - start < budget_s / 2:
            t0 = time.perf_counter()
            O.to_tau(O.to_matsubara(pt_fake[:1], F), B)
            t_tr += time.perf_counter() - t0
            n_tr += 1
        if time.perf_counter() - start > budget_s:
            break
    per_eval = (t_p0 / n_p0) * nk * ntau + (t_sig / n_sig) * nk * ntau + (t_dys / n_dys) * nk * nwb \
        + (t_tr / n_tr) * nk
    sample = (f"{n_p0} P0 (q,tau) units, {n_sig} Sigma (k,tau) units, {n_dys} aux Dyson solves, "
              f"{n_tr} transform pairs in {time.perf_counter() - start:.1f} s; extrapolated to "
              f"{nk * ntau} + {nk * ntau} + {nk * nwb} + {nk} units per evaluation")
    return 1.0 / per_eval, sample, time.perf_counter() - start


class CpuMeter:
    """Cores a block of host work actually kept busy: process CPU time over wall time."""

    def __enter__(self):
        self.c0, self.w0 = time.process_time(), time.perf_counter()
        return self

    def __exit__(self, *a):
        self.cpu = time.process_time() - self.c0
        self.wall = time.perf_counter() - self.w0

    @property
    def cores(self):
        return round(self.cpu / max(self.wall, 1e-9), 1)


def source_hash(rec):
    """sha256 of the kernel's source: the lines from rec["region"][0] up to rec["region"][1] of
    rec["source"] (the whole file without a region); None if the file or a marker is missing."""
    try:
        text = open(os.path.join(ROOT, rec["source"]), encoding="utf-8").read()
    except OSError:
        return None
    if rec.get("region"):
        a = text.find(rec["region"][0])
        b = text.find(rec["region"][1], a + 1) if a >= 0 else -1
        if a < 0 or b < 0:
            return None
        text = text[a:b]
    return hashlib.sha256(text.encode()).hexdigest()


def ncu_traffic(kernel, algorithmic_bytes_per_launch):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if its source is unchanged:
    the capture's DRAM bytes per algorithmic byte (a smaller case of the same kernel) times the
    bench launches' algorithmic bytes."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    if source_hash(rec) != rec["source_sha256"]:
        return None
    return rec["dram_per_algorithmic_byte"] * algorithmic_bytes_per_launch


def in_turns(rank, world, fn, barrier, per_turn=2):
    """fn() on every rank, per_turn ranks at a time (turn rank // per_turn), a barrier after each
    turn; returns this rank's fn()."""
    out = None
    for turn in range((world + per_turn - 1) // per_turn):
        if rank // per_turn == turn:
            out = fn()
        barrier()
    return out


def max_over_ranks(value, dist=None):
    """The largest value over all ranks (the timing rule for a multi-rank run)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank):
    from paper_2406_18479_gb300 import inputs as I
    if rank != 0:
        return
    w = I.WORKLOADS[args.workload]
    h, v, g = I.make_inputs(w)
    vals = []
    sample = ""
    for _ in range(args.warmup):
        oracle_sample(w, h, v, g, budget_s=2.0)
    t_all = time.perf_counter()
    with CpuMeter() as cpu:
        for _ in range(args.steps):
            val, sample, _ = oracle_sample(w, h, v, g, budget_s=args.ref_budget)
            vals.append(val)
    wall = time.perf_counter() - t_all
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic (seeded)",
        "config": {"workload": w.name, "nk": w.nk, "nao": w.nao, "naux": w.naux, "ntau": w.ntau,
                   "beta": w.beta, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu.cores, "kind": "oracle",
                         "sample": sample + f"; numpy with its BLAS, cores = CPU time / wall time of the "
                                            f"timed samples ({os.cpu_count()} available)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def job_flops(w):
    """Algorithmic flops of one self-energy evaluation of a job (both contractions, symmetric count)."""
    return 16.0 * w.nk ** 2 * w.ntau * (2.0 * w.naux * w.nao ** 3 + w.naux ** 2 * w.nao ** 2)


def serving_measure(precision, n_jobs, slots=4, budget_gb=160.0, max_tflop=None, seed=5, alpha=0.5,
                    tol=1e-6, itermax=10):
    """scGW job stream through gw_submit / gw_poll.

    Jobs are the first n_jobs of the seeded stream (70% molecules, 30% 2x2x2 / 3x3x3 solids,
    naux = 4 nao, 80 tau nodes), optionally without those above max_tflop per evaluation. Two
    passes over the same jobs: closed loop (all submitted at once) gives the capacity in jobs/s;
    then an open loop with Poisson arrivals at 0.8 x that capacity gives the latency percentiles.
    """
    from paper_2406_18479_gb300 import gw, inputs as I
    stream = I.serving_stream(n_jobs, seed)
    if max_tflop is not None:
        stream = [(gap, w) for gap, w in stream if job_flops(w) <= max_tflop * 1e12]
    t_gen = time.perf_counter()
    jobs = []
    for gap, w in stream:
        h, v, g = I.make_inputs(w)
        cfg = gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, mu=w.mu, precision=precision)
        jobs.append((gap, w, cfg, h, v, g))
    t_gen = time.perf_counter() - t_gen
    srv = gw.gw_server(int(budget_gb * 2 ** 30), slots)

    def run(gaps):
        ids = []
        t0 = time.perf_counter()
        tnext = t0
        for (gap, w, cfg, h, v, g), dt in zip(jobs, gaps):
            tnext += dt
            pause = tnext - time.perf_counter()
            if pause > 0:
                time.sleep(pause)
            ids.append(srv.submit(cfg, h, v, g, alpha=alpha, tol=tol, itermax=itermax))
        return [srv.poll(i, -1)[1] for i in ids]

    try:
        closed = run([0.0] * len(jobs))
        span = max(r["t_end"] for r in closed) - min(r["t_submit"] for r in closed)
        capacity = len(jobs) / span
        rate = 0.8 * capacity
        opened = run([gap / rate for gap, *_ in jobs])
    finally:
        srv.destroy()
    lat = np.array([r["t_end"] - r["t_submit"] for r in opened])
    wait = np.array([r["t_start"] - r["t_submit"] for r in opened])
    ok = [r["status"] in (gw.GW_OK, gw.GW_ENOTCONV) for r in opened + closed]
    span_o = max(r["t_end"] for r in opened) - min(r["t_submit"] for r in opened)
    evals = sum(r["iterations"] for r in opened)
    return {
        "precision": precision, "jobs": len(jobs), "slots": slots, "hbm_budget_gb": budget_gb,
        "sample": (f"first {n_jobs} jobs of the seeded stream (seed {seed})"
                   + (f", jobs above {max_tflop} TFLOP per evaluation left out" if max_tflop else "")
                   + f": {sum(1 for j in jobs if not j[1].solid)} molecules, "
                   f"{sum(1 for j in jobs if j[1].solid)} solids"),
        "alpha": alpha, "tol": tol, "itermax": itermax,
        "capacity_jobs_per_s": capacity, "arrival_rate_jobs_per_s": rate,
        "jobs_per_s": len(jobs) / span_o,
        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
        "p50_queue_s": float(np.percentile(wait, 50)),
        "sigma_evals": evals, "converged": sum(1 for r in opened if r["status"] == gw.GW_OK),
        "all_ok": all(ok), "tflop_per_eval_mean": float(np.mean([job_flops(j[1]) for j in jobs]) / 1e12),
        "input_generation_s": t_gen,
    }


def fp64_compare(w, V, G, Sig_mixed, ctx, grid, args, t_mixed_ms):
    """Mixed against the GPU FP64 path. A full FP64 evaluation up to FP64_FULL_MAX_TFLOP of work;
    above it, a sample of momentum transfers (Eq. sigma_gw sums over q, gw_sigma_eval_q gives the
    part of one q): q = 0, whose -q is itself, so that its cost is the average per-q cost of a
    full evaluation (P0 at half the tau nodes by the mirror relation, Sigma at all). Reports the
    largest |dSigma_q| over the sample, and two extrapolations to the full sum over nk values of q:
    sqrt(nk) x that (errors of independent q adding like a random walk) and nk x that (the triangle
    inequality, a bound)."""
    import torch
    from paper_2406_18479_gb300 import gw

    def make64():
        c = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64", v_packed=args.v_packed)
        if grid is not None:
            gw.gw_set_grids(c, *grid)
        gw.gw_set_coulomb(c, V)
        return c

    def timed(stream, fn):
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1)

    if algorithmic_flops(w.nk3, w.nao, w.naux, w.ntau, gw.gw_sample_count(w.ntau, 0)) <= FP64_FULL_MAX_TFLOP * 1e12:
        gw.gw_sigma_eval(ctx, G, Sig_mixed)
        torch.cuda.synchronize()
        mixed = Sig_mixed.cpu()
        ctx.destroy()
        torch.cuda.empty_cache()
        c64 = make64()
        S64 = torch.empty_like(Sig_mixed)
        ms64 = timed(c64.stream, lambda: gw.gw_sigma_eval(c64, G, S64))
        ref = S64.cpu()
        c64.destroy()
        return {"method": "full evaluation", "ms_per_eval": ms64, "speedup_mixed_over_fp64": ms64 / t_mixed_ms,
                "max_abs_dSigma_Ha": float((mixed - ref).abs().max()),
                "max_abs_Sigma_Ha": float(ref.abs().max())}
    q = 0
    gw.gw_sigma_eval_q(ctx, G, Sig_mixed, q, q + 1)
    torch.cuda.synchronize()
    mixed = Sig_mixed.cpu()
    ctx.destroy()
    torch.cuda.empty_cache()
    c64 = make64()
    S64 = torch.empty_like(Sig_mixed)
    ms_q = timed(c64.stream, lambda: gw.gw_sigma_eval_q(c64, G, S64, q, q + 1))
    ref = S64.cpu()
    c64.destroy()
    d = float((mixed - ref).abs().max())
    ms64 = ms_q * w.nk
    return {"method": f"sample of q: q = {q} (the part of Sigma from one momentum transfer, Eq. sigma_gw)",
            "q": [q], "ms_per_q_fp64": ms_q,
            "ms_per_eval": ms64, "ms_per_eval_note": "extrapolated: nk x the FP64 time of q = 0",
            "speedup_mixed_over_fp64": ms64 / t_mixed_ms,
            "max_abs_dSigma_q_Ha": d, "max_abs_Sigma_q_Ha": float(ref.abs().max()),
            "max_abs_dSigma_Ha_estimate": d * float(np.sqrt(w.nk)),
            "max_abs_dSigma_Ha_bound": d * w.nk,
            "estimate_note": "sqrt(nk) x the sampled q (independent per-q errors); bound: nk x it"}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2406_18479_gb300 import gw, inputs as I

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    base = I.WORKLOADS[args.workload]
    w = I.Workload(base.name, base.nk3, base.nao, base.naux, base.ntau, base.nomega, base.beta, base.mu,
                   base.decay, base.seed + rank, base.solid)
    t_in = time.perf_counter()
    keep_v = rank == 0 and world == 1 and not args.no_cpu_baseline and args.ir_lambda <= 0

    def make_inputs():
        h, v, g = I.make_inputs(w)
        grid, wr = None, w
        if args.ir_lambda > 0:
            # the same system on an IR grid (the tau node count follows from Lambda and eps)
            grid = gw.gw_ir_grids(w.beta, args.ir_lambda, args.ir_eps)
            wr = I.Workload(f"{w.name}_ir{args.ir_lambda:g}", w.nk3, w.nao, w.naux, len(grid[0]), len(grid[0]),
                            w.beta, w.mu, w.decay, w.seed, w.solid)
            g = I.g0_tau(h, w.mu, w.beta, grid[0])
        V = torch.from_numpy(I.pack_v(v) if args.v_packed else v).cuda()
        G = torch.from_numpy(g).cuda()
        return h, (v if keep_v else None), g, grid, wr, V, G

    # the host copy of a 4x4x4 solid's V is 71 GB: ranks on one node build their inputs two at a
    # time, each freeing its host V once it is on the device
    h, v, g, grid, w, V, G = in_turns(rank, world, make_inputs, barrier)
    v_bytes = V.numel() * 16
    input_s = time.perf_counter() - t_in
    ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=args.precision, tau_chunk=args.tau_chunk,
                       v_packed=args.v_packed, slice_pass=args.slice_pass)
    if grid is not None:
        gw.gw_set_grids(ctx, *grid)
    Sig = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    gw.gw_set_coulomb(ctx, V)
    stream = ctx.stream
    # warm-up; the last warm-up evaluation is profiled per launch (CUDA events on the stream) for the
    # kernel shares and the roofline, so that the timed evaluations run without instrumentation
    for i in range(args.warmup):
        if i == args.warmup - 1:
            gw.gw_profile_enable(ctx, True)
        gw.gw_sigma_eval(ctx, G, Sig)
    gw.gw_synchronize(ctx)
    prof = gw.gw_profile_read(ctx)
    gw.gw_profile_enable(ctx, False)
    gw.gw_synchronize(ctx)

    # ---- device-resident timed region (no per-launch instrumentation)
    # one event before the first step and one after every step: the total and the per-step spread
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches0 = gw.gw_launch_count(ctx)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            gw.gw_sigma_eval(ctx, G, Sig)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    launches = gw.gw_launch_count(ctx) - launches0
    t_max = max_over_ranks(ms, dist)

    # ---- end to end through the public API with host buffers (pinned): about half a minute of
    #      steps (at least one)
    G_host = torch.from_numpy(g).pin_memory()
    S_host = torch.empty(Sig.shape, dtype=Sig.dtype).pin_memory()
    k_e2e = max(1, min(args.steps, int(np.ceil(30000.0 / max(t_max / args.steps, 1e-3)))))
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        f0.record(stream)
        for _ in range(k_e2e):
            G.copy_(G_host, non_blocking=True)
            gw.gw_sigma_eval(ctx, G, Sig)
            S_host.copy_(Sig, non_blocking=True)
        f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), dist)

    # ---- FP64 comparison for the mixed precisions (full, or on a sample of q); frees ctx
    fp64 = None
    if args.precision != "fp64" and args.fp64_compare:
        fp64 = fp64_compare(w, V, G, Sig, ctx, grid, args, t_max / args.steps)
    else:
        ctx.destroy()
    del V
    torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    fp64_peak, fp64_peak_note = fp64_peak_tflops()
    serving = None
    if world == 1 and args.serving_jobs > 0:
        serving = serving_measure(args.precision, args.serving_jobs)
        if args.precision != "fp64" and args.fp64_compare:
            # mixed and FP64 on the same jobs: those of the sample at most this many TFLOP per
            # evaluation, so that the FP64 pass takes seconds
            lim = args.serving_fp64_max_tflop
            serving["vs_fp64"] = {"max_tflop_per_eval": lim,
                                  args.precision: serving_measure(args.precision, args.serving_jobs, max_tflop=lim),
                                  "fp64": serving_measure("fp64", args.serving_jobs, max_tflop=lim)}

    nwb = gw.gw_sample_count(w.ntau, 0)
    flops = algorithmic_flops(w.nk3, w.nao, w.naux, w.ntau, nwb)
    steps = args.steps
    value = world * steps / (t_max / 1e3)
    peaks, peak_src = measured_peaks()
    bf16_peak = peaks["bf16_tflops_sustained"]
    alg = stage_flops(w.nk3, w.nao, w.naux, w.ntau)
    prof_total = sum(y["ms"] for y in prof.values())
    kernels = {}
    for k, x in prof.items():
        e = {"launches": x["launches"], "ms": round(x["ms"], 3), "share": round(x["ms"] / prof_total, 4)}
        if k.endswith("_tc") and x["ms"] > 0:
            ex = x["flops"] / (x["ms"] * 1e-3) / 1e12
            e["executed_bf16_tflops"] = round(ex, 1)
            e["tensor_pipe_frac_of_sustained_peak"] = round(ex / bf16_peak, 4)
            if k in alg:
                e["algorithmic_tflops"] = round(alg[k] / (x["ms"] * 1e-3) / 1e12, 2)
        kernels[k] = e
    # dominant kernel by device time (of the profiled evaluation)
    dname, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    per_launch_ms = d["ms"] / d["launches"]
    if dname.endswith("_tc"):
        bound, unit = "tensor", "TFLOP/s"
        achieved = d["flops"] / d["launches"] / (per_launch_ms * 1e-3) / 1e12
        peak = bf16_peak
        peak_note = (f"bf16 dense sustained ({peak_src}); achieved counts the executed bf16 flops "
                     f"(10 slice products of 4 real MMAs per complex multiply-add)")
    elif dname in ("slice_planes", "elementwise", "reduce"):
        bound, unit = "hbm", "GB/s"
        achieved = d["bytes"] / d["launches"] / (per_launch_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        peak_note = f"HBM copy ({peak_src})"
    else:
        bound, unit = "alu", "TFLOP/s"
        achieved = d["flops"] / d["launches"] / (per_launch_ms * 1e-3) / 1e12
        peak, peak_note = fp64_peak, "FP64: " + fp64_peak_note
    traffic = ncu_traffic(dname, d["bytes"] / d["launches"])
    clocks = clk.summary()
    p_bytes = w.nk * w.ntau * w.naux ** 2 * 16
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": t_max / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "c128 (f64)",
                  "bf16x4": "bf16 (four exact slices per operand), f32 accumulate, f64 transforms/Dyson"}[args.precision],
        "data": "synthetic (seeded H(k), V, G0 shaped like the paper's Si example)",
        "config": {"workload": w.name, "nk": w.nk, "nao": w.nao, "naux": w.naux, "ntau": w.ntau,
                   "nomega": nwb, "beta": w.beta, "precision": args.precision, "tau_chunk": args.tau_chunk,
                   "slice_output": "separate slicing pass" if args.slice_pass else "from the producing GEMM where the sizes allow",
                   "l2": f"inputs larger than L2 (V {v_bytes / 1e9:.1f} GB, P {p_bytes / 1e9:.1f} GB per pass)",
                   "grid": (f"IR Lambda={args.ir_lambda:g} eps={args.ir_eps:g}" if grid is not None
                            else "Chebyshev"),
                   "v_layout": "packed k1<=k2" if args.v_packed else "all pairs",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "tflops_algorithmic": flops * world * steps / (t_max / 1e3) / 1e12,
        "tflop_per_eval_algorithmic": flops / 1e12,
        "step_ms": {"median": float(np.median(step_ms)), "p99": float(np.percentile(step_ms, 99)),
                    "min": float(np.min(step_ms)), "max": float(np.max(step_ms))},
        "roofline": {"kernel": dname, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_note},
        "kernels": kernels,
        "kernels_note": "one profiled warm-up evaluation (CUDA events per launch); the timed steps ran without",
        "fp64_peak_tflops": {"value": fp64_peak, "source": fp64_peak_note},
        "gpu_launches": launches,
        "e2e": {"value": world * k_e2e / (e2e_ms / 1e3), "unit": UNIT, "steps": k_e2e,
                "h2d_bytes_per_step": int(G.numel() * 16), "d2h_bytes_per_step": int(Sig.numel() * 16)},
        "clocks": clocks,
        "input_generation_s": input_s,
    }
    if fp64 is not None:
        line["fp64"] = fp64
    if serving is not None:
        line["serving"] = serving
    if world == 1 and args.batched_default:
        # the 48-molecule batch: per-system loop against concurrent streams and the captured grouped
        # flow (one step each; bench.py --batched times every mode and the tuner)
        line["batched"] = batched_measure(args.precision, steps=1, max_streams=args.batch_streams, tune=False,
                                          modes=("serial", "streams", "grouped_graph"))
    if keep_v:
        with CpuMeter() as cpu:
            val, sample, spent = oracle_sample(w, h, v, g, budget_s=args.ref_budget)
        line["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": cpu.cores, "kind": "oracle",
                                "sample": sample + f"; cores = CPU time / wall time ({os.cpu_count()} available)"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def batched_measure(precision, n_systems=48, steps=3, max_streams=8, tune=True, seed=4,
                    modes=("serial", "streams", "graph", "grouped", "grouped_graph")):
    """Self-energy evaluations of n Gamma-only systems (nao uniform on {10..120}, naux = 4 nao,
    80 tau nodes, beta = 100) per second: per-system loop, concurrent streams, one captured
    graph, the grouped inversion (eager and captured), then the two graph modes again after the
    per-system tuner."""
    import torch
    from paper_2406_18479_gb300 import gw, inputs as I
    ws = I.batched_molecules(n_systems, seed)
    cfgs = [gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=precision) for w in ws]
    V, G, S = [], [], []
    for w in ws:
        h, v, g = I.make_inputs(w)
        V.append(torch.from_numpy(v).cuda())
        G.append(torch.from_numpy(g).cuda())
        S.append(torch.empty((1, w.ntau, w.nao, w.nao), dtype=torch.complex128, device="cuda"))
    b = gw.gw_batch(cfgs, max_streams=max_streams)
    b.set_coulomb(V)
    stream = b.stream
    print(f"batch of {n_systems}: inputs ready", file=sys.stderr, flush=True)

    def timed(mode):
        b.sigma_eval(G, S, mode)               # warm-up (and, for the graph, the capture)
        b.sigma_eval(G, S, mode)
        b.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            b.sigma_eval(G, S, mode)
        e1.record(stream)
        b.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {"systems": n_systems, "precision": precision, "streams": max_streams, "steps": steps,
           "nao": [w.nao for w in ws], "tflop_per_batch": sum(job_flops(w) for w in ws) / 1e12}
    ms = {}
    for m in modes:
        ms[m] = timed(m)
        print(f"  {m}: {ms[m]:.1f} ms per batch", file=sys.stderr, flush=True)
    if tune:
        t0 = time.perf_counter()
        out["tau_batches"] = b.autotune(G, S)
        out["tile_widths"] = [wd for _, wd in b.tuned()]
        out["tune_s"] = time.perf_counter() - t0
        for m in ("graph", "grouped_graph"):
            ms[m + "_tuned"] = timed(m)
            print(f"  {m}_tuned: {ms[m + '_tuned']:.1f} ms per batch", file=sys.stderr, flush=True)
    b.destroy()
    out["ms_per_batch"] = ms
    out["systems_per_s"] = {m: n_systems / (v / 1e3) for m, v in ms.items()}
    out["tflops_algorithmic"] = {m: out["tflop_per_batch"] / (v / 1e3) for m, v in ms.items()}
    return out


def run_batched(args, rank, local_rank):
    """One JSON line for the 48-molecule batch alone (rank 0; other ranks exit)."""
    import torch
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    with ClockSampler(local_rank) as clk:
        r = batched_measure(args.precision, steps=args.steps, max_streams=args.batch_streams)
    best_mode = min(r["ms_per_batch"], key=r["ms_per_batch"].get)
    best = r["ms_per_batch"][best_mode]
    line = {"metric": "sigma_evals/s over a batch of 48 molecules (nao 10..120)",
            "value": r["systems"] / (best / 1e3), "unit": "sigma_evals/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 2, "ms_per_step": best, "higher_is_better": True, "dtype": args.precision,
            "data": "synthetic (seeded molecules)",
            "config": {"workload": "batched_molecules_48", "precision": args.precision, "mode": best_mode},
            "batched": r, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_serving(args, rank, local_rank):
    """One JSON line for the scGW job stream alone (rank 0; other ranks exit)."""
    import torch
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    n = args.serving_jobs if args.serving_jobs > 0 else 200
    with ClockSampler(local_rank) as clk:
        s = serving_measure(args.precision, n, slots=args.serving_slots, max_tflop=args.serving_max_tflop)
    line = {"metric": "scGW jobs/s with p50/p99 latency (Poisson stream at 0.8 x capacity)",
            "value": s["jobs_per_s"], "unit": "jobs/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": args.precision, "data": "synthetic (seeded molecules and solids)",
            "config": {"workload": "scgw_job_stream", "jobs": s["jobs"], "precision": args.precision},
            "serving": s, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def _event_ms(stream, fn, steps):
    """Average CUDA-event time of fn() over steps calls on stream, after one untimed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_loop(args, rank, local_rank):
    """One JSON line for the self-consistency loop of Sec. 2.4 on the bench workload: iterations/s
    of gw_scgw (static part, GW self-energy, DIIS over five vectors, Dyson) and the cost of each
    piece beside the self-energy evaluation (rank 0; other ranks exit)."""
    import torch
    from paper_2406_18479_gb300 import gw, inputs as I
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    w = I.WORKLOADS[args.workload]
    h, v, g = I.make_inputs(w)
    V, G0, H = (torch.from_numpy(x).cuda() for x in (v, g, h))
    ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=args.precision, tau_chunk=args.tau_chunk)
    gw.gw_set_coulomb(ctx, V)
    st = ctx.stream
    Sig = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    Sinf = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    Gw = torch.empty_like(G0)
    e = torch.empty((w.nk, ctx.nwf, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    pieces = {}
    with ClockSampler(local_rank) as clk:
        pieces["sigma_eval"] = _event_ms(st, lambda: gw.gw_sigma_eval(ctx, G0, Sig), 2)
        pieces["sigma_inf"] = _event_ms(st, lambda: gw.gw_sigma_inf(ctx, G0, Sinf), 3)
        pieces["dyson"] = _event_ms(st, lambda: gw.gw_dyson_G(ctx, H, Sig, Gw), 3)
        pieces["commutator_residual"] = _event_ms(st, lambda: gw.gw_commutator_residual(ctx, H, Sinf, Sig, G0, e), 3)
        gw.gw_dyson_G(ctx, H, Sig, Gw)
        n1 = gw.gw_particle_number(ctx, Gw)
        t0 = time.perf_counter()
        gw.gw_find_mu(ctx, H, Sig, n1, -1.0, 1.0, 1e-10, Gw)
        pieces["find_mu"] = (time.perf_counter() - t0) * 1e3
        gw.gw_set_mu(ctx, w.mu)
        n = w.nk * w.nao * w.nao * (1 + w.ntau)
        d = gw.gw_diis(n, 5, stream=st)
        pairs = [(torch.randn(n, dtype=torch.complex128, device="cuda"),
                  torch.randn(n, dtype=torch.complex128, device="cuda")) for _ in range(6)]
        out = torch.empty(n, dtype=torch.complex128, device="cuda")
        t0 = time.perf_counter()
        for a, b in pairs:
            d.push(a, b)
            d.extrapolate(out)
        torch.cuda.synchronize()
        pieces["diis_push_extrapolate"] = (time.perf_counter() - t0) * 1e3 / len(pairs)
        d.destroy()
        iters = max(2, args.steps)
        opt = gw.scgw_options(alpha=0.5, tol=0.0, itermax=iters, static_part=True, diis_size=5)
        Gl = G0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, r = gw.gw_scgw(ctx, H, Gl, Sig, Sinf, opt)
        loop_s = time.perf_counter() - t0
    ctx.destroy()
    line = {"metric": "scGW iterations/s (static part, GW self-energy, DIIS, Dyson; Sec. 2.4)",
            "value": r["iterations"] / loop_s, "unit": "iterations/s", "n_gpus": 1, "steps": iters,
            "warmup": 1, "ms_per_step": loop_s * 1e3 / r["iterations"], "higher_is_better": True,
            "dtype": args.precision, "data": "synthetic (seeded H(k), V, G0 shaped like the paper's Si example)",
            "config": {"workload": w.name, "precision": args.precision, "diis_size": 5, "static_part": True},
            "pieces_ms": pieces, "loop_status": rc, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def gf2_exchange_flops(nao, naux, ntau, nk=1):
    """FP64 flops of the GF2 exchange as contracted: (2 nao^4 naux + nao^5) complex MACs per
    (k, k1, k2, tau), 8 real flops each."""
    return 8.0 * nk ** 3 * ntau * (2.0 * nao ** 4 * naux + nao ** 5)


def run_gf2(args, rank, local_rank):
    """One JSON line for the second-order self-energy (Eq. sigma2) on a molecule (nk = 1,
    naux = 4 nao, 80 tau nodes, beta = 100): evaluations/s, with the FP64 exchange's rate
    against the FP64 pipe (rank 0; other ranks exit)."""
    import torch
    from paper_2406_18479_gb300 import gw, inputs as I
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    w = I.molecule(f"molecule_nao{args.gf2_nao}", args.gf2_nao, ntau=80, beta=100.0, seed=4)
    h, v, g = I.make_inputs(w)
    V, G0 = torch.from_numpy(v).cuda(), torch.from_numpy(g).cuda()
    ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=args.precision)
    gw.gw_set_coulomb(ctx, V)
    st = ctx.stream
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    steps = max(1, args.steps)
    with ClockSampler(local_rank) as clk:
        ms = _event_ms(st, lambda: gw.gw_gf2_self_energy(ctx, G0, S), steps)
        gw.gw_synchronize(ctx)
        gw.gw_profile_enable(ctx, True)
        ms_x = _event_ms(st, lambda: gw.gw_gf2_exchange(ctx, G0, S), steps)
        prof = gw.gw_profile_read(ctx)
        gw.gw_profile_enable(ctx, False)
        ms_gw = _event_ms(st, lambda: gw.gw_sigma_eval(ctx, G0, S), steps)
    ctx.destroy()
    fx = gf2_exchange_flops(w.nao, w.naux, w.ntau)
    # the exchange's dominant kernel class by device time: the FP64 GEMMs or the tensor-core products
    slots = {k: x for k, x in prof.items() if k in ("gf2_exchange_fp64", "gf2_outer_tc")}
    dname, d = max(slots.items(), key=lambda kv: kv[1]["ms"])
    per_launch = d["ms"] / d["launches"]
    achieved = d["flops"] / d["launches"] / (per_launch * 1e-3) / 1e12
    if dname == "gf2_outer_tc":
        peaks, peak_src = measured_peaks()
        bound, peak, peak_note = "tensor", peaks["bf16_tflops_sustained"], f"bf16 dense sustained ({peak_src})"
    else:
        peak, peak_note = fp64_peak_tflops()
        bound, peak_note = "alu", "FP64: " + peak_note
    line = {"metric": "GF2 self-energy evaluations/s (Eq. sigma2)", "value": 1e3 / ms, "unit": "sigma_evals/s",
            "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": ms, "higher_is_better": True,
            "dtype": {"fp64": "c128 (f64)",
                      "bf16x4": "bf16 slices for the direct term and the exchange's nao^4 naux products, "
                                "f64 for the rest"}[args.precision],
            "data": "synthetic (seeded molecule)",
            "config": {"workload": w.name, "nao": w.nao, "naux": w.naux, "ntau": w.ntau, "beta": w.beta,
                       "precision": args.precision},
            "exchange_ms": ms_x, "exchange_tflops_algorithmic": fx / (ms_x * 1e-3) / 1e12,
            "gw_sigma_eval_ms": ms_gw,
            # profiled over the untimed first call and the timed ones
            "exchange_kernels_ms_per_call": {k: round(x["ms"] / (steps + 1), 3) for k, x in prof.items()},
            "roofline": {"kernel": dname, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_note},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16x4", "bf16x3", "fp64"], default=None,
                    help="bf16x4: four bf16 slices per operand (bf16x3 is its former name)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false",
                    help="skip the one FP64 evaluation that gives the mixed/FP64 speed-up and max|dSigma|")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--tau-chunk", type=int, default=0, help="tau nodes per contraction batch (0: automatic)")
    ap.add_argument("--slice-pass", action="store_true",
                    help="slice every GEMM operand in a separate pass (no slice-output epilogues)")
    ap.add_argument("--serving-jobs", type=int, default=12,
                    help="jobs of the scGW stream measured beside the main line (0: none)")
    ap.add_argument("--serving", action="store_true",
                    help="measure only the scGW job stream and print its own line")
    ap.add_argument("--serving-max-tflop", type=float, default=None,
                    help="leave out stream jobs above this many TFLOP per evaluation")
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-fp64-max-tflop", type=float, default=0.5,
                    help="jobs of the serving sample compared in mixed and FP64: at most this many TFLOP per evaluation")
    ap.add_argument("--batched", action="store_true",
                    help="measure only the 48-molecule batch (loop vs streams vs graph) and print its own line")
    ap.add_argument("--batch-streams", type=int, default=8)
    ap.add_argument("--no-batched", dest="batched_default", action="store_false",
                    help="leave the 48-molecule batch out of the default line")
    ap.add_argument("--v-packed", action="store_true",
                    help="pass V packed (pairs k1 <= k2 only) to the library")
    ap.add_argument("--ir-lambda", type=float, default=0.0,
                    help="run the workload on an IR grid with this Lambda (0: the workload's Chebyshev grid)")
    ap.add_argument("--ir-eps", type=float, default=1e-10)
    ap.add_argument("--loop", action="store_true",
                    help="measure only the self-consistency loop (gw_scgw and its pieces) and print its own line")
    ap.add_argument("--gf2", action="store_true",
                    help="measure only the second-order self-energy on a molecule and print its own line")
    ap.add_argument("--gf2-nao", type=int, default=26)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.precision is None or args.precision == "bf16x3":
        args.precision = "bf16x4"
    if args.steps is None:
        if args.precision == "fp64":
            args.steps = 2
        elif args.batched or args.loop or args.gf2:
            args.steps = 3
        else:
            # about a minute of timed work: 2 steps of a 4x4x4 solid (~43 s each), 10 of smaller ones
            from paper_2406_18479_gb300 import inputs as I
            w = I.WORKLOADS.get(args.workload)
            big = w is not None and sum(stage_flops(w.nk3, w.nao, w.naux, w.ntau).values()) > 1e15
            args.steps = 2 if big else 10
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.batched:
        run_batched(args, rank, local_rank)
    elif args.serving:
        run_serving(args, rank, local_rank)
    elif args.loop:
        run_loop(args, rank, local_rank)
    elif args.gf2:
        run_gf2(args, rank, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
