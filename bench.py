#!/usr/bin/env python
"""Benchmark: sigma_min grid points per second on the dense complex Gaussian
workload (n = 2000, entries N(0, 1/n) in real and imaginary parts, seed 2;
200 x 200 grid over [-1.5, 1.5]^2; Schur factor prepared on the host and not
timed), with the accuracy of the timed run checked against stored oracle
values (rel err <= 1e-8 under the pass rule of tests/parity.py).

One step = one pseudo_grid call over all 40,000 points with the shift-
batched inverse Lanczos path in mixed precision (tensor-core solves and
double-single-accurate refinement residuals, FP64 fallback for the points
that need it).  The timed region is bracketed by barriers + device
synchronisation; L2 is flushed (256 MB write) between timed steps.  Also
reported: the end-to-end number through the host-buffer C-ABI call, the
roofline of the dominant kernel from per-kernel CUDA-event times, the
recycled Rayleigh--Ritz-SVD path (k = 16, r = 4; mixed and FP64) on the full
grid, the plain FP64 inverse Lanczos (shift-batched and per point) on
samples of the grid, and the CPU oracle on a bounded sample.  Under torchrun
every rank runs its own copy of the workload (independent replicas, weak
scaling); the step time is the maximum over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload multi [--matrices M]   # many matrices through pseudo_grid_batch
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "sigma_min grid points/sec at rel err <= 1e-8 vs FP64 oracle"
WORKLOAD = "dense complex Gaussian n=2000 (seed 2), 200x200 grid over [-1.5,1.5]^2"
GOLDEN = ROOT / "tests" / "golden" / "gaussian2000_samples.json"


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "fallback": True}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def make_workload():
    from paper_2606_26785_b300 import workloads

    t0 = time.time()
    W = workloads.make("gaussian")
    return W, time.time() - t0


def check_accuracy(sigma, W):
    """Compare the sampled points with the stored oracle values."""
    from tests.parity import check_sigma

    g = json.loads(GOLDEN.read_text())
    idx = np.array(g["index"])
    ref = np.array(g["sigma_ref"])
    rep = check_sigma(np.asarray(sigma)[idx], ref, n=W.n, fro=g["fro_norm"], schur_err=W.schur_err,
                      oracle_off=np.array(g["oracle_off"]), rtol=1e-8)
    return rep


def _nominal_fp32_tflops(peaks):
    """FP32 FMA pipe: 148 SMs x 128 lanes x 2 flops x max SM clock."""
    return 148 * 128 * 2 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6 / 1e12


N_BENCH = 2000
FP64_MEASURED_TFLOPS = 1.13  # B300 FP64 FMA rate measured with independent DFMA chains on all SMs


def _tf32x3_tflops(peaks):
    """Effective FP32-product rate of the tensor-core solve: the measured
    sustained bf16 GEMM rate x the nominal TF32 / bf16 ratio (1.1 / 2.25 dense),
    divided by the 3 TF32 products (hi*hi + hi*lo + lo*hi) that stand in for one
    FP32 product."""
    bf16 = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1800.0) * 0.78))
    return bf16 * (1.1 / 2.25) / 3.0


# DRAM bytes (read + write) per column of a launch, from one ncu capture of each
# tensor-core kernel on 4,096 columns of the bench matrix (bench.py
# --profile-kernel solve|product); traffic grows with the columns of a launch
# (A re-reads per column tile, B images per column group).
DRAM_BYTES_PER_COLUMN = {"trsv32": (1.694567e9 + 0.3204608e9) / 4096, "trmv_ds": (1.939070e9 + 0.111231e9) / 4096}


def roofline(kst, peaks, tensor_solve=True):
    """Dominant kernel class of a profiled step and its achieved rate."""
    name, k = max(kst.items(), key=lambda kv: kv[1]["ms"])
    if k["launches"] == 0 or k["ms"] <= 0:
        return None
    per_launch_ms = k["ms"] / k["launches"]
    flops = k["flops"] / k["launches"]
    fp32 = _nominal_fp32_tflops(peaks)
    if name == "trsv32" and tensor_solve:
        achieved = flops / (per_launch_ms / 1e3) / 1e12
        peak = _tf32x3_tflops(peaks)
        cols = flops / (4.0 * N_BENCH * N_BENCH)
        return {"kernel": "trsv32 (tcgen05 3xTF32)", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": DRAM_BYTES_PER_COLUMN["trsv32"] * cols, "traffic_unit": "bytes per launch (ncu, scaled)",
                "launches": k["launches"],
                "avg_launch_ms": per_launch_ms, "algorithmic_flops_per_launch": flops, "share_of_step": None,
                "peak_source": "measured cuBLAS bf16 sustained x 1.1/2.25 (TF32/bf16 nominal) / 3 (3xTF32)"}
    if name in ("trsv32",):
        peak, unit, bound = fp32, "TFLOP/s", "alu"
    elif name == "trmv_ds" and tensor_solve:
        # the double-single-accurate product on the tensor cores: 28 bf16 slice
        # products stand in for one real product
        achieved = flops / (per_launch_ms / 1e3) / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1800.0) * 0.78)) / 28.0
        cols = flops / (4.0 * N_BENCH * N_BENCH)
        return {"kernel": "trmv_ds (tcgen05 bf16 slices)", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": DRAM_BYTES_PER_COLUMN["trmv_ds"] * cols, "traffic_unit": "bytes per launch (ncu, scaled)",
                "launches": k["launches"],
                "avg_launch_ms": per_launch_ms, "algorithmic_flops_per_launch": flops, "share_of_step": None,
                "peak_source": "measured cuBLAS bf16 sustained / 28 (slice pairs per real product)"}
    elif name == "trmv_ds":
        # double-single: 12 FP32 operations per real multiply-add (2 algorithmic flops)
        peak, unit, bound = fp32 / 6.0, "TFLOP/s", "alu"
    elif name == "lanczos":
        achieved = k["bytes"] / k["launches"] / (per_launch_ms / 1e3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "launches": k["launches"],
                "avg_launch_ms": per_launch_ms, "peak_source": "measured"}
    else:
        peak, unit, bound = FP64_MEASURED_TFLOPS, "TFLOP/s", "alu"
    achieved = flops / (per_launch_ms / 1e3) / 1e12
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": None, "launches": k["launches"], "avg_launch_ms": per_launch_ms,
            "algorithmic_flops_per_launch": flops, "share_of_step": None,
            "peak_source": "derived from 148 SMs x 128 FP32 lanes x max clock" if name in ("trsv32", "trmv_ds")
            else "measured FP64 DFMA probe"}


def cpu_baseline(W, budget_points=1):
    import oracle

    threads = os.cpu_count() or 1
    rng = np.random.Generator(np.random.PCG64(11))
    idx = rng.choice(W.z.size, size=budget_points, replace=False)
    t0 = time.time()
    oracle.sigma_min_grid(W.C, W.z[idx], threads=threads)
    dt = time.time() - t0
    return {"value": budget_points / dt, "unit": "points/s", "cores": threads, "kind": "oracle",
            "sample": f"{budget_points} grid point(s) of the same workload, one-sided Jacobi SVD of the n=2000 "
                      f"C - zI using all {threads} host threads inside the point; {dt:.1f} s"}


def max_over_ranks(ms, dist, device):
    """Step time of the whole job: the slowest rank's (every rank passes its
    own mean step time; dist is None in a single-process run)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank, world, ms):
    """Whole-job points/s: the points all ranks processed over the job's step
    time in milliseconds."""
    return points_per_rank * world / (ms / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="invlanc", choices=["recycle", "invlanc"],
                    help="method timed as the main line (the other one is reported under comparisons)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-extras", action="store_true", help="skip the comparison paths and the CPU baseline")
    ap.add_argument("--profile-kernel", choices=["solve", "product"],
                    help="for kernel profilers: 3 warm-up calls then 1 timed call of the tensor-core solve or the "
                         "tensor-core double-single-accurate product on 4096 columns of the bench matrix")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for profilers: mixed inverse Lanczos on 4096 grid points, one untimed run")
    ap.add_argument("--workload", default="gaussian2000", choices=["gaussian2000", "multi"],
                    help="multi: the multi-matrix workload through pseudo_grid_batch (one GPU, its own JSON line)")
    ap.add_argument("--matrices", type=int, default=16, help="with --workload multi: how many of the 64 matrices")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "multi":
        return run_multi(args)

    import torch

    import paper_2606_26785_b300 as p

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    W, t_schur = make_workload()
    h = p.Pseudo(W.T)
    if args.profile_kernel:
        rng = np.random.default_rng(0)
        ncols = 4096
        X0 = torch.from_numpy(rng.standard_normal((W.n, ncols)) + 1j * rng.standard_normal((W.n, ncols))).cuda()
        zk = torch.from_numpy(W.z[::9][:ncols].copy()).cuda()

        def call():
            if args.profile_kernel == "solve":
                X = X0.clone()
                h.solve(X, zk, adjoint=False, precision=p.MIXED)
            else:
                h.matvec(X0, z=zk, precision=p.MIXED)

        for _ in range(3):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile_kernel": args.profile_kernel, "columns": ncols, "workload": WORKLOAD,
                          "ms_incl_conversions": e0.elapsed_time(e1)}))
        return
    if args.profile_case:
        zs = torch.from_numpy(W.z[::9][:4096].copy()).cuda()
        o = p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8, maxiter_lanczos=32)
        h.grid(zs[:64], (), opts=o)
        torch.cuda.synchronize()
        h.grid(zs, (), opts=o)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "invlanc mixed, 4096 points of " + WORKLOAD, "stats": h.stats()}))
        return
    prec = p.MIXED if args.precision == "mixed" else p.FP64
    rtol = 1e-8 if prec == p.MIXED else 1e-10
    if args.mode == "recycle":
        opts = p.default_opts(mode=p.RECYCLE, precision=prec, r=4, p_max=4, grid_nx=W.nx, grid_ny=W.ny,
                              batch_b=20, rtol=rtol)
    else:
        opts = p.default_opts(mode=p.INVLANC, precision=prec, rtol=rtol)
    z = torch.from_numpy(W.z).cuda()
    need = h.workspace_bytes(W.z.size, opts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    eps = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10)

    def step():
        return h.grid(z, eps, opts=opts, workspace=ws)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    h.reset_stats()
    times = []
    clocks = Clocks(os.environ.get("PSEUDO_BENCH_CLOCKS_CSV", os.path.join(tempfile.gettempdir(), "bench_clocks.csv")))
    lc0 = p._abi.load().pseudo_launch_count()
    with clocks:
        for _ in range(args.steps):
            flush.zero_()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = step()
            e1.record()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            times.append(e0.elapsed_time(e1))
    launches = p._abi.load().pseudo_launch_count() - lc0
    ms = float(np.mean(times))
    ms = max_over_ranks(ms, dist, "cuda")
    st = h.stats()
    sigma = out["sigma"].cpu().numpy()
    acc = check_accuracy(sigma, W)
    npts = W.z.size
    value = job_throughput(npts, world, ms)
    peaks = _peaks()

    # one profiled step: per-kernel CUDA-event times on the launching stream
    h.reset_stats()
    opts.profile = 1
    step()
    torch.cuda.synchronize()
    opts.profile = 0
    kst = h.kernel_stats()
    prof_ms = h.stats()["ms_total"]
    rf = roofline(kst, peaks, tensor_solve=opts.fp32_solver == 0)
    if rf is not None:
        rf["share_of_step"] = max(kst.values(), key=lambda v: v["ms"])["ms"] / max(prof_ms, 1e-9)

    # end to end through the host-buffer C-ABI call (z in, results out, copies inside)
    zpin = torch.from_numpy(W.z.copy()).pin_memory().numpy()
    outs = {"sigma": torch.empty(npts, dtype=torch.float64).pin_memory().numpy(),
            "res": torch.empty(npts, dtype=torch.float64).pin_memory().numpy(),
            "flags": torch.empty(npts, dtype=torch.int32).pin_memory().numpy(),
            "member": torch.empty(npts, dtype=torch.int32).pin_memory().numpy().view(np.uint32)}
    hopts = p.Opts.from_buffer_copy(opts)
    hopts.io_host = 1
    del ws
    e2e_ws = torch.empty(h.workspace_bytes(npts, hopts), dtype=torch.uint8, device="cuda")
    h.grid_host(zpin, eps, opts=hopts, workspace=e2e_ws, out=outs)
    e2e_t = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.grid_host(zpin, eps, opts=hopts, workspace=e2e_ws, out=outs)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(float(np.mean(e2e_t)) * 1e3, dist, "cuda")
    e2e = {"value": job_throughput(npts, world, e2e_ms), "unit": "points/s",
           "h2d_bytes_per_step": int(npts * 16 * world), "d2h_bytes_per_step": int(npts * (8 + 8 + 4 + 4) * world)}

    extras = {}
    cpu = None
    if not args.no_extras and rank == 0:
        def full_grid(name, o2, rtol2):
            need2 = h.workspace_bytes(npts, o2)
            ws2 = torch.empty(need2, dtype=torch.uint8, device="cuda")
            h.reset_stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            o = h.grid(z, eps, opts=o2, workspace=ws2)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st2 = h.stats()
            extras[name] = {"points": npts, "points_per_s": npts / dt, "seconds": dt,
                            "accuracy": check_accuracy_rtol(o["sigma"].cpu().numpy(), W, rtol2),
                            "accepted": st2["n_accepted"], "refined": st2["n_refined"]}
            del ws2

        other = "recycle" if args.mode == "invlanc" else "invlanc"
        if other == "recycle":
            full_grid("recycle_mixed_k16", p.default_opts(mode=p.RECYCLE, precision=p.MIXED, r=4, p_max=4, grid_nx=W.nx,
                                                          grid_ny=W.ny, batch_b=20, rtol=1e-8), 1e-8)
        else:
            full_grid("invlanc_mixed", p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8), 1e-8)
        full_grid("recycle_fp64_k16", p.default_opts(mode=p.RECYCLE, precision=p.FP64, r=4, p_max=4, grid_nx=W.nx,
                                                     grid_ny=W.ny, batch_b=20, rtol=1e-10), 1e-10)
        # plain FP64 inverse Lanczos (the per-point baseline and its shift-batched form) on bounded samples
        sub = torch.from_numpy(W.z[::20].copy()).cuda()
        for name, kw, zz in (
            ("invlanc_fp64_batched", dict(mode=p.INVLANC, precision=p.FP64, rtol=1e-10), sub),
            ("invlanc_fp64_per_point", dict(mode=p.INVLANC, precision=p.FP64, rtol=1e-10, shift_batch=1), sub[:8]),
        ):
            o2 = p.default_opts(**kw)
            h.grid(zz[:4], eps, opts=o2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.grid(zz, eps, opts=o2)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            extras[name] = {"points": int(zz.numel()), "points_per_s": zz.numel() / dt, "sample": "every 20th grid point"}
        cpu = cpu_baseline(W)

    result = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if prec == p.MIXED else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": args.mode, "precision": args.precision, "k": 16, "r": 4,
                   "batch_b": 20, "points": npts, "l2": "flushed (256 MB write) between timed steps",
                   "schur_seconds_host_untimed": t_schur},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": rf,
        "cpu_baseline": cpu,
        "clocks": clocks.summary(),
        "accuracy": acc,
        "counters_per_step": {k: (v / max(1, args.steps)) for k, v in st.items()},
        "kernels_profiled_step": kst,
        "comparisons": extras,
    }
    if rank == 0:
        print(json.dumps(result))


def check_accuracy_rtol(sigma, W, rtol):
    from tests.parity import check_sigma

    g = json.loads(GOLDEN.read_text())
    idx = np.array(g["index"])
    return check_sigma(np.asarray(sigma)[idx], np.array(g["sigma_ref"]), n=W.n, fro=g["fro_norm"],
                       schur_err=W.schur_err, oracle_off=np.array(g["oracle_off"]), rtol=rtol)


BATCH_GOLDEN = ROOT / "tests" / "golden" / "batch16_samples.json"


def run_multi(args):
    """The multi-matrix workload: independent complex Gaussian matrices
    N(0, 1/n), n log-uniform in [256, 2048] (seed 40), each on its own 64 x 64
    grid over [-1.5, 1.5]^2; the first --matrices of its sequence (host Schur
    factors not timed).  One step = one pseudo_grid_batch call over all of
    them in mixed precision; the same matrices one after another with
    pseudo_grid are timed beside it.  Accuracy: the stored oracle values of
    the 8 smallest of the first 16 matrices."""
    import torch

    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import workloads
    from tests.parity import check_sigma

    nm = args.matrices
    t0 = time.time()
    mats = workloads.gaussian_batch(64, 40)[:nm]
    Ts, errs = [], []
    for C in mats:
        T, _, e = workloads.schur(C)
        Ts.append(T)
        errs.append(e)
    t_prep = time.time() - t0
    sizes = [C.shape[0] for C in mats]
    zh = workloads.grid(-1.5, 1.5, -1.5, 1.5, 64, 64)
    z = torch.from_numpy(zh).cuda()
    hs = [p.Pseudo(T) for T in Ts]
    opts = p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    eps = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10)
    npts = nm * zh.size

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    for _ in range(args.warmup):
        outs, _ = p.grid_batch(hs, [z] * nm, eps, opts=opts)
    lc0 = p._abi.load().pseudo_launch_count()
    t_batch = [timed(lambda: p.grid_batch(hs, [z] * nm, eps, opts=opts)) for _ in range(args.steps)]
    launches = (p._abi.load().pseudo_launch_count() - lc0) // max(1, args.steps)
    outs = t_batch[-1][1][0]
    ms = float(np.mean([t for t, _ in t_batch]))
    ms_seq = float(np.mean([timed(lambda: [h.grid(z, eps, opts=opts) for h in hs])[0]
                            for _ in range(max(1, min(2, args.steps)))]))
    acc = None
    if BATCH_GOLDEN.exists():
        g = json.loads(BATCH_GOLDEN.read_text())
        smp = [s_ for s_ in g["samples"] if s_["matrix"] < nm]
        m0 = min(nm, g["count"])
        if smp and g["sizes"][:m0] == sizes[:m0]:
            got = np.array([outs[s_["matrix"]]["sigma"][s_["index"]].item() for s_ in smp])
            bad = 0
            worst = 0.0
            for v, s_ in zip(got, smp):
                rep = check_sigma(np.array([v]), np.array([s_["sigma_ref"]]), n=s_["n"], fro=s_["fro_norm"],
                                  schur_err=errs[s_["matrix"]], oracle_off=np.array([s_["oracle_off"]]), rtol=1e-8)
                bad += rep["n_bad"]
                worst = max(worst, abs(v - s_["sigma_ref"]) / s_["sigma_ref"])
            acc = {"n_points": len(smp), "n_bad": int(bad), "max_rel_err": worst}
    print(json.dumps({
        "metric": METRIC, "value": npts / (ms / 1e3), "unit": "points/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64+f32",
        "data": "synthetic", "gpu_launches": int(launches),
        "config": {"workload": f"multi-matrix: first {nm} of 64 complex Gaussian matrices N(0,1/n), "
                               "n log-uniform in [256,2048] (seed 40), 64x64 grid each over [-1.5,1.5]^2",
                   "sizes": sizes, "points": npts, "host_schur_s": t_prep},
        "sequential_pseudo_grid": {"ms": ms_seq, "points_per_s": npts / (ms_seq / 1e3)},
        "accuracy": acc}))


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands (one-sided Jacobi SVD of
    C - zI) on a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle

    W, _ = make_workload()
    threads = os.cpu_count() or 1
    rng = np.random.Generator(np.random.PCG64(11))
    idx = rng.choice(W.z.size, size=threads, replace=False)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.time()
        oracle.sigma_min_grid(W.C, W.z[idx[:1]], threads=threads)
        if s >= args.warmup:
            times.append(time.time() - t0)
    sec = float(np.mean(times))
    v = 1.0 / sec
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
                      "higher_is_better": True, "config": {"workload": WORKLOAD},
                      "cpu_baseline": {"kind": "oracle", "cores": threads, "value": v, "unit": "points/s",
                                       "sample": "1 grid point per step, all host threads inside the point"},
                      "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    main()
