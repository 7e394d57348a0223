#!/usr/bin/env python
"""Benchmark: sigma_min grid points per second on the strongly nonnormal
upper-triangular workload (T given, its own Schur factor: n = 8000, diagonal
uniform in the unit disk, strictly upper part 3 (A + iB) / sqrt(n) with A, B
iid N(0, 1), seed 3; 300 x 300 grid over [-1.5, 1.5]^2), with the accuracy of
the timed run checked against stored oracle values (tests/golden/
triangular8000_samples.json, rel err <= 1e-8 under the pass rule of
tests/parity.py) and against the FP64 path on a sample of the grid.

One step = one pseudo_grid call over one of 20 strided batches of the grid
(4,500 points; 20 consecutive steps cover all 90,000 points once) with the
shift-batched inverse Lanczos path in mixed precision (tensor-core solves and
double-single-accurate refinement residuals, FP64 fallback for the points
that need it), its loop decided on the device (one CUDA graph per call).  The timed region is bracketed by barriers + device
synchronisation; L2 is flushed (256 MB write) between timed steps.  Also
reported: the end-to-end number through the host-buffer C-ABI call, the
roofline of the dominant kernel from per-kernel CUDA-event times, the plain
FP64 inverse Lanczos (shift-batched and per point) on samples of the grid,
the dense complex Gaussian workload (n = 2000) in mixed precision, the
64-matrix workload through pseudo_grid_batch, FP64 inverse Lanczos on
rectangular pencils (m >= 2n, one QR per point), the recycled Rayleigh--Ritz-
SVD path on a banded Toeplitz + noise matrix next to inverse Lanczos, and the
CPU oracle on a bounded sample.  Under torchrun
every rank runs its own copy of the workload (independent replicas, weak
scaling); the step time is the maximum over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload gaussian2000        # the dense Gaussian n = 2000 line
    python bench.py --workload multi [--matrices M]   # many matrices through pseudo_grid_batch
    python bench.py --accuracy-full                # also compare with FP64 at every grid point
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
WORKLOADS = {
    "triangular8000": ("upper-triangular complex T n=8000 (seed 3), diagonal uniform in the unit disk, strictly "
                       "upper 3(A+iB)/sqrt(n); 300x300 grid over [-1.5,1.5]^2",
                       ROOT / "tests" / "golden" / "triangular8000_samples.json"),
    "gaussian2000": ("dense complex Gaussian n=2000 (seed 2), 200x200 grid over [-1.5,1.5]^2",
                     ROOT / "tests" / "golden" / "gaussian2000_samples.json"),
}
# a timing sample of the oracle at n = 8000: the first rounds of its Jacobi
# iteration (one round = n/2 disjoint column-pair rotations) at one grid point
ORACLE_ROUNDS_SAMPLE = 96


T_START = time.time()


def log(msg):
    """Progress on stderr (the JSON result line goes to stdout)."""
    sys.stderr.write(f"[bench {time.time() - T_START:7.1f} s] {msg}\n")
    sys.stderr.flush()


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


def make_workload(name):
    from paper_2606_26785_b300 import workloads

    t0 = time.time()
    W = workloads.make("triangular" if name == "triangular8000" else "gaussian")
    return W, time.time() - t0


def check_accuracy(sigma, W, golden, rtol=1e-8, member=None):
    """Compare the sampled points with the stored oracle values."""
    from tests.parity import check_sigma

    if not golden.exists():
        return {"n_points": 0, "note": f"{golden.name} not present"}
    g = json.loads(golden.read_text())
    idx = np.array(g["index"])
    ref = np.array(g["sigma_ref"])
    kw = {}
    if member is not None:
        from paper_2606_26785_b300 import workloads

        kw = dict(eps_levels=workloads.EPS_LEVELS, member=np.asarray(member)[idx])
    rep = check_sigma(np.asarray(sigma)[idx], ref, n=W.n, fro=g["fro_norm"], schur_err=W.schur_err,
                      oracle_off=np.array(g["oracle_off"]), rtol=rtol, **kw)
    rep["source"] = golden.name
    return rep


def compare_with_fp64(sig, s64, fro, n, rtol=1e-8, member=None, member64=None, eps_levels=()):
    """Mixed against the GPU FP64 path at the same points: |a - b| <= rtol a +
    4 n eps ||T||_F where a >= 1e-8 ||T||_F, and |a - b| <= rtol a alone where
    a >= 1e-6 ||T||_F; membership bits equal except inside a level's band."""
    sig, s64 = np.asarray(sig), np.asarray(s64)
    atol = 4.0 * n * 2.220446049250313e-16 * fro
    incl, rel_only = s64 >= 1e-8 * fro, s64 >= 1e-6 * fro
    err = np.abs(sig - s64)
    bad = (incl & ~(err <= rtol * s64 + atol)) | (rel_only & ~(err <= rtol * s64))
    rep = {"n_points": int(sig.size), "n_included": int(incl.sum()), "n_rel_only": int(rel_only.sum()),
           "n_bad": int(bad.sum()), "atol": atol,
           "max_rel_err_included": float((err[incl] / s64[incl]).max()) if incl.any() else 0.0,
           "max_rel_err_rel_only": float((err[rel_only] / s64[rel_only]).max()) if rel_only.any() else 0.0}
    if member is not None and member64 is not None:
        band = rtol * s64 + atol
        mm = 0
        for i, e in enumerate(eps_levels):
            a = (np.asarray(member).astype(np.uint32) >> np.uint32(i)) & 1
            b = (np.asarray(member64).astype(np.uint32) >> np.uint32(i)) & 1
            mm += int(((a != b) & (np.abs(s64 - e) > band)).sum())
        rep["member_mismatch"] = mm
    return rep


# Arithmetic rates of this machine's B300 measured by paper_2606_26785_b300/probe/peaks.cu
# (python -m paper_2606_26785_b300.probe.peaks): FP64 FMA 1.010, FP64 tensor-core MMA
# (m8n8k4) 1.053 and FP32 FMA 73.48 TFLOP/s.  The FP64 roofline is the larger FP64 rate.
FP64_MEASURED_TFLOPS = 1.053
FP32_MEASURED_TFLOPS = 73.48
# double-single on the FP32 units: 44 FP32 instructions per complex multiply-add
# (8 algorithmic flops) in the solve, 12 per real multiply-add (2 flops) in the product
DS_SOLVE_TFLOPS = FP32_MEASURED_TFLOPS / 2.0 * 8.0 / 44.0


def _nominal_fp32_tflops(peaks):
    """FP32 FMA pipe as measured (probe above)."""
    return FP32_MEASURED_TFLOPS


def _tf32x3_tflops(peaks):
    """Effective FP32-product rate of the tensor-core solve: the measured
    sustained bf16 GEMM rate x the nominal TF32 / bf16 ratio (1.1 / 2.25 dense),
    divided by the 3 TF32 products (hi*hi + hi*lo + lo*hi) that stand in for one
    FP32 product."""
    bf16 = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1800.0) * 0.78))
    return bf16 * (1.1 / 2.25) / 3.0


# DRAM bytes (read + write) per column of a launch, from one ncu capture of each
# tensor-core kernel on 4,096 columns (bench.py --profile-kernel solve|product
# [--profile-n 4000]); traffic grows with the columns of a launch (A re-reads
# per column group, B images per column group).  n = 2000: the narrow solve
# (16 columns per CTA) and the product on the Gaussian matrix.  n = 8000: the
# wide solve (32 columns per CTA) captured on the leading 4000 x 4000 block of
# the triangular matrix and scaled by (8000 / 4000)^2, the growth of the A
# stream every CTA reads; a lower estimate, since the larger A misses L2 more.
DRAM_BYTES_PER_COLUMN = {("trsv32", 2000): (1.694567e9 + 0.3204608e9) / 4096,
                         ("trmv_ds", 2000): (1.939070e9 + 0.111231e9) / 4096,
                         ("trsv32", 8000): (8.017367296e9 + 0.663716864e9) / 4096 * 4.0}


def _traffic(kernel, n, cols):
    per = DRAM_BYTES_PER_COLUMN.get((kernel, n))
    return None if per is None else per * cols


def roofline(kst, peaks, n, tensor_solve=True):
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
        cols = flops / (4.0 * n * n)
        return {"kernel": "trsv32 (tcgen05 3xTF32)", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": _traffic("trsv32", n, cols), "traffic_unit": "bytes per launch (ncu, scaled)",
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
        cols = flops / (4.0 * n * n)
        return {"kernel": "trmv_ds (tcgen05 bf16 slices)", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": _traffic("trmv_ds", n, cols), "traffic_unit": "bytes per launch (ncu, scaled)",
                "launches": k["launches"],
                "avg_launch_ms": per_launch_ms, "algorithmic_flops_per_launch": flops, "share_of_step": None,
                "peak_source": "measured cuBLAS bf16 sustained / 28 (slice pairs per real product)"}
    elif name == "trmv_ds":
        # double-single: 12 FP32 operations per real multiply-add (2 algorithmic flops)
        peak, unit, bound = fp32 / 6.0, "TFLOP/s", "alu"
    elif name == "trsv_ds":
        peak, unit, bound = DS_SOLVE_TFLOPS, "TFLOP/s", "alu"
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
            "peak_source": {"trsv32": "measured FP32 FMA rate (probe)",
                            "trmv_ds": "measured FP32 FMA rate / 6 (12 FP32 instructions per real multiply-add)",
                            "trsv_ds": "measured FP32 FMA rate / 2 x 8 / 44 (FP32 instructions per complex "
                                       "multiply-add of the double-single solve)"}.get(
                name, "measured FP64 rate (tensor-core MMA, probe)")}


def oracle_sample(W, workload, threads):
    """Time the oracle as it stands on a bounded sample of the workload and
    scale it to points/s.  Gaussian n = 2000: one whole grid point.
    Triangular n = 8000 (a point takes over an hour): the first
    ORACLE_ROUNDS_SAMPLE rounds of the Jacobi iteration at one grid point,
    scaled by the rounds a whole point takes there (sweeps recorded by the
    stored oracle run x (n - 1) rounds per sweep)."""
    import oracle

    rng = np.random.Generator(np.random.PCG64(11))
    i = int(rng.choice(W.z.size))
    if workload != "triangular8000":
        t0 = time.time()
        oracle.sigma_min_grid(W.C, W.z[[i]], threads=threads)
        dt = time.time() - t0
        return 1.0 / dt, dt, f"1 grid point of the same workload, one-sided Jacobi SVD of the n={W.n} C - zI " \
                             f"using {threads} host threads inside the point; {dt:.1f} s"
    g = json.loads(WORKLOADS[workload][1].read_text()) if WORKLOADS[workload][1].exists() else {}
    sweeps = float(np.median(g["oracle_sweeps"])) if g.get("oracle_sweeps") else None
    t0 = time.time()
    oracle.jacobi_rounds(W.C, W.z[i], ORACLE_ROUNDS_SAMPLE, threads=threads)
    dt = time.time() - t0
    if sweeps is None:
        return None, dt, "sweep count of a whole point unknown (no stored oracle run)"
    per_point = dt / ORACLE_ROUNDS_SAMPLE * sweeps * (W.n - 1 + W.n % 2)
    return 1.0 / per_point, dt, (f"{ORACLE_ROUNDS_SAMPLE} of the {int(sweeps * (W.n - 1 + W.n % 2))} Jacobi rounds a "
                                 f"whole point takes ({sweeps:g} sweeps, from the stored oracle run) at one grid point "
                                 f"of the n={W.n} workload, {threads} host threads, {dt:.1f} s; scaled to one point")


def cpu_baseline(W, workload):
    threads = os.cpu_count() or 1
    v, dt, what = oracle_sample(W, workload, threads)
    return {"value": v, "unit": "points/s", "cores": threads, "kind": "oracle", "sample": what}


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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batches", type=int, default=20,
                    help="the grid is cut into this many strided batches (every B-th point); step i processes "
                         "batch i mod B, so B consecutive steps cover every grid point once")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-extras", action="store_true", help="skip the comparison paths and the CPU baseline")
    ap.add_argument("--recycle-ranks", default="32",
                    help="recycled ranks k of the Toeplitz recycling comparison (comma-separated; 8,32,64 for all "
                         "three, about 140 s each)")
    ap.add_argument("--extras-budget", type=float, default=480.0,
                    help="seconds of wall time the comparison paths may take; the ones that would start later are "
                         "reported as skipped")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the inverse-Lanczos loop from the host (device_loop = 0): the same kernels as plain "
                         "launches, which a kernel profiler sees one by one (it does not profile the kernels of "
                         "graphs with conditional nodes)")
    ap.add_argument("--accuracy-full", action="store_true",
                    help="also run the FP64 path on every grid point and compare (about ten minutes at n = 8000)")
    ap.add_argument("--profile-kernel", choices=["solve", "product", "solve_ds", "solve_fp64"],
                    help="for kernel profilers: 3 warm-up calls then 1 timed call of the tensor-core solve, the "
                         "tensor-core double-single-accurate product, the double-single solve or the FP64 solve on "
                         "--profile-columns columns of the matrix")
    ap.add_argument("--profile-columns", type=int, default=4096)
    ap.add_argument("--profile-n", type=int, default=0,
                    help="with --profile-kernel: a leading n x n block of the workload's matrix (0 = all of it)")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for profilers: mixed inverse Lanczos on 4096 grid points, one untimed run")
    ap.add_argument("--profile-recycle", action="store_true",
                    help="small case for profilers: the recycling path (mixed, k = 16, r = 4) on the banded Toeplitz + "
                         "noise matrix at n = 1200 on a 30 x 30 grid, one untimed run")
    ap.add_argument("--workload", default="triangular8000", choices=["triangular8000", "gaussian2000", "multi"],
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
    from paper_2606_26785_b300 import workloads

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.profile_recycle:
        from paper_2606_26785_b300 import workloads as wl

        T, _, _ = wl.schur(wl.toeplitz_noisy(1200, 5))
        hr = p.Pseudo(T)
        zr = torch.from_numpy(wl.grid(-1.5, 1.5, -1.0, 1.0, 30, 30)).cuda()
        o = p.default_opts(mode=p.RECYCLE, precision=p.MIXED, rtol=1e-8, r=4, p_max=4, grid_nx=30, grid_ny=30,
                           batch_b=20)
        hr.grid(zr, (), opts=o)
        torch.cuda.synchronize()
        print(json.dumps({"profile_recycle": "toeplitz+noise n=1200, 30x30 grid, recycle mixed k=16",
                          "stats": hr.stats()}))
        return
    label, golden = WORKLOADS[args.workload]
    W, t_prep = make_workload(args.workload)
    fro = float(np.linalg.norm(W.T))
    if args.profile_kernel:
        nk = args.profile_n or W.n
        h = p.Pseudo(np.ascontiguousarray(W.T[:nk, :nk]))
        rng = np.random.default_rng(0)
        ncols = args.profile_columns
        X0 = torch.from_numpy(rng.standard_normal((nk, ncols)) + 1j * rng.standard_normal((nk, ncols))).cuda()
        zk = torch.from_numpy(W.z[:: max(1, W.z.size // ncols)][:ncols].copy()).cuda()

        solve_prec = {"solve": p.MIXED, "solve_ds": p.DOUBLE_SINGLE, "solve_fp64": p.FP64}

        def call():
            if args.profile_kernel in solve_prec:
                X = X0.clone()
                h.solve(X, zk, adjoint=False, precision=solve_prec[args.profile_kernel])
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
        print(json.dumps({"profile_kernel": args.profile_kernel, "columns": ncols, "n": nk, "workload": label,
                          "ms_incl_conversions": e0.elapsed_time(e1)}))
        return
    h = p.Pseudo(W.T)
    if args.profile_case:
        zs = torch.from_numpy(W.z[::9][:4096].copy()).cuda()
        o = p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8, maxiter_lanczos=32)
        h.grid(zs[:64], (), opts=o)
        torch.cuda.synchronize()
        h.grid(zs, (), opts=o)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "invlanc mixed, 4096 points of " + label, "stats": h.stats()}))
        return
    prec = p.MIXED if args.precision == "mixed" else p.FP64
    rtol = 1e-8 if prec == p.MIXED else 1e-10
    opts = p.default_opts(mode=p.INVLANC, precision=prec, rtol=rtol, device_loop=0 if args.host_loop else 1)
    npts = W.z.size
    NB = max(1, min(args.batches, npts))
    bidx = [np.arange(b, npts, NB) for b in range(NB)]
    zb = [torch.from_numpy(W.z[ix].copy()).cuda() for ix in bidx]
    need = max(h.workspace_bytes(ix.size, opts) for ix in bidx)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    eps = workloads.EPS_LEVELS
    sigma = np.full(npts, np.nan)
    member = np.zeros(npts, np.uint32)
    flags = np.zeros(npts, np.int32)
    done = np.zeros(NB, bool)

    def step(i):
        return h.grid(zb[i % NB], eps, opts=opts, workspace=ws)

    def keep(i, out):
        b = i % NB
        sigma[bidx[b]] = out["sigma"].cpu().numpy()
        member[bidx[b]] = out["member"].cpu().numpy().astype(np.uint32)
        flags[bidx[b]] = out["flags"].cpu().numpy()
        done[b] = True

    log(f"workload ready ({t_prep:.1f} s host prep); {NB} batches of about {npts // NB} points")
    for i in range(args.warmup):
        keep(i, step(i))
    torch.cuda.synchronize()
    log("warm-up done")
    h.reset_stats()
    times, counted = [], 0
    clocks = Clocks(os.environ.get("PSEUDO_BENCH_CLOCKS_CSV", os.path.join(tempfile.gettempdir(), "bench_clocks.csv")))
    lc0 = p._abi.load().pseudo_launch_count()
    with clocks:
        for i in range(args.warmup, args.warmup + args.steps):
            flush.zero_()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = step(i)
            e1.record()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            times.append(e0.elapsed_time(e1))
            counted += bidx[i % NB].size
            keep(i, out)
    launches = p._abi.load().pseudo_launch_count() - lc0
    st = h.stats()
    ms = float(np.mean(times))
    ms = max_over_ranks(ms, dist, "cuda")
    pts_per_step = counted / max(1, args.steps)
    # outputs of every batch (the ones the timed steps did not keep are recomputed
    # untimed: the results are deterministic) for the accuracy checks
    log(f"timed {args.steps} steps: {np.mean(times):.0f} ms per step")
    for b in range(NB):
        if not done[b]:
            keep(b, step(b))
    acc = {"oracle": check_accuracy(sigma, W, golden, rtol, member=member),
           "flags": {"converged": int(((flags & p._abi.PT_NOT_CONVERGED) == 0).sum()),
                     "not_converged": int(((flags & p._abi.PT_NOT_CONVERGED) != 0).sum()),
                     "fp64_fallback": int(((flags & p._abi.PT_IR_FALLBACK) != 0).sum()),
                     "singular_to_working_precision": int(((flags & p._abi.PT_SINGULAR) != 0).sum())}}
    value = job_throughput(pts_per_step, world, ms)
    peaks = _peaks()

    # one profiled step: per-kernel CUDA-event times on the launching stream
    h.reset_stats()
    opts.profile = 1
    step(0)
    torch.cuda.synchronize()
    opts.profile = 0
    kst = h.kernel_stats()
    prof_ms = h.stats()["ms_total"]
    solver = opts.fp32_solver if opts.fp32_solver != p._abi.SOLVER_AUTO else p.tuned_config(W.n)["fp32_solver"]
    rf = roofline(kst, peaks, W.n, tensor_solve=solver in (p._abi.SOLVER_TENSOR_CORES, p._abi.SOLVER_TC16,
                                                           p._abi.SOLVER_TC32))
    if rf is not None:
        rf["share_of_step"] = max(kst.values(), key=lambda v: v["ms"])["ms"] / max(prof_ms, 1e-9)

    # end to end through the host-buffer C-ABI call (z in, results out, copies inside)
    log("end-to-end steps")
    hopts = p.Opts.from_buffer_copy(opts)
    hopts.io_host = 1
    del ws
    e2e_ws = torch.empty(max(h.workspace_bytes(ix.size, hopts) for ix in bidx), dtype=torch.uint8, device="cuda")
    zpin = [torch.from_numpy(W.z[ix].copy()).pin_memory().numpy() for ix in bidx]

    def host_outs(m):
        return {"sigma": torch.empty(m, dtype=torch.float64).pin_memory().numpy(),
                "res": torch.empty(m, dtype=torch.float64).pin_memory().numpy(),
                "flags": torch.empty(m, dtype=torch.int32).pin_memory().numpy(),
                "member": torch.empty(m, dtype=torch.int32).pin_memory().numpy().view(np.uint32)}

    outs = [host_outs(ix.size) for ix in bidx]
    h.grid_host(zpin[0], eps, opts=hopts, workspace=e2e_ws, out=outs[0])
    e2e_t, e2e_pts = [], 0
    n_e2e = max(1, min(args.steps, 5))
    for i in range(n_e2e):
        b = i % NB
        flush.zero_()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.grid_host(zpin[b], eps, opts=hopts, workspace=e2e_ws, out=outs[b])
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        e2e_pts += bidx[b].size
    del e2e_ws
    e2e_ms = max_over_ranks(float(np.mean(e2e_t)) * 1e3, dist, "cuda")
    e2e_step = e2e_pts / n_e2e
    e2e = {"value": job_throughput(e2e_step, world, e2e_ms), "unit": "points/s",
           "h2d_bytes_per_step": int(e2e_step * 16 * world),
           "d2h_bytes_per_step": int(e2e_step * (8 + 8 + 4 + 4) * world), "steps": n_e2e}

    extras = {}
    cpu = None
    if not args.no_extras and rank == 0:
        # plain FP64 inverse Lanczos on a sample of the grid: its speed (shift-batched and
        # per point) and the mixed result's error against it there
        log("FP64 inverse Lanczos on a sample")
        stride = 97 if W.n >= 8000 else 20
        idx = np.arange(0, npts, stride)
        sub = torch.from_numpy(W.z[idx].copy()).cuda()
        o64 = p.default_opts(mode=p.INVLANC, precision=p.FP64, rtol=1e-10)
        h.grid(sub[:4], eps, opts=o64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = h.grid(sub, eps, opts=o64)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        extras["invlanc_fp64_batched"] = {"points": int(idx.size), "points_per_s": idx.size / dt,
                                          "sample": f"every {stride}th grid point"}
        acc["vs_fp64_sample"] = compare_with_fp64(sigma[idx], r64["sigma"].cpu().numpy(), fro, W.n, rtol,
                                                  member[idx], r64["member"].cpu().numpy(), eps)
        acc["vs_fp64_sample"]["sample"] = f"every {stride}th grid point"
        o1 = p.default_opts(mode=p.INVLANC, precision=p.FP64, rtol=1e-10, shift_batch=1)
        t0 = time.perf_counter()
        h.grid(sub[:8], eps, opts=o1)
        torch.cuda.synchronize()
        extras["invlanc_fp64_per_point"] = {"points": 8, "points_per_s": 8 / (time.perf_counter() - t0),
                                            "sample": f"the first 8 of every {stride}th grid point"}
        if args.accuracy_full:
            t0 = time.perf_counter()
            f64 = h.grid(torch.from_numpy(W.z).cuda(), eps, opts=o64)
            torch.cuda.synchronize()
            acc["vs_fp64_every_point"] = compare_with_fp64(sigma, f64["sigma"].cpu().numpy(), fro, W.n, rtol, member,
                                                           f64["member"].cpu().numpy(), eps)
            acc["vs_fp64_every_point"]["fp64_seconds"] = time.perf_counter() - t0
        if args.workload == "triangular8000":
            h.close()
            t_ex = time.time()
            for name, fn in (("gaussian2000_invlanc_mixed", lambda: gaussian_line(p, torch, eps)),
                             ("multi_matrix_64", lambda: multi_line(64, 2, 1)),
                             ("rectangular_invlanc_fp64", lambda: rect_line(p, torch, eps)),
                             ("toeplitz_recycling", lambda: toeplitz_recycling(
                                 p, torch, eps, [int(k) for k in args.recycle_ranks.split(",")]))):
                if time.time() - t_ex > args.extras_budget:
                    extras[name] = {"skipped": f"comparison budget of {args.extras_budget:.0f} s spent"}
                    continue
                log(f"comparison {name}")
                t1 = time.time()
                extras[name] = fn()
                extras[name]["wall_seconds"] = time.time() - t1
        log("CPU baseline")
        cpu = cpu_baseline(W, args.workload)

    result = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if prec == p.MIXED else "f64", "data": "synthetic",
        "config": {"workload": label, "mode": "invlanc", "precision": args.precision, "points": npts,
                   "batch": f"{npts // NB}-{-(-npts // NB)} grid points per step (every {NB}th point, offset = step "
                            f"index mod {NB}); {NB} consecutive steps cover the grid once",
                   "points_per_step": pts_per_step,
                   "l2": "flushed (256 MB write) between timed steps; T's packed copies exceed L2",
                   "host_prep_seconds_untimed": t_prep},
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


def rect_line(p, torch, eps):
    """FP64 inverse Lanczos on rectangular pencils (m >= 2n, one QR of [T - zI; B]
    per point): points/s of a whole grid, and the FP64 rate of the per-point
    factorisation (8 n^3 / 3 flops per point) from a profiled run."""
    from paper_2606_26785_b300 import workloads

    out = {}
    for name, n in (("rect_gaussian", 150), ("toeplitz_folding", 120), ("rect_gaussian", 600)):
        W = workloads.make(name, n=n)
        h = p.Pseudo(W.T)
        z = torch.from_numpy(W.z).cuda()
        o = p.default_opts(mode=p.INVLANC, precision=p.FP64, rtol=1e-10)
        h.grid(z, eps, opts=o)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.grid(z, eps, opts=o)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        h.reset_stats()
        h.grid(z, eps, opts=p.default_opts(mode=p.INVLANC, precision=p.FP64, rtol=1e-10, profile=1))
        ks = h.kernel_stats()
        qr_ms = ks["rect_qr"]["ms"]
        qr_tf = 8.0 * n ** 3 / 3.0 * z.numel() / (qr_ms / 1e3) / 1e12 if qr_ms > 0 else None
        out[f"{name}_n{n}"] = {
            "m": int(W.C.shape[0]), "n": n, "points": int(z.numel()), "points_per_s": z.numel() / dt,
            "qr_ms": qr_ms, "qr_fp64_tflops": qr_tf,
            "qr_frac_of_fp64": qr_tf / FP64_MEASURED_TFLOPS if qr_tf else None,
            "solve_ms": ks["trsv64"]["ms"], "lanczos_steps": h.stats()["lanczos_steps"]}
        h.close()
    return out


def gaussian_line(p, torch, eps):
    """The dense complex Gaussian workload (n = 2000, 200 x 200 grid) in mixed
    precision inverse Lanczos, with its 32 stored oracle values."""
    W, t_schur = make_workload("gaussian2000")
    h = p.Pseudo(W.T)
    z = torch.from_numpy(W.z).cuda()
    o = p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    h.grid(z, eps, opts=o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = h.grid(z, eps, opts=o)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    acc = check_accuracy(out["sigma"].cpu().numpy(), W, WORKLOADS["gaussian2000"][1], 1e-8,
                         member=out["member"].cpu().numpy())
    h.close()
    return {"workload": WORKLOADS["gaussian2000"][0], "points": int(W.z.size), "points_per_s": W.z.size / dt,
            "seconds": dt, "accuracy": acc, "host_schur_seconds_untimed": t_schur}


TOEPLITZ_GOLDEN = ROOT / "tests" / "golden" / "toeplitz1200_samples.json"


def toeplitz_recycling(p, torch, eps, ranks=(8, 32, 64)):
    """The recycled Rayleigh--Ritz-SVD path (Alg. 3) next to inverse Lanczos on
    the banded Toeplitz + noise matrix (superdiagonal 1, subdiagonal 0.25,
    complex Gaussian noise 1e-3/sqrt(n), seed 5) at n = 1200 on a 50 x 50 grid
    over the workload's window [-1.5, 1.5] x [-1, 1], in mixed precision at
    the given recycled ranks k (r = 4): acceptance counts, points/s, the
    agreement of every converged result with inverse Lanczos, and the stored
    oracle values (tests/golden/toeplitz1200_samples.json) at the points
    reported converged."""
    from paper_2606_26785_b300 import workloads
    from tests.parity import check_sigma

    g = json.loads(TOEPLITZ_GOLDEN.read_text())
    n, nx, ny = g["n"], g["nx"], g["ny"]
    t0 = time.time()
    C = workloads.toeplitz_noisy(n, 5)
    T, _, serr = workloads.schur(C)
    t_schur = time.time() - t0
    log(f"toeplitz n={n}: host Schur {t_schur:.1f} s")
    fro = float(np.linalg.norm(C))
    z = workloads.grid(-1.5, 1.5, -1.0, 1.0, nx, ny)
    zt = torch.from_numpy(z).cuda()
    idx = np.array(g["index"])
    h = p.Pseudo(T)
    res = {}

    def run(name, o):
        h.reset_stats()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out = h.grid(zt, eps, opts=o)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        st = h.stats()
        log(f"toeplitz {name}: {dt:.1f} s, accepted {int(st['n_accepted'])}")
        sig, fl = out["sigma"].cpu().numpy(), out["flags"].cpu().numpy()
        conv = (fl[idx] & p._abi.PT_NOT_CONVERGED) == 0
        orep = check_sigma(sig[idx][conv], np.array(g["sigma_ref"])[conv], n=n, fro=g["fro_norm"], schur_err=serr,
                           oracle_off=np.array(g["oracle_off"])[conv], rtol=1e-8)
        orep["not_converged_of_stored"] = int((~conv).sum())
        res[name] = {"points_per_s": z.size / dt, "seconds": dt, "accepted": int(st["n_accepted"]),
                     "refined": int(st["n_refined"]), "not_converged": int(st["n_not_converged"]),
                     "lobpcg_iters": int(st["lobpcg_iters"]), "sv_R": int(st["sv_R"]),
                     "rtilde_capped": int(st["n_rtilde_capped"]), "oracle": orep}
        return sig, fl

    o_inv = p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    h.grid(zt[:64], eps, opts=o_inv)
    s_ref, f_ref = run("invlanc_mixed", o_inv)
    for k in ranks:
        o = p.default_opts(mode=p.RECYCLE, precision=p.MIXED, rtol=1e-8, r=4, p_max=k // 4, grid_nx=nx, grid_ny=ny,
                           batch_b=20)
        sig, fl = run(f"recycle_mixed_k{k}", o)
        both = ((fl | f_ref) & p._abi.PT_NOT_CONVERGED) == 0
        rep = compare_with_fp64(sig[both], s_ref[both], fro, n, 2e-8)
        rep["note"] = "against inverse Lanczos (mixed) at the points both report converged; band 2e-8"
        res[f"recycle_mixed_k{k}"]["vs_invlanc"] = rep
    h.close()
    return {"workload": f"banded Toeplitz + noise n={n} (seed 5), {nx}x{ny} grid over [-1.5,1.5]x[-1,1]",
            "host_schur_seconds_untimed": t_schur, "schur_err": serr, **res}


BATCH_GOLDEN = ROOT / "tests" / "golden" / "batch16_samples.json"


def multi_line(nm, steps, warmup):
    """The multi-matrix workload: independent complex Gaussian matrices
    N(0, 1/n), n log-uniform in [256, 2048] (seed 40), each on its own 64 x 64
    grid over [-1.5, 1.5]^2; the first nm of its sequence (host Schur factors
    not timed).  One step = one pseudo_grid_batch call over all of them in
    mixed precision (solver kernel and Lanczos slots from the tuned table); the
    same matrices one after another with pseudo_grid are timed beside it.
    Accuracy: the stored oracle values of the 8 smallest of the first 16
    matrices."""
    import torch

    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import workloads
    from tests.parity import check_sigma

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
    eps = workloads.EPS_LEVELS
    npts = nm * zh.size

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    # preallocated workspace and outputs, as a serving loop keeps them
    ws = torch.empty(p.grid_batch_workspace_bytes(hs, [zh.size] * nm, opts), dtype=torch.uint8, device="cuda")
    outs = None
    for _ in range(max(1, warmup)):
        outs, _ = p.grid_batch(hs, [z] * nm, eps, opts=opts, workspace=ws, out=outs)
    for h in hs:
        h.reset_stats()
    lc0 = p._abi.load().pseudo_launch_count()
    t_batch = [timed(lambda: p.grid_batch(hs, [z] * nm, eps, opts=opts, workspace=ws, out=outs))
               for _ in range(steps)]
    launches = (p._abi.load().pseudo_launch_count() - lc0) // max(1, steps)
    ms = float(np.mean([t for t, _ in t_batch]))
    del ws
    # the same matrices one after another (one shared workspace, preallocated
    # outputs; each call replays its handle's cached loop graph)
    wseq = torch.empty(max(h.workspace_bytes(zh.size, opts) for h in hs), dtype=torch.uint8, device="cuda")
    seq_out = [h.grid(z, eps, opts=opts, workspace=wseq) for h in hs]
    ms_seq = float(np.mean([timed(lambda: [h.grid(z, eps, opts=opts, workspace=wseq, out=o_)
                                           for h, o_ in zip(hs, seq_out)])[0]
                            for _ in range(max(1, min(2, steps)))]))
    del wseq, seq_out
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
    for h in hs:
        h.close()
    return {"value": npts / (ms / 1e3), "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "gpu_launches": int(launches),
            "workload": f"multi-matrix: first {nm} of 64 complex Gaussian matrices N(0,1/n), n log-uniform in "
                        "[256,2048] (seed 40), 64x64 grid each over [-1.5,1.5]^2",
            "sizes": sizes, "points": npts, "host_schur_s": t_prep,
            "sequential_pseudo_grid": {"ms": ms_seq, "points_per_s": npts / (ms_seq / 1e3)},
            "speedup_over_sequential": ms_seq / ms, "accuracy": acc}


def run_multi(args):
    """--workload multi: the multi-matrix workload (multi_line) as its own JSON line."""
    r = multi_line(args.matrices, args.steps, args.warmup)
    print(json.dumps({
        "metric": METRIC, "value": r["value"], "unit": "points/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "dtype": "f64+f32",
        "data": "synthetic", "gpu_launches": r["gpu_launches"],
        "config": {"workload": r["workload"], "sizes": r["sizes"], "points": r["points"],
                   "host_schur_s": r["host_schur_s"]},
        "sequential_pseudo_grid": r["sequential_pseudo_grid"], "speedup_over_sequential": r["speedup_over_sequential"],
        "accuracy": r["accuracy"]}))


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands (one-sided Jacobi SVD of
    C - zI) on a bounded sample of the same workload each step (see
    oracle_sample), on the host cores of rank 0."""
    if rank != 0:
        return
    wl = "triangular8000" if args.workload == "multi" else args.workload
    label, _ = WORKLOADS[wl]
    W, _ = make_workload(wl)
    threads = os.cpu_count() or 1
    vals, secs, what = [], [], ""
    for s in range(args.warmup + args.steps):
        v, dt, what = oracle_sample(W, wl, threads)
        if s >= args.warmup:
            vals.append(v)
            secs.append(dt)
    v = None if any(x is None for x in vals) else float(1.0 / np.mean([1.0 / x for x in vals]))
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
                      "higher_is_better": True, "config": {"workload": label},
                      "cpu_baseline": {"kind": "oracle", "cores": threads, "value": v, "unit": "points/s",
                                       "sample": what},
                      "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    main()
