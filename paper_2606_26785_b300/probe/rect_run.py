"""One FP64 inverse-Lanczos grid on a rectangular pencil (m >= 2n rows, one QR
of [T - zI; B] per point): a warm-up call, then one timed call; prints the
points per second and the per-kernel-class device times of a profiled call.
The small, self-contained case that the profiles of the rectangular kernels
(rect_qr_kernel, rect_solve_kernel) are taken on.

    python -m paper_2606_26785_b300.probe.rect_run [--name rect_gaussian] [--n 150] [--grid 40] [--host-loop]
"""
import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--name", default="rect_gaussian", choices=["rect_gaussian", "toeplitz_folding"])
    ap.add_argument("--n", type=int, default=150)
    ap.add_argument("--grid", type=int, default=40)
    ap.add_argument("--host-loop", action="store_true", help="every call takes the host-driven loop (plain "
                    "launches, as a profiler capture wants them)")
    args = ap.parse_args()
    import torch

    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import workloads

    W = workloads.make(args.name, n=args.n, nx=args.grid, ny=args.grid)
    h = p.Pseudo(W.T)
    z = torch.from_numpy(W.z).cuda()
    o = p.default_opts(mode=p.INVLANC, precision=p.FP64, rtol=1e-10, device_loop=0 if args.host_loop else 1)
    h.grid(z, workloads.EPS_LEVELS, opts=o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.grid(z, workloads.EPS_LEVELS, opts=o)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h.reset_stats()
    h.grid(z, workloads.EPS_LEVELS, opts=p.default_opts(mode=p.INVLANC, precision=p.FP64, rtol=1e-10, profile=1))
    ks = {k: v for k, v in h.kernel_stats().items() if v["launches"]}
    print(json.dumps({"workload": args.name, "m": int(W.C.shape[0]), "n": W.n, "points": int(z.numel()),
                      "points_per_s": z.numel() / dt, "kernels": ks, "stats": h.stats()}))
    h.close()


if __name__ == "__main__":
    main()
