"""Time the device-driven inverse-Lanczos loop (device_loop = 1: one CUDA graph
per call, conditional nodes decide every step) against the host-driven loop
(device_loop = 0) on single-matrix calls of a few sizes, with preallocated
workspace and outputs (a repeated call replays the cached graph).  Prints one
JSON line per case: median milliseconds per call of each loop.

    python -m paper_2606_26785_b300.probe.loop_compare
"""
import json
import time


def main():
    import numpy as np
    import torch

    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import workloads

    cases = [("grcar", 100, 50, p.FP64), ("grcar", 100, 50, p.MIXED), ("gaussian", 256, 64, p.MIXED),
             ("gaussian", 1024, 64, p.MIXED), ("gaussian", 2000, 100, p.MIXED)]
    for name, n, g, prec in cases:
        W = workloads.make(name, n=n, nx=g, ny=g)
        h = p.Pseudo(W.T)
        z = torch.from_numpy(W.z).cuda()
        rtol = 1e-10 if prec == p.FP64 else 1e-8
        row = {"workload": name, "n": n, "points": int(z.numel()), "precision": "fp64" if prec == p.FP64 else "mixed"}
        for loop in (0, 1):
            o = p.default_opts(mode=p.INVLANC, precision=prec, rtol=rtol, device_loop=loop)
            ws = torch.empty(h.workspace_bytes(z.numel(), o), dtype=torch.uint8, device="cuda")
            out = h.grid(z, workloads.EPS_LEVELS, opts=o, workspace=ws)
            ts = []
            for _ in range(5):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h.grid(z, workloads.EPS_LEVELS, opts=o, workspace=ws, out=out)
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - t0) * 1e3)
            row["device_loop" if loop else "host_loop"] = {"ms": float(np.median(ts)),
                                                          "points_per_s": z.numel() / (np.median(ts) / 1e3)}
            del ws
        h.close()
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
