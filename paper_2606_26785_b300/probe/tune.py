"""Offline sweep behind the library's tuned table (csrc/autotune_table.h).

For a representative matrix order of each bucket (orders 256 .. 2048, the
range of the multi-matrix workload; dense complex Gaussian N(0, 1/n), seed
100 + n; Schur factor on the host, untimed), time the mixed-precision
inverse-Lanczos path on a 64 x 64 grid over [-1.5, 1.5]^2 for every
combination of

  * the FP32 solver kernel: the tensor cores (tcgen05, 3xTF32) with 16 (3) or
    32 (4) right-hand sides per CTA, or the CUDA cores (1);
  * the number of Lanczos slots (shifts per solve launch);

and keep the fastest per bucket.  With --write the table is rewritten (the
library must then be rebuilt); without it the sweep is only printed.

    python -m paper_2606_26785_b300.probe.tune [--write] [--orders 256,362,...]
"""
from __future__ import annotations

import argparse
import datetime
import json
import time
from pathlib import Path


HERE = Path(__file__).resolve().parent
TABLE = HERE.parent / "csrc" / "autotune_table.h"
ORDERS = (256, 362, 512, 724, 1024, 1448, 2048)
SLOTS = (1024, 2048, 4096, 8192)
SOLVERS = (3, 4, 1)  # tensor cores 16 and 32 columns per CTA, CUDA cores


def sweep(orders, repeats=2):
    import torch

    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import workloads

    z = torch.from_numpy(workloads.grid(-1.5, 1.5, -1.5, 1.5, 64, 64)).cuda()
    rows = []
    for n in orders:
        T, _, _ = workloads.schur(workloads.gaussian(n, 100 + n))
        h = p.Pseudo(T)
        best = None
        for solver in SOLVERS:
            for slots in SLOTS:
                o = p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8, fp32_solver=solver,
                                   shift_batch=slots)
                h.grid(z, (), opts=o)
                torch.cuda.synchronize()
                ts = []
                for _ in range(repeats):
                    t0 = time.perf_counter()
                    h.grid(z, (), opts=o)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                t = min(ts)
                rows.append({"n": n, "fp32_solver": solver, "slots": slots, "seconds": t, "points_per_s": z.numel() / t})
                if best is None or t < best[0]:
                    best = (t, solver, slots)
        h.close()
        print(json.dumps({"n": n, "best": {"fp32_solver": best[1], "slots": best[2],
                                           "points_per_s": z.numel() / best[0]}}), flush=True)
    return rows


def table_text(rows, orders, gpu):
    best = {}
    for r in rows:
        b = best.get(r["n"])
        if b is None or r["seconds"] < b["seconds"]:
            best[r["n"]] = r
    # bucket edges halfway (geometrically) between the swept orders; orders above
    # the last swept one keep the untuned defaults (tensor cores, 8192 slots)
    edges = [int(round((a * b) ** 0.5)) for a, b in zip(orders[:-1], orders[1:])] + [int(round(orders[-1] * 1.41))]
    # a slot count at or above the sweep's 4,096 points cannot be told from a
    # larger one there: such entries get the largest count
    def slots(r):
        return max(SLOTS) if r["slots"] >= 4096 else r["slots"]

    lines = [f"    {{{e}, {best[n]['fp32_solver']}, {slots(best[n])}}},"
             f"  // n = {n}: {best[n]['points_per_s']:.0f} points/s" for n, e in zip(orders, edges)]
    lines.append("    {1 << 30, 0, 8192},  // larger orders: not swept (the defaults)")
    stamp = datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%d")
    return "\n".join([
        "// Tuned choices of the mixed-precision inverse-Lanczos path per matrix order,",
        "// written by paper_2606_26785_b300/probe/tune.py (an offline sweep over the FP32",
        "// solver kernel, with the tensor-core solve's column-group form, and the number",
        "// of Lanczos slots on one GPU).  Entry i applies to n <= n_max[i] (the last",
        "// entry to every larger n).",
        f"// sweep: {gpu}, {stamp}; 64 x 64 grid, mixed precision, rtol 1e-8",
        "#pragma once",
        "namespace pseudo {",
        "struct TunePoint {",
        "    int n_max;        // largest matrix order of the bucket",
        "    int fp32_solver;  // 0 tensor cores (form by order), 1 CUDA cores, 3 / 4 tensor cores,",
        "                      // 16 / 32 right-hand sides per CTA",
        "    int slots;        // Lanczos slots (shifts per solve launch)",
        "};",
        "static const TunePoint kTuneTable[] = {",
        *lines,
        "};",
        "}  // namespace pseudo",
        "",
    ])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", action="store_true")
    ap.add_argument("--orders", default=",".join(map(str, ORDERS)))
    args = ap.parse_args()
    import torch

    orders = tuple(int(v) for v in args.orders.split(","))
    rows = sweep(orders)
    text = table_text(rows, orders, torch.cuda.get_device_name(0))
    print(json.dumps({"rows": rows}))
    if args.write:
        TABLE.write_text(text)
    print(text)


if __name__ == "__main__":
    main()
