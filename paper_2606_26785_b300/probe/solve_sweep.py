"""Time the mixed-precision multi-shift solve (the tensor-core kernel for
handles that select it) on leading n x n blocks of the upper-triangular
n = 8000 workload, for several orders and column counts, with the error of a
few columns against the FP64 solve.  Prints one JSON line per case (median
CUDA-event milliseconds of the last 4 of 6 calls, both directions unless
--upper-only).

    python -m paper_2606_26785_b300.probe.solve_sweep --orders 2048,8000 --columns 1184,4736
    python -m paper_2606_26785_b300.probe.solve_sweep --lib /tmp/wide/libpseudo_b300.so ...

``--lib`` times another build of the library (compile-time tuning constants,
``python -m paper_2606_26785_b300.build --define ... --out ...``).
"""
import argparse
import json
from pathlib import Path


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lib", type=Path, default=None)
    ap.add_argument("--orders", default="8000")
    ap.add_argument("--columns", default="1184,2368,3552,4736,7104,9472")
    ap.add_argument("--upper-only", action="store_true")
    a = ap.parse_args()
    from paper_2606_26785_b300 import _abi

    if a.lib is not None:
        _abi._LIB = a.lib.resolve()
    import numpy as np
    import torch

    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import workloads

    W = workloads.make("triangular")
    rng = np.random.default_rng(0)
    for nk in (int(x) for x in a.orders.split(",")):
        h = p.Pseudo(np.ascontiguousarray(W.T[:nk, :nk]))
        for ncols in (int(x) for x in a.columns.split(",")):
            X0 = torch.from_numpy(rng.standard_normal((nk, ncols)) + 1j * rng.standard_normal((nk, ncols))).cuda()
            zk = torch.from_numpy(W.z[:: max(1, W.z.size // ncols)][:ncols].copy()).cuda()
            for adj in (False,) if a.upper_only else (False, True):
                X = X0.clone()
                ts = []
                for _ in range(6):
                    X.copy_(X0)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    h.solve(X, zk, adjoint=adj, precision=p.MIXED)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = float(np.median(ts[2:]))
                k = min(32, ncols)
                Xr = X0[:, :k].clone()
                h.solve(Xr, zk[:k], adjoint=adj, precision=p.FP64)
                err = (X[:, :k] - Xr).abs().pow(2).sum(0).sqrt() / Xr.abs().pow(2).sum(0).sqrt()
                print(json.dumps({"lib": str(_abi.lib_path()), "n": nk, "columns": ncols, "adjoint": adj,
                                  "ms": round(ms, 3), "tflops": round(4.0 * nk * nk * ncols / (ms * 1e-3) / 1e12, 2),
                                  "rel_err_vs_fp64_max": float(err.max())}), flush=True)
            del X0
        h.close()


if __name__ == "__main__":
    main()
