"""Write oracle reference values at sampled grid points of the dense complex
Gaussian workload (n = 2000, 200 x 200 grid over [-1.5, 1.5]^2, seed 2).

Calls only ``oracle`` (one-sided Jacobi SVD of the original C - zI) and the
seeded generators; nothing from the CUDA path.  Sample: 24 grid points drawn
uniformly (seed 7) and the 8 grid points nearest to eigenvalues of C that lie
inside the grid window (eigenvalues from the Schur diagonal).

    python tests/golden/make_gaussian_samples.py [n] [nx]
"""
import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2606_26785_b300 import workloads  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 2000
    nx = int(sys.argv[2]) if len(sys.argv) > 2 else 200
    W = workloads.make("gaussian", n=n, nx=nx, ny=nx)
    rng = np.random.Generator(np.random.PCG64(7))
    uni = rng.choice(W.z.size, size=24, replace=False)
    lam = np.diag(W.T)
    lam = lam[(np.abs(lam.real) < 1.45) & (np.abs(lam.imag) < 1.45)]
    near = []
    for l in lam[:: max(1, lam.size // 8)][:8]:
        near.append(int(np.argmin(np.abs(W.z - l))))
    idx = sorted(set(int(i) for i in uni) | set(near))
    t0 = time.time()
    sig, off = oracle.sigma_min_grid(W.C, W.z[idx])
    dt = time.time() - t0
    out = {
        "workload": f"gaussian n={n} seed=2 grid {nx}x{nx} over [-1.5,1.5]^2",
        "n": n, "nx": nx, "ny": nx,
        "index": idx,
        "z": [[float(v.real), float(v.imag)] for v in W.z[idx]],
        "sigma_ref": [float(v) for v in sig],
        "oracle_off": [float(v) for v in off],
        "fro_norm": float(np.linalg.norm(W.C)),
        "oracle_seconds": dt,
        "oracle_threads": oracle.max_threads(),
    }
    path = Path(__file__).resolve().parent / f"gaussian{n}_samples.json"
    path.write_text(json.dumps(out, indent=1))
    print(path, dt)


if __name__ == "__main__":
    main()
