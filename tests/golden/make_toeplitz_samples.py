"""Write oracle reference values at sampled grid points of the banded
Toeplitz + noise workload (superdiagonal 1, subdiagonal 0.25, complex Gaussian
perturbation 1e-3/sqrt(n) per entry, seed 5) at n = 1200 on a 50 x 50 grid
over [-1.5, 1.5] x [-1, 1] (the full-size workload's window).  12 points drawn
uniformly (seed 23) among those whose distance to the symbol ellipse's
interior keeps sigma above the parity floor (|Re z| / 1.25)^2 + (|Im z| /
0.75)^2 >= 0.8, so the sample is not all excluded points.

Calls only ``oracle`` (one-sided Jacobi SVD of the original C - zI) and the
seeded generators; nothing from the CUDA path.

    python tests/golden/make_toeplitz_samples.py
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

N, NX, NY = 1200, 50, 50


def main():
    C = workloads.toeplitz_noisy(N, 5)
    z = workloads.grid(-1.5, 1.5, -1.0, 1.0, NX, NY)
    ok = (np.abs(z.real) / 1.25) ** 2 + (np.abs(z.imag) / 0.75) ** 2 >= 0.8
    rng = np.random.Generator(np.random.PCG64(23))
    idx = sorted(int(i) for i in rng.choice(np.flatnonzero(ok), size=12, replace=False))
    t0 = time.time()
    sig, off = oracle.sigma_min_grid(C, z[idx])
    out = {"workload": f"toeplitz+noise n={N} seed=5 grid {NX}x{NY} over [-1.5,1.5]x[-1,1]", "n": N, "nx": NX,
           "ny": NY, "index": idx, "z": [[float(v.real), float(v.imag)] for v in z[idx]],
           "sigma_ref": [float(v) for v in sig], "oracle_off": [float(v) for v in off],
           "fro_norm": float(np.linalg.norm(C)), "oracle_seconds": time.time() - t0,
           "oracle_threads": oracle.max_threads()}
    path = Path(__file__).resolve().parent / f"toeplitz{N}_samples.json"
    path.write_text(json.dumps(out, indent=1))
    print(path, out["oracle_seconds"])


if __name__ == "__main__":
    main()
