"""Write oracle reference values at sampled grid points of the multi-matrix
workload: complex Gaussian matrices N(0, 1/n) with n log-uniform in
[256, 2048] (sizes seed 40, matrix i seed 4000 + i), each on its own 64 x 64
grid over [-1.5, 1.5]^2.  The stored sample covers the first 16 matrices of
the sequence: 3 grid points (seed 17) on each of the 8 smallest of them.

Calls only ``oracle`` (one-sided Jacobi SVD of the original C - zI) and the
seeded generators; nothing from the CUDA path.

    python tests/golden/make_batch_samples.py
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

COUNT, SEED, NX = 16, 40, 64


def main():
    sizes = workloads.gaussian_batch_sizes(64, SEED)[:COUNT]
    mats = workloads.gaussian_batch(64, SEED)[:COUNT]
    z = workloads.grid(-1.5, 1.5, -1.5, 1.5, NX, NX)
    small = sorted(range(COUNT), key=lambda i: sizes[i])[:8]
    rng = np.random.Generator(np.random.PCG64(17))
    samples = []
    t0 = time.time()
    for m in sorted(small):
        idx = sorted(int(i) for i in rng.choice(z.size, size=3, replace=False))
        sig, off = oracle.sigma_min_grid(mats[m], z[idx])
        for i, s, o in zip(idx, sig, off):
            samples.append({"matrix": m, "n": sizes[m], "index": i, "z": [float(z[i].real), float(z[i].imag)],
                            "sigma_ref": float(s), "oracle_off": float(o),
                            "fro_norm": float(np.linalg.norm(mats[m]))})
    out = {"workload": f"first {COUNT} of 64 complex Gaussian matrices, sizes seed {SEED}, "
                       f"grid {NX}x{NX} over [-1.5,1.5]^2", "count": COUNT, "sizes": sizes, "nx": NX,
           "samples": samples, "oracle_seconds": time.time() - t0, "oracle_threads": oracle.max_threads()}
    path = Path(__file__).resolve().parent / "batch16_samples.json"
    path.write_text(json.dumps(out, indent=1))
    print(path, out["oracle_seconds"])


if __name__ == "__main__":
    main()
