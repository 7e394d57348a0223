"""Write oracle reference values at a few grid points of the strongly
nonnormal triangular workload (n = 8000, seed 3; 300 x 300 grid over
[-1.5, 1.5]^2).  Calls only ``oracle`` (one-sided Jacobi SVD of C - zI with
C := T, dense) and the seeded generators.  Each point costs tens of minutes
on a few cores, so only a handful of points (seeded choice, seed 13) are
stored.

    python tests/golden/make_triangular_samples.py [count] [n] [nx]
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
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 2
    n = int(sys.argv[2]) if len(sys.argv) > 2 else 8000
    nx = int(sys.argv[3]) if len(sys.argv) > 3 else 300
    T = workloads.triangular(n, 3)
    z = workloads.grid(-1.5, 1.5, -1.5, 1.5, nx, nx)
    rng = np.random.Generator(np.random.PCG64(13))
    idx = sorted(int(i) for i in rng.choice(z.size, size=count, replace=False))
    res = []
    t0 = time.time()
    for i in idx:
        s, off = oracle.sigma_min_grid(T, z[[i]])
        res.append((float(s[0]), float(off[0])))
        print(i, res[-1], time.time() - t0, flush=True)
    out = {"workload": f"triangular n={n} seed=3 grid {nx}x{nx} over [-1.5,1.5]^2", "n": n, "nx": nx, "ny": nx,
           "index": idx, "z": [[float(z[i].real), float(z[i].imag)] for i in idx],
           "sigma_ref": [r[0] for r in res], "oracle_off": [r[1] for r in res],
           "fro_norm": float(np.linalg.norm(T)), "oracle_seconds": time.time() - t0,
           "oracle_threads": oracle.max_threads()}
    path = Path(__file__).resolve().parent / f"triangular{n}_samples.json"
    path.write_text(json.dumps(out, indent=1))
    print(path)


if __name__ == "__main__":
    main()
