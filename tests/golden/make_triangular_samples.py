"""Write oracle reference values at a few grid points of the strongly
nonnormal triangular workload (n = 8000, seed 3; 300 x 300 grid over
[-1.5, 1.5]^2).  Calls only ``oracle`` (one-sided Jacobi SVD of C - zI with
C := T, dense) and the seeded generators.

Points: the midpoints of the bottom and left grid edges and two opposite
corners, in that order.  Inside the unit disk that holds the spectrum this
matrix has sigma_min far below the parity floor 1e-8 ||T||_F (about 1e-31 at
the centre), so the sample sits on the grid's rim, where sigma_min is of
order 1e-3 (edge midpoints) and 5e-2 (corners).  Each point costs one to two
hours on a few host cores, so the file is rewritten after every point and a
partial file is a valid (shorter) sample.

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


def rim_points(nx):
    mid = nx // 2
    # (ix, iy): bottom-edge midpoint, left-edge midpoint, top-right and bottom-left corners
    return [(mid, 0), (0, mid), (nx - 1, nx - 1), (0, 0)]


def main():
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    n = int(sys.argv[2]) if len(sys.argv) > 2 else 8000
    nx = int(sys.argv[3]) if len(sys.argv) > 3 else 300
    T = workloads.triangular(n, 3)
    z = workloads.grid(-1.5, 1.5, -1.5, 1.5, nx, nx)
    idx = [iy * nx + ix for ix, iy in rim_points(nx)[:count]]
    path = Path(__file__).resolve().parent / f"triangular{n}_samples.json"
    done = []
    t0 = time.time()
    for i in idx:
        t1 = time.time()
        sig, off, sweeps = oracle.singular_values(T, z[i], threads=oracle.max_threads(), return_sweeps=True)
        done.append((i, float(sig[0]), float(off), time.time() - t1, sweeps))
        out = {"workload": f"triangular n={n} seed=3 grid {nx}x{nx} over [-1.5,1.5]^2", "n": n, "nx": nx,
               "ny": nx, "index": [d[0] for d in done],
               "z": [[float(z[d[0]].real), float(z[d[0]].imag)] for d in done],
               "sigma_ref": [d[1] for d in done], "oracle_off": [d[2] for d in done],
               "fro_norm": float(np.linalg.norm(T)), "schur_err": 0.0,
               "oracle_seconds_per_point": [d[3] for d in done], "oracle_sweeps": [d[4] for d in done],
               "oracle_seconds": time.time() - t0,
               "oracle_threads": oracle.max_threads()}
        path.write_text(json.dumps(out, indent=1))
        print(i, done[-1], flush=True)
    print(path)


if __name__ == "__main__":
    main()
