"""Acceptance rate of the recycled Rayleigh--Ritz-SVD under each grid
traversal, measured with the oracle's NumPy restatements (no GPU).

Runs the recycling loop of Alg. 3 with the NumPy restatements of Alg. 1
(``recycle_ref.recy_sing``) and Alg. 2 (``recycle_ref.update_recy``) over a
small grid, visiting the points in a given order.  A point is accepted when
its recycled Ritz triplet meets eq. (tolC) with ||M(z)|| = ||T||_2 + |z| and
the paper's parameters (eta = 1e-4, tau = 1e-10, omega = 1.6, eps = 1e-14
||T||_2^2); otherwise it is "refined" exactly (the r smallest right singular
vectors of T - zI from a library SVD stand in for LOBPCG-SVD) and the result
is appended to the recycled subspace.  r = 4, p_max = 4 (k = 16).

    python -m tests.traversal_acceptance {toeplitz|grcar|gaussian}

prints, per order, how many of the grid points were accepted.  This measures
the property Sec. 5 asks about (how much the traversal matters), independent
of the GPU path's own refinement accuracy.
"""
from __future__ import annotations

import sys
import time

import numpy as np

from oracle import recycle_ref
from oracle.traversal import batch_zigzag, hilbert, morton
from paper_2606_26785_b300 import workloads

CASES = {
    # name: (generator, grid window, grid size)
    "toeplitz": (lambda w: w.toeplitz_noisy(100, 5), (-1.5, 1.5, -1.0, 1.0), 40),
    "grcar": (lambda w: w.grcar(100), (-1.0, 3.0, -3.5, 3.5), 50),
    "gaussian": (lambda w: w.gaussian(100, 2), (-1.5, 1.5, -1.5, 1.5), 40),
}


def accepted_count(T, z, order, r=4, p_max=4, eta=1e-4, tau=1e-10, omega=1.6) -> int:
    n = T.shape[0]
    norm2 = np.linalg.norm(T, 2)
    eps = 1e-14 * norm2 ** 2
    st = recycle_ref.RecycleState(T=T, r=r)
    acc = 0
    for i in order:
        zi = z[i]
        M = norm2 + abs(zi)
        if st.V is not None:
            out = recycle_ref.recy_sing(st, zi, eps, tau)
            if out["wnorm"][0] <= max(eta * out["xi"][0] * M, M * M * np.finfo(np.float64).eps):
                acc += 1
                continue
        _, _, Vh = np.linalg.svd(T - zi * np.eye(n))
        recycle_ref.update_recy(st, Vh.conj().T[:, ::-1][:, :r], omega, p_max)
    return acc


def orders(nx: int, ny: int):
    return [("row zigzag (b = 1)", batch_zigzag(nx, ny, 1)), ("batch zigzag b = 5", batch_zigzag(nx, ny, 5)),
            ("batch zigzag b = 10", batch_zigzag(nx, ny, 10)), ("batch zigzag b = 20", batch_zigzag(nx, ny, 20)),
            ("Hilbert", hilbert(nx, ny)), ("Morton", morton(nx, ny))]


def main(name: str) -> None:
    gen, (x0, x1, y0, y1), m = CASES[name]
    T = workloads.schur(gen(workloads))[0]
    z = workloads.grid(x0, x1, y0, y1, m, m)
    for label, order in orders(m, m):
        t0 = time.time()
        a = accepted_count(T, z, order)
        print(f"{name:9s} {label:20s} accepted {a:4d} of {z.size} ({100.0 * a / z.size:4.1f}%)  "
              f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "toeplitz")
