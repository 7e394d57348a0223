"""Plain reference versions of the kernel-level steps (test infrastructure).

* ``shifted_solve(T, z, B, adjoint)``: column by column back substitution
  (T - z_c I) x_c = b_c, or forward substitution with (T - z_c I)^H -- the
  solves with R(z) and R(z)^* of Alg. 3 (M = T, S = I after the Schur
  reduction of SM2.1, so R(z) = T - zI).
* ``shifted_matvec(T, z, X, adjoint)``: (T - z_c I)^{op} x_c.

Both read only the upper triangle of T, loop in the textbook order, and use
numpy only for elementwise arithmetic.  Pinned in tests/test_oracle_steps.py
by the defining identity A x = b evaluated with an independent dense product.
"""
from __future__ import annotations

import numpy as np


def shifted_solve(T, z, B, adjoint: bool = False):
    T = np.triu(np.asarray(T, dtype=np.complex128))
    B = np.asarray(B, dtype=np.complex128)
    n, ncols = B.shape
    X = np.zeros_like(B)
    for c in range(ncols):
        zc = complex(z[c])
        b = B[:, c].copy()
        x = np.zeros(n, dtype=np.complex128)
        if not adjoint:
            # (T - zI) x = b, rows from the bottom
            for i in range(n - 1, -1, -1):
                s = b[i] - np.dot(T[i, i + 1:], x[i + 1:])
                x[i] = s / (T[i, i] - zc)
        else:
            # (T - zI)^H x = b: lower triangular with entries conj(T[k, i])
            for i in range(n):
                s = b[i] - np.dot(np.conj(T[:i, i]), x[:i])
                x[i] = s / np.conj(T[i, i] - zc)
        X[:, c] = x
    return X


def shifted_matvec(T, z, X, adjoint: bool = False):
    T = np.triu(np.asarray(T, dtype=np.complex128))
    X = np.asarray(X, dtype=np.complex128)
    n, ncols = X.shape
    Y = np.zeros_like(X)
    for c in range(ncols):
        zc = complex(z[c]) if z is not None else 0.0
        x = X[:, c]
        y = np.zeros(n, dtype=np.complex128)
        for i in range(n):
            if not adjoint:
                y[i] = np.dot(T[i, i:], x[i:]) - zc * x[i]
            else:
                y[i] = np.dot(np.conj(T[: i + 1, i]), x[: i + 1]) - np.conj(zc) * x[i]
        Y[:, c] = y
    return Y
