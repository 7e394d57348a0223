"""Seeded synthetic workloads: matrices, Schur factors and grids.

This module holds NO arithmetic of the pseudospectra method.  It only draws
inputs and performs the one-time preliminary reduction that happens before the
method starts (the complex Schur form C = Q T Q^H of SM2.1: M = T, S = I).
Both the CUDA path and the CPU oracle take their inputs from here; neither is
imported by it.

Recipes (numpy ``Generator(PCG64(seed))``; a complex draw is a real n x n
standard-normal block followed by an imaginary n x n block, row-major):

* ``grcar(n)``: 1 on the diagonal and the first three superdiagonals, -1 on the
  subdiagonal (the classic nonnormal test matrix).
* ``gaussian(n, seed)``: C = (A + iB)/sqrt(n), A, B iid N(0, 1); so real and
  imaginary parts of each entry are N(0, 1/n).
* ``triangular(n, seed)``: upper-triangular T with diagonal uniform in the unit
  disk (radius sqrt(U), angle 2*pi*U') and strictly upper part 3(A + iB)/sqrt(n)
  -- a strongly nonnormal triangular matrix that is its own Schur factor.
* ``toeplitz_noisy(n, seed)``: banded Toeplitz (superdiagonal 1, subdiagonal
  0.25, diagonal 0) plus E, e_ij = 1e-3/sqrt(n) * (a + ib)/sqrt(2).
* ``gaussian_batch(count, seed)``: sizes n_i = round(exp(U[ln 256, ln 2048]))
  drawn with ``seed``, matrix i = ``gaussian(n_i, 100*seed + i)``.
* ``grid(...)``: equispaced Cartesian grid, endpoints included in both axes,
  flattened as z[iy*nx + ix] = x[ix] + i*y[iy].
* ``rect_gaussian(n, m, seed)``: rectangular m x n, entries (A + iB)/sqrt(n).
* ``toeplitz_folding(n, m)``: the m x n section (m >= 2n) of the banded
  Toeplitz operator with superdiagonal 1 and subdiagonal 0.25 (a matrix
  folding: a rectangular truncation of an infinite matrix, Sec. 1).
* ``rect_gaussian_short``: a Gaussian C with n < m < 2n (m = n + 3n/8).

For a rectangular C (m >= 2n), ``rect_reduce`` is the preliminary reduction
of SM2.2 followed by two more unitary steps that keep the singular values of
C - zI: C_l = Q_1 R_l (thin QR), C_u = U T U^H (Schur), R_l U = Q_2 B (QR), so
that [T - zI; B] = diag(U^H, Q_2^H) [C_u - zI; R_l] U with T and B upper
triangular; the library takes the 2n x n pencil [T; B].  With n < m < 2n,
C is first extended by 2n - m zero rows: [C; 0] - z[I; 0] = [C - zI; 0] has
the singular values of C - zI, and the extended matrix has m = 2n (B then
has only m - n nonzero rows).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EPS_LEVELS = tuple(10.0 ** (-e) for e in range(1, 11))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    a = rng.standard_normal(shape)
    b = rng.standard_normal(shape)
    return a + 1j * b


def grcar(n: int) -> np.ndarray:
    C = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        for d in range(4):
            if i + d < n:
                C[i, i + d] = 1.0
        if i + 1 < n:
            C[i + 1, i] = -1.0
    return C


def gaussian(n: int, seed: int) -> np.ndarray:
    return _complex_normal(_rng(seed), (n, n)) / math.sqrt(n)


def triangular(n: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    rho = np.sqrt(rng.random(n))
    phi = 2.0 * np.pi * rng.random(n)
    U = 3.0 * _complex_normal(rng, (n, n)) / math.sqrt(n)
    T = np.triu(U, 1)
    T[np.arange(n), np.arange(n)] = rho * np.exp(1j * phi)
    return T


def toeplitz_noisy(n: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    C = (1e-3 / math.sqrt(n)) * _complex_normal(rng, (n, n)) / math.sqrt(2.0)
    i = np.arange(n - 1)
    C[i, i + 1] += 1.0
    C[i + 1, i] += 0.25
    return C


def gaussian_batch_sizes(count: int, seed: int, lo: int = 256, hi: int = 2048) -> list[int]:
    u = _rng(seed).random(count)
    return [int(round(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo))))) for x in u]


def gaussian_batch(count: int, seed: int, lo: int = 256, hi: int = 2048) -> list[np.ndarray]:
    return [gaussian(n, 100 * seed + i) for i, n in enumerate(gaussian_batch_sizes(count, seed, lo, hi))]


def grid(xmin: float, xmax: float, ymin: float, ymax: float, nx: int, ny: int) -> np.ndarray:
    x = np.linspace(xmin, xmax, nx)
    y = np.linspace(ymin, ymax, ny)
    return (x[None, :] + 1j * y[:, None]).ravel().astype(np.complex128)


def schur(C: np.ndarray):
    """Complex Schur form C = Q T Q^H (LAPACK zgees through SciPy) and its
    backward error ||C - Q T Q^H||_F.  This is the one-time preliminary
    reduction that precedes the method; it is never timed as part of it."""
    import scipy.linalg

    T, Q = scipy.linalg.schur(np.asarray(C, dtype=np.complex128), output="complex")
    T = np.triu(T)
    err = float(np.linalg.norm(C - (Q @ T) @ Q.conj().T))
    return T, Q, err


def rect_gaussian(n: int, m: int, seed: int) -> np.ndarray:
    return _complex_normal(_rng(seed), (m, n)) / math.sqrt(n)


def toeplitz_folding(n: int, m: int) -> np.ndarray:
    C = np.zeros((m, n), dtype=np.complex128)
    i = np.arange(n - 1)
    C[i, i + 1] = 1.0
    i = np.arange(min(n, m - 1))
    C[i + 1, i] = 0.25
    return C


def rect_reduce(C: np.ndarray):
    """The 2n x n pencil [T; B] of a rectangular C (m > n rows): T and B upper
    triangular with sigma([T - zI; B]) = sigma(C - zI) for every z, and the
    backward error of the three factorisations (sum of their Frobenius-norm
    residuals).  One-time host work before the method, never timed with it.
    With m < 2n the rows of C are first extended by zeros to 2n."""
    import scipy.linalg

    C = np.asarray(C, dtype=np.complex128)
    m, n = C.shape
    if m <= n:
        raise ValueError("need m > n (a square C takes the Schur factor)")
    if m < 2 * n:
        C = np.vstack([C, np.zeros((2 * n - m, n), dtype=np.complex128)])
    Cu, Cl = C[:n], C[n:]
    Q1, Rl = np.linalg.qr(Cl, mode="reduced")
    T, U = scipy.linalg.schur(Cu, output="complex")
    T = np.triu(T)
    Q2, B = np.linalg.qr(Rl @ U)
    B = np.triu(B)
    err = (np.linalg.norm(Cu - (U @ T) @ U.conj().T) + np.linalg.norm(Cl - Q1 @ Rl)
           + np.linalg.norm(Rl @ U - Q2 @ B))
    return np.vstack([T, B]), float(err)


@dataclass
class Workload:
    """One synthetic problem: the dense matrix C the oracle sees, the Schur
    factor T the library sees, and the grid."""

    name: str
    C: np.ndarray
    T: np.ndarray
    z: np.ndarray
    nx: int
    ny: int
    schur_err: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.T.shape[1]


def make(name: str, nx: int | None = None, ny: int | None = None, n: int | None = None) -> Workload:
    """Build a named workload.  ``nx``/``ny``/``n`` override the default grid
    and size (for the small parity cases)."""
    if name == "grcar":
        n = n or 100
        C = grcar(n)
        nx = nx or 50
        ny = ny or 50
        z = grid(-1.0, 3.0, -3.5, 3.5, nx, ny)
    elif name == "gaussian":
        n = n or 2000
        C = gaussian(n, 2)
        nx = nx or 200
        ny = ny or 200
        z = grid(-1.5, 1.5, -1.5, 1.5, nx, ny)
    elif name == "triangular":
        n = n or 8000
        C = triangular(n, 3)
        nx = nx or 300
        ny = ny or 300
        z = grid(-1.5, 1.5, -1.5, 1.5, nx, ny)
        return Workload(name, C, C.copy(), z, nx, ny, 0.0, {"seed": 3})
    elif name == "toeplitz":
        n = n or 16000
        C = toeplitz_noisy(n, 5)
        nx = nx or 500
        ny = ny or 500
        z = grid(-1.5, 1.5, -1.0, 1.0, nx, ny)
    elif name in ("rect_gaussian", "toeplitz_folding", "rect_gaussian_short"):
        if name == "rect_gaussian":
            n = n or 150
            C = rect_gaussian(n, 2 * n + 37, 7)
            z = grid(-1.5, 1.5, -1.5, 1.5, nx or 40, ny or 40)
        elif name == "rect_gaussian_short":
            n = n or 120
            C = rect_gaussian(n, n + max(1, 3 * n // 8), 8)
            z = grid(-1.5, 1.5, -1.5, 1.5, nx or 40, ny or 40)
        else:
            n = n or 120
            C = toeplitz_folding(n, 2 * n)
            z = grid(-1.5, 1.5, -1.0, 1.0, nx or 40, ny or 40)
        M, err = rect_reduce(C)
        return Workload(name, C, M, z, nx or 40, ny or 40, err, {})
    else:
        raise ValueError(f"unknown workload {name!r}")
    T, _, err = schur(C)
    return Workload(name, C, T, z, nx, ny, err, {})
