"""Oracle for the pseudospectra hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import anything from this package.
The CUDA library never links, imports or calls it, and it never calls the
CUDA library: the two share no code.  Inputs reach both sides from the seeded
generators in ``paper_2606_26785_b300.workloads``, which hold none of the
method's arithmetic.

Contents
--------
``sigma_min_grid(C, z)``
    sigma_min(C - z I) for every z, by a plain one-sided Jacobi SVD of the
    ORIGINAL dense C in IEEE double (``jacobi_svd.c``).  This is the defining
    quantity of the epsilon-pseudospectrum (Sec. 1, eqs. (defSquare) and
    (defSquareSVD)); membership of level eps is ``sigma_min < eps`` (strict).
``singular_values(C, z)``
    the full ascending spectrum, used by the invariant pins.
``recycle_ref``
    the recycled Rayleigh--Ritz-SVD (Alg. 1) and the recycle-subspace update
    (Alg. 2) written out step by step in NumPy, used to check intermediate
    quantities of the GPU path on small cases.
``precond_ref``
    the preconditioned path of Sec. 3 (the two-level preconditioner of eq.
    (twolevel), Alg. 4 recyProj, Alg. 5 psPrecRecy with a preconditioned
    LOBPCG-SVD) for a dense C without a Schur factor, written out in NumPy;
    the CUDA library does not implement this path.
``traversal.batch_zigzag(nx, ny, b)``
    the batch-zigzag visiting order of a Cartesian grid (Sec. 2.3, eq.
    (batch)), pinned in ``tests/test_oracle_traversal.py``.

Pins (all in ``tests/test_oracle_pins.py``, run with ``-m "not gpu"``): closed
forms for normal matrices, n = 1 and n = 2 brute force, unitary invariance,
sum of squares = Frobenius norm, product = |det|, the distance-to-spectrum
bound, 1-Lipschitz continuity in z, and agreement with an independent library
SVD on small random cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "jacobi_svd.c"
_LIB_PATH = _HERE / "liboracle_jacobi.so"
_lib = None


def build_lib(force: bool = False) -> Path:
    """Compile the C Jacobi oracle (gcc, OpenMP) next to its source."""
    if _LIB_PATH.exists() and not force and _LIB_PATH.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB_PATH
    cmd = [
        "gcc", "-O3", "-mavx2", "-mfma", "-fopenmp", "-fPIC", "-shared",
        str(_SRC), "-o", str(_LIB_PATH), "-lm",
    ]
    subprocess.run(cmd, check=True)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(str(_LIB_PATH))
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_svd_shifted.argtypes = [dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int]
        lib.oracle_svd_shifted.restype = ctypes.c_int
        lib.oracle_sigma_min_grid.argtypes = [dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              dp, ctypes.c_int64, dp, dp, ctypes.c_int]
        lib.oracle_sigma_min_grid.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_jacobi_rounds.argtypes = [dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int]
        lib.oracle_jacobi_rounds.restype = ctypes.c_int
        _lib = lib
    return _lib


def _as_fortran_c128(C) -> np.ndarray:
    C = np.asarray(C, dtype=np.complex128)
    if C.ndim != 2:
        raise ValueError("C must be 2-D")
    return np.asfortranarray(C)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def singular_values(C, z: complex, threads: int = 1, return_sweeps: bool = False):
    """All singular values of C - z I (ascending) and the oracle's final
    relative off-orthogonality (and, with ``return_sweeps``, the number of
    Jacobi sweeps it took).  C is m x n with m >= n; for m > n, I is the
    m x n rectangular identity (Sec. 1)."""
    lib = _load()
    A = _as_fortran_c128(C)
    m, n = A.shape
    if m < n:
        raise ValueError("need m >= n")
    sig = np.zeros(n, dtype=np.float64)
    off = np.zeros(1, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    s = lib.oracle_svd_shifted(A.ctypes.data_as(dp), m, m, n, float(np.real(z)), float(np.imag(z)),
                               sig.ctypes.data_as(dp), off.ctypes.data_as(dp), int(threads))
    if s < 0:
        raise RuntimeError("oracle Jacobi SVD did not converge")
    if return_sweeps:
        return sig, float(off[0]), int(s)
    return sig, float(off[0])


def jacobi_rounds(C, z: complex, rounds: int, threads: int = 1):
    """Run only the first ``rounds`` rounds of the oracle's Jacobi iteration
    on C - z I (each round: n/2 disjoint column-pair rotations) and return
    nothing.  A timing sample for matrices where a whole point takes hours: a
    full point takes sweeps * (n - 1 + n % 2) rounds."""
    lib = _load()
    A = _as_fortran_c128(C)
    m, n = A.shape
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_jacobi_rounds(A.ctypes.data_as(dp), m, m, n, float(np.real(z)), float(np.imag(z)), int(rounds),
                             int(threads))


def sigma_min_grid(C, z, threads: int | None = None):
    """sigma_min(C - z_p I) for every entry of z (any shape); returns
    (sigma_min, off) with the shape of z.  ``off`` is the final relative
    off-orthogonality of each point's Jacobi run."""
    lib = _load()
    A = _as_fortran_c128(C)
    m, n = A.shape
    if m < n:
        raise ValueError("need m >= n")
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).ravel())
    zri = np.ascontiguousarray(zz.view(np.float64))
    out = np.zeros(zz.size, dtype=np.float64)
    off = np.zeros(zz.size, dtype=np.float64)
    if threads is None:
        threads = max_threads()
    dp = ctypes.POINTER(ctypes.c_double)
    bad = lib.oracle_sigma_min_grid(A.ctypes.data_as(dp), m, m, n, zri.ctypes.data_as(dp), zz.size,
                                    out.ctypes.data_as(dp), off.ctypes.data_as(dp), int(threads))
    if bad:
        raise RuntimeError(f"oracle Jacobi SVD did not converge at {bad} points")
    shape = np.shape(z)
    return out.reshape(shape), off.reshape(shape)


def membership(sigma, eps_levels):
    """Bit i of word p is set iff sigma[p] < eps_levels[i] (strict, eq.
    (defSquareSVD))."""
    sigma = np.asarray(sigma, dtype=np.float64).ravel()
    words = np.zeros(sigma.size, dtype=np.uint32)
    for i, e in enumerate(eps_levels):
        words |= (sigma < float(e)).astype(np.uint32) << np.uint32(i)
    return words


