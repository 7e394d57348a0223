"""Pins of the CPU oracle against facts fixed by mathematics, not by itself.

The oracle computes sigma(C - zI) by one-sided Jacobi (the plain definition of
Sec. 1, eq. (defSquareSVD)).  Each check below would fail for a plausible slip
in it: a wrong rotation sign or phase (no convergence / wrong values), z used
as its conjugate (closed forms with complex eigenvalues), a dropped shift
(distance bound, n = 1), a lost column (sum of squares, product = |det|).
"""
import numpy as np
import pytest

import oracle
from paper_2606_26785_b300 import workloads

pytestmark = pytest.mark.filterwarnings("ignore")


def _rand_unitary(n, rng):
    Z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def test_n1_closed_form():
    for c, z in [(2 + 1j, 0.5 - 0.25j), (-3j, 1.0), (0.7, 0.7)]:
        s, _ = oracle.singular_values(np.array([[c]]), z)
        assert abs(s[0] - abs(c - z)) <= 1e-15 * max(1, abs(c - z))


def test_n2_closed_form():
    rng = np.random.default_rng(11)
    for _ in range(20):
        A = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        z = complex(*rng.standard_normal(2))
        B = A - z * np.eye(2)
        f2 = np.sum(np.abs(B) ** 2)
        d = abs(B[0, 0] * B[1, 1] - B[0, 1] * B[1, 0])
        # eigenvalues of the 2x2 Gram: (f2 +- sqrt(f2^2 - 4 d^2))/2, and
        # smin^2 * smax^2 = d^2 keeps the small one free of cancellation
        smax2 = (f2 + np.sqrt(max(f2 * f2 - 4 * d * d, 0.0))) / 2
        smin = d / np.sqrt(smax2)
        s, _ = oracle.singular_values(A, z)
        assert abs(s[0] - smin) <= 1e-14 * np.sqrt(smax2)
        assert abs(s[1] - np.sqrt(smax2)) <= 1e-14 * np.sqrt(smax2)


@pytest.mark.parametrize("n", [3, 8, 33])
def test_normal_matrix_closed_form(n):
    rng = np.random.default_rng(n)
    lam = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Q = _rand_unitary(n, rng)
    C = Q @ np.diag(lam) @ Q.conj().T
    for z in [0.1 + 0.2j, -0.5 + 1.5j, lam[0] + 1e-3j]:
        s, _ = oracle.singular_values(C, z)
        ref = np.sort(np.abs(lam - z))
        assert np.max(np.abs(s - ref)) <= 64 * n * 2.2e-16 * np.max(np.abs(lam - z))


def test_conjugate_shift_is_not_confused():
    # C = diag(i), z = i  => sigma_min = 0; z = -i => 2.  A conj(z) slip swaps them.
    C = np.array([[1j, 0], [0, 3.0]])
    assert oracle.singular_values(C, 1j)[0][0] < 1e-15
    assert abs(oracle.singular_values(C, -1j)[0][0] - 2.0) < 1e-14


@pytest.mark.parametrize("n", [5, 24])
def test_unitary_invariance_and_det_and_frobenius(n):
    rng = np.random.default_rng(100 + n)
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Q = _rand_unitary(n, rng)
    C = Q @ T @ Q.conj().T
    for z in [0.3 - 0.1j, 1.0 + 1.0j]:
        sT, _ = oracle.singular_values(T, z)
        sC, _ = oracle.singular_values(C, z)
        scale = np.max(sT)
        assert np.max(np.abs(sT - sC)) <= 200 * n * 2.2e-16 * scale
        # sum of squares = ||C - zI||_F^2
        fro2 = np.sum(np.abs(C - z * np.eye(n)) ** 2)
        assert abs(np.sum(sC ** 2) - fro2) <= 1e-12 * fro2
        # product = |det(C - zI)| = prod |t_ii - z| (logs, to stay in range)
        logdet = np.sum(np.log(np.abs(np.diag(T) - z)))
        assert abs(np.sum(np.log(sC)) - logdet) <= 1e-9 * max(1.0, abs(logdet))
        # sigma_min <= dist(z, spectrum)
        assert sC[0] <= np.min(np.abs(np.diag(T) - z)) * (1 + 1e-12)


def test_lipschitz_in_z():
    W = workloads.make("grcar", nx=12, ny=12, n=24)
    s, _ = oracle.sigma_min_grid(W.C, W.z)
    s = s.reshape(W.ny, W.nx)
    z = W.z.reshape(W.ny, W.nx)
    dx = np.abs(np.diff(s, axis=1)) - np.abs(np.diff(z, axis=1))
    dy = np.abs(np.diff(s, axis=0)) - np.abs(np.diff(z, axis=0))
    assert dx.max() <= 1e-12 and dy.max() <= 1e-12


@pytest.mark.parametrize("m,n", [(6, 6), (40, 40), (30, 17), (65, 64)])
def test_agrees_with_library_svd(m, n):
    rng = np.random.default_rng(m * 1000 + n)
    C = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    Id = np.eye(m, n)
    for z in [0.0, 0.25 + 0.5j]:
        s, off = oracle.singular_values(C, z)
        ref = np.sort(np.linalg.svd(C - z * Id, compute_uv=False))
        assert np.max(np.abs(s - ref)) <= 100 * m * 2.2e-16 * ref[-1]
        assert off <= m * 2.3e-16


def test_grid_entry_matches_single_point_and_threads():
    W = workloads.make("grcar", nx=5, ny=4, n=30)
    a, _ = oracle.sigma_min_grid(W.C, W.z, threads=1)
    b, _ = oracle.sigma_min_grid(W.C, W.z, threads=4)
    c = np.array([oracle.singular_values(W.C, z, threads=3)[0][0] for z in W.z])
    assert np.max(np.abs(a - b)) <= 1e-14 and np.max(np.abs(a - c)) <= 1e-13


def test_membership_is_strict():
    w = oracle.membership([0.1, 0.05, 1e-3], [0.1, 0.01])
    assert list(w) == [0b00, 0b01, 0b11]


# ------------------------------------------------- rectangular C (m > n, Sec. 1)
# For C in C^{m x n}, m >= n, the shift uses the m x n rectangular identity:
# only the leading n x n block is shifted.

@pytest.mark.parametrize("m,n", [(2, 1), (7, 3), (12, 5), (9, 4)])
def test_rectangular_orthogonal_columns_closed_form(m, n):
    # C = [D; E; 0] with D, E diagonal: column j of C - zI is (d_j - z) e_j +
    # e_j e_{n+j}, so the columns are orthogonal and sigma_j = sqrt(|d_j - z|^2 +
    # |e_j|^2).  A shift applied to the wrong rows, or to all m rows, fails this.
    rng = np.random.default_rng(m * 10 + n)
    d = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    e = np.zeros(n, dtype=complex)
    k = min(n, m - n)
    e[:k] = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    C = np.zeros((m, n), dtype=complex)
    C[np.arange(n), np.arange(n)] = d
    C[n + np.arange(k), np.arange(k)] = e[:k]
    for z in [0.3 - 0.1j, d[0], -1.0 + 2.0j]:
        s, _ = oracle.singular_values(C, z)
        ref = np.sort(np.sqrt(np.abs(d - z) ** 2 + np.abs(e) ** 2))
        assert np.max(np.abs(s - ref)) <= 64 * m * 2.2e-16 * max(1.0, ref.max())


def test_rectangular_zero_bottom_is_the_square_normal_case():
    # C = [Q diag(lam) Q^H; 0]: the zero rows change nothing, sigma = |lam - z|
    rng = np.random.default_rng(5)
    n = 6
    lam = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Q = _rand_unitary(n, rng)
    C = np.vstack([Q @ np.diag(lam) @ Q.conj().T, np.zeros((2 * n + 1, n))])
    for z in [0.2 + 0.4j, lam[2] + 1e-6]:
        s, _ = oracle.singular_values(C, z)
        assert np.max(np.abs(s - np.sort(np.abs(lam - z)))) <= 1e-13 * max(1.0, np.abs(lam - z).max())


@pytest.mark.parametrize("m,n", [(4, 2), (9, 4), (20, 7)])
def test_rectangular_matches_library_svd(m, n):
    # a library SVD of the explicitly shifted matrix is an independent check
    rng = np.random.default_rng(100 + m)
    C = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    for z in [0.0, 1.0 - 0.5j]:
        A = C.copy()
        A[np.arange(n), np.arange(n)] -= z
        ref = np.sort(np.linalg.svd(A, compute_uv=False))
        s, _ = oracle.singular_values(C, z)
        assert np.max(np.abs(s - ref)) <= 1e-13 * ref.max()
