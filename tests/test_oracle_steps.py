"""Pins of the step-level oracle: a solve must satisfy its defining equation
(checked with an independent dense product), a product must equal the dense
product, and the adjoint must be the conjugate transpose (a transposed or
unconjugated operand fails here)."""
import numpy as np
import pytest

from oracle import steps


@pytest.mark.parametrize("n,adj", [(1, False), (5, False), (5, True), (33, True), (33, False)])
def test_solve_satisfies_equation(n, adj):
    rng = np.random.default_rng(n)
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) + 2 * np.eye(n)
    z = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    B = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    X = steps.shifted_solve(T, z, B, adj)
    for c in range(3):
        A = T - z[c] * np.eye(n)
        if adj:
            A = A.conj().T
        assert np.linalg.norm(A @ X[:, c] - B[:, c]) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(X[:, c])


def test_matvec_and_adjoint():
    rng = np.random.default_rng(3)
    n = 17
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    z = np.array([0.3 + 0.1j, -1j])
    X = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    Y = steps.shifted_matvec(T, z, X)
    YH = steps.shifted_matvec(T, z, X, adjoint=True)
    for c in range(2):
        A = T - z[c] * np.eye(n)
        assert np.allclose(Y[:, c], A @ X[:, c], rtol=1e-13, atol=1e-13)
        assert np.allclose(YH[:, c], A.conj().T @ X[:, c], rtol=1e-13, atol=1e-13)
    # lower triangle of the input is ignored
    T2 = T + np.tril(np.ones((n, n)), -1)
    assert np.allclose(steps.shifted_matvec(T2, z, X), Y)
