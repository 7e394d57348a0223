"""Host-side input generators: shapes, recipes and determinism."""
import numpy as np
import pytest

from paper_2606_26785_b300 import workloads


def test_grcar_structure():
    C = workloads.grcar(7)
    assert C[0, 0] == 1 and C[0, 3] == 1 and C[0, 4] == 0 and C[1, 0] == -1 and C[2, 0] == 0


def test_grid_layout_inclusive_and_row_major():
    z = workloads.grid(-1, 3, -2, 2, 5, 3)
    assert z.shape == (15,)
    assert z[0] == -1 - 2j and z[4] == 3 - 2j and z[5] == -1 + 0j and z[-1] == 3 + 2j


def test_seeded_and_schur():
    a = workloads.gaussian(40, 2)
    b = workloads.gaussian(40, 2)
    assert np.array_equal(a, b)
    T, Q, err = workloads.schur(a)
    assert np.allclose(np.tril(T, -1), 0)
    assert err < 1e-12 * np.linalg.norm(a)


def test_triangular_recipe():
    T = workloads.triangular(50, 3)
    assert np.allclose(np.tril(T, -1), 0)
    assert np.all(np.abs(np.diag(T)) <= 1.0)


def test_batch_sizes_range():
    s = workloads.gaussian_batch_sizes(64, 40)
    assert len(s) == 64 and min(s) >= 256 and max(s) <= 2048


@pytest.mark.parametrize("name,n", [("rect_gaussian", 12), ("toeplitz_folding", 15), ("rect_gaussian_short", 16)])
def test_rect_reduce_keeps_singular_values(name, n):
    """The host reduction of a rectangular C (SM2.2 plus a Schur form of the
    top block and a QR of R_l U; a C with n < m < 2n is first extended by zero
    rows to 2n): [T; B] is 2n x n with both blocks upper triangular, and
    sigma([T - zI; B]) = sigma(C - zI) -- both sides by the oracle, within the
    reduction's backward error."""
    import oracle

    W = workloads.make(name, n=n, nx=3, ny=3)
    M = W.T
    assert M.shape == (2 * n, n)
    assert np.all(np.tril(M[:n], -1) == 0) and np.all(np.tril(M[n:], -1) == 0)
    assert W.schur_err < 1e-12 * max(1.0, np.linalg.norm(W.C))
    for z in W.z:
        a, _ = oracle.singular_values(W.C, z)
        b, _ = oracle.singular_values(M, z)
        assert np.max(np.abs(a - b)) <= 8 * W.schur_err + 1e-13 * a.max()


@pytest.mark.parametrize("m", [9, 13, 17])
def test_rect_reduce_short_c(m):
    """n < m < 2n (n = 9, m = 13 and 17; m = 9 is square and refused): B has
    only m - n nonzero rows, and the pencil keeps the singular values of the
    original m x n C - zI at a few shifts."""
    import oracle

    n = 9
    C = workloads.rect_gaussian(n, m, 11)
    if m == n:
        with pytest.raises(ValueError):
            workloads.rect_reduce(C)
        return
    M, err = workloads.rect_reduce(C)
    assert M.shape == (2 * n, n)
    assert np.all(M[n + (m - n):] == 0)
    for z in (0.3 - 0.2j, -1.1 + 0.4j, 0.0):
        a, _ = oracle.singular_values(C, z)
        b, _ = oracle.singular_values(M, z)
        assert a.shape == b.shape == (n,)
        assert np.max(np.abs(a - b)) <= 8 * err + 1e-13 * a.max()


def test_toeplitz_folding_recipe():
    C = workloads.toeplitz_folding(4, 8)
    assert C.shape == (8, 4)
    assert C[0, 1] == 1 and C[2, 3] == 1 and C[1, 0] == 0.25 and C[4, 3] == 0.25
    assert np.count_nonzero(C) == 3 + 4
