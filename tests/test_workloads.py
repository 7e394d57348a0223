"""Host-side input generators: shapes, recipes and determinism."""
import numpy as np

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
