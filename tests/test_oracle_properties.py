"""Randomised pins of the CPU oracle (hypothesis): on arbitrary small complex
matrices and shifts, the oracle's singular values agree with an independent
library SVD, and sigma_min obeys the bounds the mathematics fixes (distance
to the spectrum, Weyl's perturbation bound, the Frobenius identity)."""
import numpy as np
import pytest
from hypothesis import given, settings
from hypothesis import strategies as st

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")

# The oracle reads singular values off squared column norms, which underflow
# for entries below about 1e-154 in magnitude; no workload comes near that, so
# the drawn entries are 0 or at least 1e-100 in magnitude.
finite = st.floats(-4.0, 4.0, allow_nan=False, allow_infinity=False).map(lambda x: 0.0 if abs(x) < 1e-100 else x)


@st.composite
def matrix_and_shift(draw):
    n = draw(st.integers(1, 7))
    re = np.array(draw(st.lists(finite, min_size=n * n, max_size=n * n))).reshape(n, n)
    im = np.array(draw(st.lists(finite, min_size=n * n, max_size=n * n))).reshape(n, n)
    z = complex(draw(finite), draw(finite))
    return re + 1j * im, z


@settings(max_examples=150, deadline=None, derandomize=True)
@given(matrix_and_shift())
def test_matches_library_svd_and_frobenius(case):
    C, z = case
    n = C.shape[0]
    B = C - z * np.eye(n)
    s, _ = oracle.singular_values(C, z)
    ref = np.sort(np.linalg.svd(B, compute_uv=False))
    scale = max(np.linalg.norm(B, 2), 1e-300)
    assert np.all(np.diff(s) >= 0)
    assert np.max(np.abs(s - ref)) <= 64 * n * 2.2e-16 * scale + 1e-300
    assert abs(np.sum(s ** 2) - np.linalg.norm(B) ** 2) <= 64 * n * 2.2e-16 * np.linalg.norm(B) ** 2 + 1e-300


@settings(max_examples=100, deadline=None, derandomize=True)
@given(matrix_and_shift(), finite, finite)
def test_distance_and_weyl_bounds(case, dx, dy):
    C, z = case
    n = C.shape[0]
    lam = np.linalg.eigvals(C)
    smin = oracle.singular_values(C, z)[0][0]
    tol = 64 * n * 2.2e-16 * max(np.linalg.norm(C - z * np.eye(n), 2), 1.0)
    # sigma_min(C - zI) <= |lambda - z| for every eigenvalue lambda
    assert smin <= np.min(np.abs(lam - z)) + tol + 1e-9 * np.linalg.norm(C, 2)
    # Weyl: |sigma_min(C - zI) - sigma_min(C - wI)| <= |z - w|
    w = z + 0.1 * complex(dx, dy)
    smin_w = oracle.singular_values(C, w)[0][0]
    assert abs(smin - smin_w) <= abs(z - w) + 2 * tol


@pytest.mark.parametrize("seed", range(40))
def test_rank_deficient_matrices_converge(seed):
    """Rank-deficient C - zI (exactly parallel columns, a low-rank product,
    a zero column, z on a diagonal entry of a triangular C): the sweeps leave
    some columns at rounding-noise size, which floating point cannot
    orthogonalise further.  The oracle must still stop, with every singular
    value within the absolute bound of a library SVD (a zero singular value
    comes out at the rounding level of ||C - zI||)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    kind = seed % 4
    if kind == 0:  # two exactly parallel columns (the 2 x 2 case that once stalled)
        C = np.array([[0, 0], [1.5j, 0.5 + 0.1 * seed]], dtype=np.complex128)
        n, z = 2, 0j
    elif kind == 1:  # a rank-r product, z = 0
        r = int(rng.integers(1, n))
        U = rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))
        V = rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))
        C, z = (U @ V.conj().T) * 10.0 ** rng.uniform(-3, 3), 0j
    elif kind == 2:  # a zero column
        C = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        C[:, int(rng.integers(n))] = 0
        z = 0j
    else:  # z on a diagonal entry of a triangular matrix
        C = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        z = C[0, 0]
    B = C - z * np.eye(n)
    s, _ = oracle.singular_values(C, z)
    ref = np.sort(np.linalg.svd(B, compute_uv=False))
    assert np.max(np.abs(s - ref)) <= 64 * n * 2.2e-16 * max(np.linalg.norm(B, 2), 1e-300)
    assert s[0] <= 64 * n * 2.2e-16 * np.linalg.norm(B)
