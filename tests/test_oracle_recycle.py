"""Pins of the NumPy restatement of Alg. 1 / Alg. 2 (oracle/recycle_ref.py):
full-basis exactness of the recycled Ritz value against the Jacobi oracle, the
Courant--Fischer upper bound, and the QL / auxiliary-matrix identities after
a sequence of updates with pruning."""
import numpy as np

import oracle
from oracle import recycle_ref as rr


def _T(n, seed):
    rng = np.random.default_rng(seed)
    C = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    import scipy.linalg

    T, Q = scipy.linalg.schur(C, output="complex")
    return C, np.triu(T)


def test_full_basis_gives_exact_sigma():
    C, T = _T(8, 1)
    st = rr.RecycleState(T=T, r=4)
    rng = np.random.default_rng(2)
    for _ in range(2):
        X = rng.standard_normal((8, 4)) + 1j * rng.standard_normal((8, 4))
        rr.update_recy(st, X, omega=1.0, p_max=2)
    assert st.k == 8
    for z in [0.1 + 0.2j, -0.7j, 0.5]:
        out = rr.recy_sing(st, z, eps=0.0, tau=1e-10)
        ref = oracle.singular_values(C, z)[0][0]
        assert abs(out["xi"][0] - ref) <= 1e-12 * max(ref, 1.0) + 1e-14


def test_ritz_upper_bound_and_residual_definition():
    C, T = _T(30, 3)
    st = rr.RecycleState(T=T, r=4)
    for zz in [0.2 + 0.1j, 0.25 + 0.1j]:
        _, s, Vh = np.linalg.svd(T - zz * np.eye(30))
        rr.update_recy(st, Vh.conj().T[:, ::-1][:, :4], omega=1.6, p_max=4)
    z = 0.22 + 0.1j
    out = rr.recy_sing(st, z, eps=1e-14, tau=1e-10)
    ref = oracle.singular_values(C, z)[0][0]
    assert out["xi"][0] >= ref * (1 - 1e-12)
    # the fast residual equals the explicit one
    X = out["X"]
    N = (T - z * np.eye(30)).conj().T @ (T - z * np.eye(30))
    explicit = np.linalg.norm(N @ X - X * out["xi"][:4] ** 2, axis=0)
    assert np.allclose(out["wnorm"], explicit, rtol=1e-6, atol=1e-12)


def test_update_invariants_with_pruning():
    C, T = _T(40, 4)
    st = rr.RecycleState(T=T, r=3)
    grid = [0.1 * k + 0.05j for k in range(8)]
    for z in grid:
        _, s, Vh = np.linalg.svd(T - z * np.eye(40))
        rr.update_recy(st, Vh.conj().T[:, ::-1][:, :3], omega=1.6, p_max=4)
        errs, _ = st.check_invariants()
        assert all(v < 1e-10 for v in errs.values()), errs
        assert st.p <= 4
