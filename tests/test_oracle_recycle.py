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


# ---- eq. (tau): the r~ rule of Alg. 1, on hand-built eigenvalues ----------
# tau = 2^-33 and theta_pr = 1 make the threshold theta_pr * eps_m / tau
# exactly 2^-19 (about 1.9e-6), so every case below sits on a known side of it.
TAU = 2.0 ** -33


def test_rtilde_threshold_is_exact():
    assert 1.0 * rr.EPS_M / TAU == 2.0 ** -19


def test_rtilde_first_qualifying_gap_at_or_after_r():
    # gaps theta_2-theta_3 = 9.8e-7 (below), theta_3-theta_4 = 4e-6 (above)
    th = [1e-8, 2e-8, 1e-6, 5e-6, 0.3, 1.0]
    assert rr.rtilde(th, 2, TAU) == 3
    # the search starts at j = r: with r = 3 the first gap looked at is theta_3-theta_4
    assert rr.rtilde(th, 3, TAU) == 3
    assert rr.rtilde(th, 4, TAU) == 4
    # a qualifying gap right at j = r is taken (the search does not start at r + 1)
    assert rr.rtilde([1e-8, 2e-8, 5e-6, 6e-6, 0.3, 1.0], 2, TAU) == 2


def test_rtilde_last_admissible_gap_and_empty_set():
    # only theta_{pr-1}-theta_pr qualifies: j = pr - 1 is inside the range
    assert rr.rtilde([1e-8, 2e-8, 3e-8, 4e-8, 5e-8, 1.0], 2, TAU) == 5
    # no gap qualifies: the minimum over an empty set is read as r~ = pr
    assert rr.rtilde([1.0, 1 + 1e-7, 1 + 2e-7, 1 + 3e-7, 1 + 4e-7, 1 + 5e-7], 2, TAU) == 6
    # r = pr leaves nothing to search
    assert rr.rtilde([0.1, 0.2, 0.3, 1.0], 4, TAU) == 4


def test_rtilde_gap_test_is_strict():
    # theta_3 - theta_2 = 2^-19 equals the threshold exactly: not "greater than"
    th = [0.0, 2.0 ** -20, 3 * 2.0 ** -20, 0.25, 0.5, 1.0]
    assert th[2] - th[1] == 2.0 ** -19
    assert rr.rtilde(th, 2, TAU) == 3


def test_rtilde_threshold_scales_with_the_largest_eigenvalue():
    # gap theta_2-theta_3 = 4e-9: below 2^-19 (theta_pr = 1) but above the
    # threshold a smaller eigenvalue (theta_1 or theta_r) would give
    th = [1e-9, 1.1e-8, 1.5e-8, 0.5, 0.75, 1.0]
    assert rr.rtilde(th, 2, TAU) == 3
    # scaling every eigenvalue scales the threshold with them: same answer
    assert rr.rtilde([1e6 * t for t in th], 2, TAU) == 3


def _state_with_theta(theta, r, seed=0):
    """A recycled state whose H(0) = H1 has the prescribed eigenvalues:
    W1 = U diag(sqrt(theta)) Q^H with U, V orthonormal, so W1^H W1 = Q diag(theta) Q^H."""
    k = len(theta)
    n = 2 * k
    rng = np.random.default_rng(seed)
    Z, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    V, U = Z[:, :k], Z[:, k:]
    W1 = U @ np.diag(np.sqrt(theta)) @ Q.conj().T
    st = rr.RecycleState(T=None, r=r, V=V, W1=W1, W3=np.zeros_like(V), W4=np.zeros_like(V))
    st.H1 = W1.conj().T @ W1
    st.H2 = W1.conj().T @ V
    return st


def test_recy_sing_uses_the_rtilde_rule():
    for th, r, want in (([1e-8, 2e-8, 1e-6, 5e-6, 0.3, 1.0], 2, 3),
                        ([1e-8, 2e-8, 5e-6, 6e-6, 0.3, 1.0], 2, 2),
                        ([1e-8, 2e-8, 3e-8, 4e-8, 5e-8, 1.0], 2, 5),
                        ([1.0, 1 + 1e-7, 1 + 2e-7, 1 + 3e-7, 1 + 4e-7, 1 + 5e-7], 2, 6),
                        ([1e-9, 1.1e-8, 1.5e-8, 0.5, 0.75, 1.0], 2, 3)):
        out = rr.recy_sing(_state_with_theta(th, r), 0.0, eps=0.0, tau=TAU)
        assert np.allclose(out["theta"], th, rtol=0, atol=1e-14)
        assert out["rt"] == want, (th, out["rt"])


# ---- eq. (omegaCond): the pruning count l of Alg. 2 -----------------------
# V = the first p*r standard basis vectors, so the projection errors are
# exact: rho_0 = |b| (the component outside span V) and
# rho_j^2 = b^2 + (squares of the components on the first j blocks).

def _basis_state(n, p, r):
    V = np.eye(n, p * r, dtype=np.complex128)
    return V


def _x1(a, b, n):
    x = np.zeros((n, 1), dtype=np.complex128)
    x[: len(a), 0] = a
    x[len(a), 0] = b
    return x


A_BLOCKS = [0.3, 0.4, 0.5, 0.5, 1.0, 1.0, 0.1, 0.1]  # r = 2, p = 4: block sums 0.25, 0.5, 2, 0.02


def test_prune_count_first_violation_minus_one():
    V = _basis_state(12, 4, 2)
    x = _x1(A_BLOCKS, 1.0, 12)
    # rho_1 = sqrt(1.25) = 1.118, rho_2 = sqrt(1.75) = 1.323, rho_3 = sqrt(3.75) = 1.936
    assert rr.prune_count(V, x, 2, 1.6, 60) == 2
    # with squares instead of norms rho_2^2 = 1.75 > 1.6 would give 1
    assert rr.prune_count(V, x, 2, 1.2, 60) == 1   # rho_2 / rho_0 = 1.323 > 1.2
    assert rr.prune_count(V, x, 2, 1.1, 60) == 0   # rho_1 / rho_0 = 1.118 > 1.1
    # never violated (rho_4 = 1.942 <= 2.5): every old block is dropped, l = p
    assert rr.prune_count(V, x, 2, 2.5, 60) == 4


def test_prune_count_ratio_test_is_strict():
    # b = 3, first block (4, 0): rho_1 = 5 exactly, rho_1 / rho_0 = fl(5/3) = omega: kept
    V = _basis_state(8, 2, 2)
    x = _x1([4.0, 0.0, 9.0, 0.0], 3.0, 8)
    assert rr.prune_count(V, x, 2, 5.0 / 3.0, 60) == 1
    assert rr.prune_count(V, x, 2, np.nextafter(5.0 / 3.0, 0.0), 60) == 0


def test_prune_count_p_max_cap_and_skip():
    V = _basis_state(12, 4, 2)
    x = _x1(A_BLOCKS, 1.0, 12)
    # l = 0 by eq. (omegaCond); p - l + 1 = 5 blocks exceed p_max = 3: l = p + 1 - p_max = 2
    assert rr.prune_count(V, x, 2, 1.1, 3) == 2
    # l = 2 keeps p - l + 1 = 3 <= 3 blocks: the cap does not bind
    assert rr.prune_count(V, x, 2, 1.6, 3) == 2
    # l = 1 keeps 4 > 3: raised to 2
    assert rr.prune_count(V, x, 2, 1.2, 3) == 2
    # p_max = 1 keeps only the new block
    assert rr.prune_count(V, x, 2, 1.6, 1) == 4
    # x1 inside span V: nothing is appended
    assert rr.prune_count(V, _x1(A_BLOCKS, 0.0, 12), 2, 1.6, 60) == -1


def test_update_recy_drops_the_counted_blocks():
    n, p, r = 12, 4, 2
    V = _basis_state(n, p, r)
    T = np.triu(np.arange(1, n * n + 1, dtype=np.float64).reshape(n, n) / (n * n)).astype(np.complex128)
    st = rr.RecycleState(T=T, r=r, V=V.copy(), L=np.eye(p * r, dtype=np.complex128),
                         X_blocks=[V[:, j * r:(j + 1) * r].copy() for j in range(p)])
    rr._refresh_aux_for(st)
    x2 = np.zeros((n, 1), dtype=np.complex128)
    x2[10, 0] = 1.0
    X = np.hstack([_x1(A_BLOCKS, 1.0, n), x2])
    l, skipped = rr.update_recy(st, X, omega=1.6, p_max=60)
    assert (l, skipped) == (2, False)
    assert st.p == p - l + 1
    # the new basis spans the old blocks 3 and 4 and the new block (blocks 1, 2 dropped)
    Q, _ = np.linalg.qr(np.hstack([V[:, l * r:], X]))
    assert np.allclose(st.V @ st.V.conj().T, Q @ Q.conj().T, atol=1e-12)
    errs, _ = st.check_invariants()
    assert all(v < 1e-12 for v in errs.values()), errs
