"""Pins of the oracle's restatement of the preconditioned path (Sec. 3:
eq. (twolevel), Alg. 4 recyProj, Alg. 5 psPrecRecy, with Alg. SM1.2) on
small dense matrices, against what the mathematics fixes."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import precond_ref as pr
from paper_2606_26785_b300 import workloads


def _spd(rng, n, cond=1e3):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    d = np.logspace(0, np.log10(cond), n)
    return (Q * d) @ Q.conj().T


@pytest.mark.parametrize("seed,rbar", [(0, 1), (1, 3), (2, 5)])
def test_two_level_shifts_the_smallest_pencil_eigenvalues_by_one(seed, rbar):
    """The lemma after eq. (twolevel): with E the K-orthonormal eigenvectors of
    the rbar smallest eigenvalues of the pencil (N, K), the eigenvalues of
    K_E^{-1} N are those of the pencil with the rbar smallest raised by 1."""
    rng = np.random.default_rng(seed)
    n = 12
    N = _spd(rng, n, 1e6)
    K = _spd(rng, n, 1e2)
    lam, E = scipy.linalg.eigh(N, K)  # ascending, E^* K E = I
    Kinv = np.linalg.inv(K)
    A = pr.two_level_apply(lambda R: Kinv @ R, E[:, :rbar], N, N)
    got = np.sort(np.linalg.eigvals(A).real)
    want = np.sort(np.concatenate([lam[:rbar] + 1.0, lam[rbar:]]))
    assert np.allclose(got, want, rtol=1e-8, atol=1e-8 * lam.max())
    # without a projection basis it is the base preconditioner alone
    B = pr.two_level_apply(lambda R: Kinv @ R, None, N, N)
    assert np.allclose(np.sort(np.linalg.eigvals(B).real), lam, rtol=1e-8)


@pytest.mark.parametrize("seed", range(4))
def test_base_preconditioner_and_the_bound_of_eq_tauRecycle(seed):
    """K = F^* F = N(z_dag) exactly, so the pencil's largest eigenvalue there is
    1, gamma = ||F^{-1}||_2 = 1 / sigma_min(C - z_dag I), and at any z the
    largest eigenvalue of (N(z), K) stays below (sqrt(lam_dag) + gamma|z - z_dag|)^2
    (Weyl)."""
    rng = np.random.default_rng(10 + seed)
    n = 10
    C = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    zd = complex(*rng.uniform(-1, 1, 2))
    Finv, gamma, lam_dag = pr.base_preconditioner(C, zd)
    F = np.linalg.inv(Finv)
    Nd = (C - zd * np.eye(n)).conj().T @ (C - zd * np.eye(n))
    assert np.allclose(F.conj().T @ F, Nd, atol=1e-12 * np.linalg.norm(Nd))
    assert lam_dag == pytest.approx(1.0, rel=1e-12)
    smin = np.linalg.svd(C - zd * np.eye(n), compute_uv=False).min()
    assert gamma == pytest.approx(1.0 / smin, rel=1e-10)
    for _ in range(5):
        z = zd + complex(*rng.uniform(-0.5, 0.5, 2))
        Nz = (C - z * np.eye(n)).conj().T @ (C - z * np.eye(n))
        lam_n = scipy.linalg.eigh(Nz, F.conj().T @ F, eigvals_only=True).max()
        assert lam_n <= (np.sqrt(lam_dag) + gamma * abs(z - zd)) ** 2 * (1 + 1e-10)


def _proj_state(rng, n, nblocks, rbar):
    C = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    Finv, _, _ = pr.base_preconditioner(C, 0.3 + 0.1j)
    ps = pr.ProjState(C @ Finv, Finv)
    for _ in range(nblocks):
        Xb, _ = np.linalg.qr(rng.standard_normal((n, rbar)) + 1j * rng.standard_normal((n, rbar)))
        ps.blocks.append(Xb)
    ps.refresh()
    return C, Finv, ps


def test_recy_proj_is_exact_on_a_full_basis():
    """V_bar spanning C^n: the Ritz values are the smallest eigenvalues of
    T_bar(z) = F^{-*} N(z) F^{-1}, the residuals vanish, and the projection
    vectors are F^{-1} times the Ritz vectors."""
    rng = np.random.default_rng(3)
    n, rbar = 12, 3
    C, Finv, ps = _proj_state(rng, n, 4, rbar)
    z = 0.1 - 0.4j
    out = pr.recy_proj(ps, z, rbar)
    Mb = (C - z * np.eye(n)) @ Finv
    lam = np.linalg.eigvalsh(Mb.conj().T @ Mb)
    assert np.allclose(out["theta"], lam[:rbar], rtol=1e-9, atol=1e-12 * lam.max())
    assert np.max(np.linalg.norm(out["W"], axis=0)) <= 1e-9 * lam.max()
    assert np.allclose(out["E"], Finv @ out["X"], atol=1e-10 * np.linalg.norm(Finv))


@pytest.mark.parametrize("seed", range(3))
def test_recy_proj_residual_matches_the_explicit_residual(seed):
    """On a partial basis the affine formula of Alg. 4 (W_bar_3 - z W_bar_4 -
    conj(z) W_bar_5 + |z|^2 W_bar_6) G - X Theta equals T_bar(z) X - X Theta,
    and every Ritz value bounds the matching eigenvalue from above."""
    rng = np.random.default_rng(20 + seed)
    n, rbar = 14, 2
    C, Finv, ps = _proj_state(rng, n, 3, rbar)
    z = complex(*rng.uniform(-1, 1, 2))
    out = pr.recy_proj(ps, z, rbar)
    Mb = (C - z * np.eye(n)) @ Finv
    Tb = Mb.conj().T @ Mb
    explicit = Tb @ out["X"] - out["X"] * out["theta"]
    assert np.allclose(out["W"], explicit, atol=1e-10 * np.linalg.norm(Tb))
    lam = np.linalg.eigvalsh(Tb)
    assert np.all(out["theta"] >= lam[:rbar] * (1 - 1e-10))


@pytest.mark.parametrize("seed", range(3))
def test_lobpcg_svd_against_the_jacobi_oracle(seed):
    """Alg. SM1.2 with a tight eta returns the smallest singular values of
    C - zI (Jacobi oracle of the original C), from above.  Preconditioned by
    K = N(z) itself it converges in a handful of steps, where the plain
    iteration needs over a hundred (or runs out of its cap)."""
    rng = np.random.default_rng(30 + seed)
    n, r = 40, 3
    C = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    z = complex(*rng.uniform(-0.8, 0.8, 2))
    Mz = C - z * np.eye(n)
    s_ref, _ = oracle.singular_values(C, z)
    X0 = pr._orthonormal_random(n, r, seed)
    Ninv = np.linalg.inv(Mz.conj().T @ Mz)
    X, xi, it, conv = pr.lobpcg_svd(Mz, X0, r, 1e-12, prec=lambda R: Ninv @ R)
    assert conv and it <= 30
    assert np.all(xi >= s_ref[:r] * (1 - 1e-12))
    assert np.max(np.abs(xi - s_ref[:r]) / s_ref[:r]) <= 1e-9
    assert np.allclose(np.linalg.norm(X, axis=0), 1.0) and np.allclose(X.conj().T @ X, np.eye(r), atol=1e-10)
    _, _, it_plain, conv_plain = pr.lobpcg_svd(Mz, X0, r, 1e-12, maxit=100)
    assert it_plain > 3 * it or not conv_plain


@pytest.mark.parametrize("name,n,eta", [("grcar", 24, 1e-4), ("gaussian", 24, 1e-4), ("gaussian", 20, 1e-10)])
def test_ps_prec_recy_against_the_jacobi_oracle(name, n, eta):
    """Alg. 5 end to end on an 8 x 8 grid: every returned value is a Ritz value
    of N(z), hence at least sigma_min(C - zI) (Jacobi oracle), and a pair that
    meets eq. (tolC) or (tolSVD) lies within eta ||C - zI||_2 of it (the
    backward-stability bound of those criteria)."""
    W = workloads.make(name, n=n, nx=8, ny=8)
    C = W.C
    sig, st = pr.ps_prec_recy(C, W.z, W.nx, W.ny, b=4, r=2, rbar=3, eta=eta)
    ref, _ = oracle.sigma_min_grid(C, W.z)
    norms = np.array([np.linalg.norm(C - z * np.eye(n), 2) for z in W.z])
    print(name, n, eta, st)
    assert st["not_converged"] == 0
    assert st["accepted"] + st["refined"] == W.z.size
    assert np.all(sig >= ref - 64 * n * 2.2e-16 * norms)
    assert np.all(sig - ref <= eta * norms + 64 * n * 2.2e-16 * norms)


@pytest.mark.parametrize("seed", range(6))
def test_projection_pruning_agrees_with_the_block_triangular_form(seed):
    """Eq. (omegaCond) computed two ways: ProjState.update takes the projection
    errors from their definition (fresh bases of the kept blocks), Alg. 2 as
    restated in recycle_ref tracks them through its block-lower-triangular
    factor.  With S_bar = I (F = I) and the same blocks, both drop the same
    number of blocks and keep the same span."""
    from oracle import recycle_ref as rr

    rng = np.random.default_rng(40 + seed)
    n, r, nb = 16, 2, 5
    C = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    ps = pr.ProjState(C, np.eye(n, dtype=np.complex128))
    st = rr.RecycleState(T=C, r=r)
    base = np.linalg.qr(rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))[0]
    for j in range(nb):
        # slowly drifting blocks, so that some pruning counts are 0 and some larger
        X = base + (0.05 + 0.3 * (seed % 3)) * j * (rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))
        X, _ = np.linalg.qr(X)
        l1 = ps.update(X, 1.6, 1, 4)
        l2, skipped = rr.update_recy(st, X, 1.6, 4, rb=1)
        assert (l1 == -1) == skipped
        if not skipped:
            assert l1 == l2
        Vp = ps.V
        assert np.linalg.norm(st.V - Vp @ (Vp.conj().T @ st.V)) <= 1e-10
