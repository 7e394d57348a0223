"""NumPy restatement of the paper's preconditioned path (Sec. 3) -- TEST
INFRASTRUCTURE ONLY (see the package docstring for who may import it).

The CUDA library does not implement this path.  This module writes it out for
a dense square C taken as it is (M = C, S = I, no Schur factor), so that its
parts can be pinned and its behaviour studied:

* ``two_level_apply``: the inverse of the two-level preconditioner, eq.
  (twolevel): K_Z^{-1} R = K^{-1} R + Z (Z^* N(z) Z)^{-1} Z^* R.
* ``base_preconditioner``: K = F^* F = N(z_dag) with F the triangular factor
  of a QR factorisation of C - z_dag I, gamma = ||F^{-1}||_2 and the largest
  eigenvalue of the pencil (N(z_dag), K) (= 1 for this K), the quantities of
  eq. (tauRecycle).
* ``lobpcg_svd``: Alg. SM1.2, LOBPCG for the smallest singular triplets of a
  matrix, with a preconditioner applied to the residual block, the
  Hetmaniuk--Lehoucq update and the stopping rule of eq. (tolSVD).
* ``ProjState`` and ``recy_proj``: the recycling subspace for projection of
  eq. (recyProj) with its auxiliary matrices (eqs. (H), (W12), (W3456) for the
  formal products M_bar = C F^{-1}, S_bar = F^{-1}) and Alg. 4: eigenpairs of
  H_bar(z), Ritz vectors, projection vectors and the residual.
* ``ps_prec_recy``: Alg. 5 over a grid in batch-zigzag order, with the
  singular-subspace steps of ``recycle_ref`` (Alg. 1, Alg. 2) on M = C.

Library primitives (numpy qr / svd / eigh / solve / inv) serve as the steps
the paper names qr, svd, eig and as the explicit inverse of F; nothing is
blocked or fused.  Readings where the text leaves a choice:
* the base preconditioner is exact at z_dag (K = N(z_dag)), so the largest
  pencil eigenvalue there is 1;
* ||T_bar(z)|| in eq. (tolTz) and ||M(z)|| in eqs. (tolC), (tolSVD) are the
  exact 2-norms (this is an oracle: it can afford them);
* the projection subspace keeps blocks of r_bar columns and is not updated
  when no computed sigma_bar_j^2 lies below tau_min (r_breve = 0);
* a LOBPCG-SVD run without a recycled start takes a seeded random
  orthonormal block;
* Hetmaniuk--Lehoucq: G_X = the first r columns of the Rayleigh--Ritz
  coefficients, G_P = G_X with the X rows set to zero, orthogonalised against
  G_X (twice) and orthonormalised; preconditioned residuals are
  orthogonalised against [X P] the same way, and directions that only
  rounding leaves (below 1e-10 of the block's norm) are dropped from the
  search basis, which must stay orthonormal for the Rayleigh--Ritz-SVD;
* the pruning test of eq. (omegaCond) uses projection errors computed from
  their definition (a fresh orthonormal basis of the kept blocks), which is
  what Alg. 2's block-triangular factor tracks incrementally.

Pinned in tests/test_oracle_precond.py by the eigenvalue shift of the
two-level preconditioner (the lemma after eq. (twolevel)), the bound of eq.
(tauRecycle) (Weyl), the exactness of recyProj on a full basis and its
residual formula against the explicit residual, LOBPCG-SVD against the Jacobi
oracle (and its fast convergence with the exact preconditioner), and
Alg. 5 end to end against the Jacobi oracle within the backward-stability
bound of eq. (tolC).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .recycle_ref import RecycleState, recy_sing, update_recy
from .traversal import batch_zigzag

EPS_M = np.finfo(np.float64).eps


def two_level_apply(Kinv, Z, Nz, R):
    """K_Z^{-1} R of eq. (twolevel): Kinv applies K^{-1} to a block, Z is the
    n x k projection basis (None or k = 0: the base preconditioner alone) and
    Nz the matrix N(z)."""
    out = Kinv(R)
    if Z is None or Z.shape[1] == 0:
        return out
    G = Z.conj().T @ (Nz @ Z)
    return out + Z @ np.linalg.solve(G, Z.conj().T @ R)


def base_preconditioner(C, z_dag):
    """K = F^* F = N(z_dag) from the QR factorisation C - z_dag I = Q F.
    Returns (F^{-1}, gamma = ||F^{-1}||_2, the largest eigenvalue of the
    pencil (N(z_dag), K))."""
    n = C.shape[1]
    _, F = np.linalg.qr(C - z_dag * np.eye(C.shape[0], n))
    Finv = np.linalg.inv(F)
    gamma = float(np.linalg.norm(Finv, 2))
    Mz = (C - z_dag * np.eye(C.shape[0], n)) @ Finv
    lam_n = float(np.linalg.norm(Mz, 2) ** 2)
    return Finv, gamma, lam_n


def _orthonormal_random(n, r, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))
    return Q


def _rr_svd(Cz, S):
    """Rayleigh--Ritz-SVD on the orthonormal basis S: thin QR of Cz S, SVD of
    its R.  Returns Ritz singular values ascending and the coefficient matrix
    G (columns in the same order)."""
    _, R = np.linalg.qr(Cz @ S)
    _, s, Vh = np.linalg.svd(R)
    order = np.argsort(s)
    return s[order], Vh.conj().T[:, order]


def _orth_against(B, W, scale):
    """An orthonormal basis of the part of W outside span B (B orthonormal):
    W projected off B twice, then the left singular vectors whose singular
    values exceed 1e-10 * scale (the norm W had before); directions that only
    rounding left behind are dropped rather than normalised into noise."""
    for _ in range(2):
        W = W - B @ (B.conj().T @ W)
    if W.shape[1] == 0:
        return W
    U, s, _ = np.linalg.svd(W, full_matrices=False)
    U = U[:, s > 1e-10 * max(scale, np.finfo(np.float64).tiny)]
    U = U - B @ (B.conj().T @ U)
    Q, _ = np.linalg.qr(U)
    return Q


def _hl(G, r, nx):
    """Hetmaniuk--Lehoucq: G_X = G[:, :r]; G_P = G_X with its first nx rows (the
    X part of the basis) zeroed, orthogonalised against G_X twice and
    orthonormalised (columns that vanish are dropped)."""
    GX = G[:, :r]
    GP = GX.copy()
    GP[:nx, :] = 0.0
    GP = _orth_against(GX, GP, float(np.linalg.norm(GX[nx:, :])) if G.shape[0] > nx else 0.0)
    return GX, GP


def lobpcg_svd(Cz, X0, rv, eta, prec=None, maxit=300):
    """Alg. SM1.2 for the r = X0.shape[1] smallest singular triplets of the
    matrix Cz, preconditioner ``prec`` (a function applied to the residual
    block; None = identity), stopping when eq. (tolSVD) holds for the first rv
    Ritz pairs.  Returns (X, xi, iterations, converged)."""
    r = X0.shape[1]
    normC = float(np.linalg.norm(Cz, 2))
    xi, G = _rr_svd(Cz, X0)
    X = X0 @ G
    W = Cz.conj().T @ (Cz @ X) - X * (xi ** 2)
    P = np.zeros((X.shape[0], 0), dtype=np.complex128)
    for it in range(1, maxit + 1):
        if prec is not None:
            W = prec(W)
        B = np.hstack([X, P])
        W = _orth_against(B, W, float(np.linalg.norm(W)))
        S = np.hstack([X, W, P])
        xi_all, G = _rr_svd(Cz, S)
        GX, GP = _hl(G, r, r)
        X = S @ GX
        P = S @ GP
        xi = xi_all[:r]
        W = Cz.conj().T @ (Cz @ X) - X * (xi ** 2)
        res = np.linalg.norm(W, axis=0)
        ok = res <= np.maximum(eta * normC * xi, normC ** 2 * EPS_M)
        rc = 0
        while rc < r and ok[rc]:
            rc += 1
        if rc >= rv:
            return X, xi, it, True
    return X, xi, maxit, False


@dataclass
class ProjState:
    """The recycling subspace for projection (eq. (recyProj)) for the formal
    products M_bar = C F^{-1}, S_bar = F^{-1}: the kept blocks X_bar^j (oldest
    first), an orthonormal basis V_bar of their span, and the auxiliary
    matrices of eqs. (H), (W12), (W3456) with bars."""

    Mb: np.ndarray
    Sb: np.ndarray
    blocks: list = field(default_factory=list)

    @property
    def k(self):
        return sum(b.shape[1] for b in self.blocks)

    def refresh(self):
        V, _ = np.linalg.qr(np.hstack(self.blocks))
        self.V = V
        self.W1, self.W2 = self.Mb @ V, self.Sb @ V
        self.H1 = self.W1.conj().T @ self.W1
        self.H2 = self.W1.conj().T @ self.W2
        self.H3 = self.W2.conj().T @ self.W2
        self.W3 = self.Mb.conj().T @ self.W1
        self.W4 = self.Mb.conj().T @ self.W2
        self.W5 = self.Sb.conj().T @ self.W1
        self.W6 = self.Sb.conj().T @ self.W2

    def update(self, Xb, omega, rbrev, p_max):
        """updateRecy for the projection subspace: drop the l oldest blocks
        chosen by eq. (omegaCond) on the first rbrev columns of Xb (projection
        errors from their definition; at most p_max blocks after the append),
        then append Xb.  Returns l, or -1 when Xb[:, :rbrev] already lies in
        the span (nothing appended)."""
        x1 = Xb[:, :rbrev]
        p = len(self.blocks)
        if p:
            V, _ = np.linalg.qr(np.hstack(self.blocks))
            rho0 = np.linalg.norm(x1 - V @ (V.conj().T @ x1))
            if rho0 <= 1e-12 * np.linalg.norm(x1):
                return -1
            l = p
            for j in range(1, p + 1):
                rest = self.blocks[j:]
                if rest:
                    Vj, _ = np.linalg.qr(np.hstack(rest))
                    rhoj = np.linalg.norm(x1 - Vj @ (Vj.conj().T @ x1))
                else:
                    rhoj = np.linalg.norm(x1)
                if rhoj / rho0 > omega:
                    l = j - 1
                    break
            if p - l + 1 > p_max:
                l = p + 1 - p_max
        else:
            l = 0
        self.blocks = self.blocks[l:] + [Xb.copy()]
        self.refresh()
        return l


def recy_proj(ps: ProjState, z: complex, rbar: int):
    """Alg. 4.  Returns dict with theta (the rbar smallest Ritz values of
    T_bar(z)), X (= V_bar G), E (= W_bar_2 G, the projection vectors) and W
    (the residual T_bar(z) X - X Theta by the affine formula)."""
    zc = np.conj(z)
    H = ps.H1 - z * ps.H2 - zc * ps.H2.conj().T + abs(z) ** 2 * ps.H3
    H = 0.5 * (H + H.conj().T)
    theta, G = np.linalg.eigh(H)
    Gr = G[:, :rbar]
    X = ps.V @ Gr
    E = ps.W2 @ Gr
    W = (ps.W3 - z * ps.W4 - zc * ps.W5 + abs(z) ** 2 * ps.W6) @ Gr - X * theta[:rbar]
    return {"theta": theta[:rbar], "X": X, "E": E, "W": W}


def ps_prec_recy(C, z, nx, ny, b=20, r=2, rbar=4, eps_rel=1e-14, tau=1e-10, omega=1.6, eta=1e-4,
                 tau_min=1e-3, tau_max=30.0, p_max=60, seed=7):
    """Alg. 5 on the nx x ny grid z (z[iy * nx + ix]) of a dense square C.
    Returns (sigma per grid point, statistics)."""
    C = np.asarray(C, dtype=np.complex128)
    n = C.shape[0]
    eye = np.eye(n)
    normC = float(np.linalg.norm(C, 2))
    eps = eps_rel * normC ** 2
    order = batch_zigzag(nx, ny, b)
    sst = RecycleState(T=C, r=r)
    z_dag = z[order[0]]
    Finv, gamma, lam_dag = base_preconditioner(C, z_dag)
    ps = ProjState(C @ Finv, Finv)
    stats = {"accepted": 0, "proj_accepted": 0, "proj_refined": 0, "rebuilt": 0, "refined": 0,
             "lobpcg_iters": 0, "proj_lobpcg_iters": 0, "not_converged": 0}
    sigma = np.zeros(z.size)
    for q, idx in enumerate(order):
        zz = complex(z[idx])
        Mz = C - zz * eye
        normMz = float(np.linalg.norm(Mz, 2))
        Xt = None
        if sst.k > 0:
            rs = recy_sing(sst, zz, eps, tau)
            if rs["wnorm"][0] <= max(eta * rs["xi"][0] * normMz, normMz ** 2 * EPS_M):
                sigma[idx] = rs["xi"][0]
                stats["accepted"] += 1
                continue
            Xt = rs["X"]
        if Xt is None:
            Xt = _orthonormal_random(n, r, seed + q)
        # the projection subspace: recycled, else refined by LOBPCG-SVD on M_bar(z)
        Ebar, lam_rbar, Xcheck = None, None, None
        if ps.k >= rbar:
            rp = recy_proj(ps, zz, rbar)
            Xcheck = rp["X"]
            Tb = float(np.linalg.norm(ps.Mb - zz * ps.Sb, 2) ** 2)
            if np.all(np.linalg.norm(rp["W"], axis=0) <= eta * Tb):
                Ebar, lam_rbar = rp["E"], float(rp["theta"][-1])
                stats["proj_accepted"] += 1

        def refine_projection(X0):
            Xb, sb, it, _ = lobpcg_svd(ps.Mb - zz * ps.Sb, X0, rbar, eta)
            stats["proj_lobpcg_iters"] += it
            stats["proj_refined"] += 1
            small = np.nonzero(sb ** 2 <= tau_min)[0]
            if small.size:
                ps.update(Xb, omega, int(small[-1]) + 1, p_max)
            return Finv @ Xb, float(sb[-1] ** 2)

        if Ebar is None:
            X0 = Xcheck if Xcheck is not None else _orthonormal_random(n, rbar, seed + 7919 + q)
            Ebar, lam_rbar = refine_projection(X0)
        lam_n = (np.sqrt(lam_dag) + gamma * abs(zz - z_dag)) ** 2
        if lam_n > tau_max or lam_rbar < tau_min:
            z_dag = zz
            Finv, gamma, lam_dag = base_preconditioner(C, z_dag)
            ps = ProjState(C @ Finv, Finv)
            stats["rebuilt"] += 1
            X0 = Xcheck if Xcheck is not None else _orthonormal_random(n, rbar, seed + 104729 + q)
            Ebar, lam_rbar = refine_projection(X0)
        # refinement of the point with the two-level preconditioner K_Ebar
        Nz = Mz.conj().T @ Mz
        Fi = Finv

        def prec(R, Fi=Fi, Ebar=Ebar, Nz=Nz):
            return two_level_apply(lambda Y: Fi @ (Fi.conj().T @ Y), Ebar, Nz, R)

        X, xi, it, conv = lobpcg_svd(Mz, Xt, 1, eta, prec=prec)
        stats["lobpcg_iters"] += it
        stats["refined"] += 1
        stats["not_converged"] += 0 if conv else 1
        sigma[idx] = xi[0]
        update_recy(sst, X, omega, p_max, rb=1)
    return sigma, stats
