"""Step-by-step NumPy restatement of the recycling method (test
infrastructure only).

* ``recy_sing``  : Alg. 1 (fast Rayleigh--Ritz-SVD on the recycled basis V)
                   with M = T, S = I after the Schur reduction (SM2.1):
                   H(z) = H1 - z H2 - conj(z) H2^H + (|z|^2 + eps) I (eq.
                   (rayleighN)); eigenpairs ascending; r~ by eq. (tau); QR of
                   (W1 - z W2) G_{1:r~} and SVD of its R (eq. (step2)); Ritz
                   vectors and the residual of eq. (fastresidual).
* ``update_recy``: Alg. 2 (omega pruning by eq. (omegaCond), block
                   Gram--Schmidt of eq. (blkGS), block-unitary restoration of
                   the QL factor, and the updates of H_q and W_q).
* ``RecycleState``: V, L, H1, H2, W1, W3, W4 with their defining identities
                   (``check_invariants``).

Library primitives (numpy eigh / qr / svd) serve as the steps the paper
names ``eig``, ``qr``, ``svd``.  Pinned in tests/test_oracle_recycle.py by the
full-basis exactness of the Ritz value, the Courant--Fischer upper bound, the
QL / auxiliary-matrix invariants after updates, hand-built eigenvalue sets
with a known r~ (``rtilde``: gaps on both sides of the threshold, at j = r,
at j = pr - 1, equal to it, none qualifying) and hand-built bases with known
projection errors rho_j and a known pruning count (``prune_count``: first
violation, never violated, a ratio equal to omega, the p_max cap).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

EPS_M = np.finfo(np.float64).eps


@dataclass
class RecycleState:
    T: np.ndarray
    r: int
    V: np.ndarray = None   # n x k
    L: np.ndarray = None   # k x k block lower triangular
    X_blocks: list = field(default_factory=list)  # the recycled X^j (for the invariant check)
    H1: np.ndarray = None  # (T V)^H (T V)
    H2: np.ndarray = None  # (T V)^H V
    W1: np.ndarray = None  # T V
    W3: np.ndarray = None  # T^H T V
    W4: np.ndarray = None  # T^H V

    @property
    def k(self):
        return 0 if self.V is None else self.V.shape[1]

    @property
    def p(self):
        return self.k // self.r

    def check_invariants(self, tol=1e-10):
        T, V = self.T, self.V
        n = T.shape[0]
        errs = {
            "orth": np.linalg.norm(V.conj().T @ V - np.eye(self.k)),
            "W1": np.linalg.norm(self.W1 - T @ V),
            "W3": np.linalg.norm(self.W3 - T.conj().T @ (T @ V)),
            "W4": np.linalg.norm(self.W4 - T.conj().T @ V),
            "H1": np.linalg.norm(self.H1 - (T @ V).conj().T @ (T @ V)),
            "H2": np.linalg.norm(self.H2 - (T @ V).conj().T @ V),
            "QL": np.linalg.norm(np.hstack(self.X_blocks) - V @ self.L),
        }
        r = self.r
        upper = 0.0
        for a in range(self.p):
            for b in range(a + 1, self.p):
                upper = max(upper, np.abs(self.L[a * r:(a + 1) * r, b * r:(b + 1) * r]).max())
        errs["L_upper_blocks"] = upper
        scale = max(1.0, np.linalg.norm(T) ** 2)
        return {k: v / (scale if k in ("W3", "H1") else max(1.0, np.linalg.norm(T))) for k, v in errs.items()}, n


def rtilde(theta, r: int, tau: float) -> int:
    """Alg. 1 step 2, eq. (tau): the smallest j with r <= j < pr (1-based)
    whose eigen-gap |theta_j - theta_{j+1}| exceeds theta_pr * eps_m / tau,
    for the ascending eigenvalues theta of H(z) (pr = len(theta)).  When no
    gap qualifies (the paper's minimum over an empty set) the whole basis is
    kept: r~ = pr."""
    theta = np.asarray(theta, dtype=np.float64)
    k = theta.size
    thresh = theta[-1] * EPS_M / tau
    for j in range(r, k):  # 1-based j in [r, pr-1] <-> theta[j-1], theta[j]
        if abs(theta[j - 1] - theta[j]) > thresh:
            return j
    return k


def recy_sing(st: RecycleState, z: complex, eps: float, tau: float):
    """Alg. 1.  Returns dict with xi (ascending, first r), X (n x r), the
    residual norms ||W~_{:,j}||, r~ and theta."""
    r, k = st.r, st.k
    V, W1, W3, W4 = st.V, st.W1, st.W3, st.W4
    zc = np.conj(z)
    H = st.H1 - z * st.H2 - zc * st.H2.conj().T + (abs(z) ** 2 + eps) * np.eye(k)
    H = 0.5 * (H + H.conj().T)
    theta, G = np.linalg.eigh(H)  # ascending
    rt = rtilde(theta, r, tau)
    Gr = G[:, :rt]
    Y = (W1 - z * V) @ Gr
    _, Rt = np.linalg.qr(Y)
    _, s, Vh = np.linalg.svd(Rt)
    order = np.argsort(s)
    xi = s[order]
    Gt = Vh.conj().T[:, order]
    C = Gr @ Gt[:, :r]
    X = V @ C
    Wt = (W3 - z * W4 - zc * W1 + abs(z) ** 2 * V) @ C - X * (xi[:r] ** 2)
    return {"xi": xi, "X": X, "C": C, "wnorm": np.linalg.norm(Wt, axis=0), "rt": rt, "theta": theta}


def prune_count(V: np.ndarray, x1: np.ndarray, r: int, omega: float, p_max: int) -> int:
    """Alg. 2 steps 2-8 with eq. (omegaCond): how many leading r-column
    blocks of V to drop before x1 (n x r-breve, the leading columns of the new
    block) is appended.  rho_0 is the part of x1 outside span V, rho_j the
    part outside the span of the blocks j+1..p; the loop stops at the first j
    with rho_j / rho_0 > omega and l = j - 1, or l = p when it never stops
    (rho_j only grows with j, so this l is the largest j for which eq.
    (omegaCond) holds).  The cap of p_max blocks then raises l to
    p + 1 - p_max if needed.  Returns -1 when x1 already lies in span V
    (rho_0 <= 1e-12 ||x1||; nothing is appended)."""
    p = V.shape[1] // r
    rho0 = np.linalg.norm(x1 - V @ (V.conj().T @ x1))
    if rho0 <= 1e-12 * np.linalg.norm(x1):
        return -1
    l = p
    for j in range(1, p + 1):
        Vj = V[:, j * r:]
        rhoj = np.linalg.norm(x1 - Vj @ (Vj.conj().T @ x1))
        if rhoj / rho0 > omega:
            l = j - 1
            break
    if p - l + 1 > p_max:
        l = p + 1 - p_max
    return l


def update_recy(st: RecycleState, X: np.ndarray, omega: float, p_max: int, rb: int = 1):
    """Alg. 2 for the new block X (n x r).  Returns (l, skipped)."""
    T, r = st.T, st.r
    if st.V is None:
        Q, U = np.linalg.qr(X)
        st.V, st.L, st.X_blocks = Q, U.copy(), [X.copy()]
        _refresh_aux_for(st)
        return 0, False
    p = st.p
    l = prune_count(st.V, X[:, :rb], r, omega, p_max)
    if l < 0:
        return -1, True
    lr = l * r
    # drop the first l blocks
    V = st.V[:, lr:]
    L = st.L[lr:, lr:]
    blocks = st.X_blocks[l:]
    W1, W3, W4 = st.W1[:, lr:], st.W3[:, lr:], st.W4[:, lr:]
    H1, H2 = st.H1[lr:, lr:], st.H2[lr:, lr:]
    kk = V.shape[1]
    # block Gram--Schmidt (eq. (blkGS)), twice
    U = V.conj().T @ X
    Xp = X - V @ U
    U2 = V.conj().T @ Xp
    Xp = Xp - V @ U2
    U = U + U2
    Vn, Unn = np.linalg.qr(Xp)
    Vfull = np.hstack([V, Vn])
    Lfull = np.zeros((kk + r, kk + r), dtype=np.complex128)
    Lfull[:kk, :kk] = L
    Lfull[:kk, kk:] = U
    Lfull[kk:, kk:] = Unn
    W1n, W4n = T @ Vn, T.conj().T @ Vn
    W3n = T.conj().T @ W1n
    W1f, W3f, W4f = np.hstack([W1, W1n]), np.hstack([W3, W3n]), np.hstack([W4, W4n])
    H1f = W1f.conj().T @ W1f
    H2f = W1f.conj().T @ Vfull
    # restore block lower-triangular L by block-unitary transforms Q_j
    for j in range(kk // r):
        rows_new = np.arange(kk, kk + r)
        rows_j = np.arange(j * r, (j + 1) * r)
        idx = np.concatenate([rows_new, rows_j])
        Yj = Lfull[idx][:, kk:]
        Qloc, _ = np.linalg.qr(Yj, mode="complete")
        Lfull[idx, :] = Qloc.conj().T @ Lfull[idx, :]
        Lfull[rows_j[:, None], np.arange(kk, kk + r)[None, :]] = 0.0
        Vfull[:, idx] = Vfull[:, idx] @ Qloc
        for M in (W1f, W3f, W4f):
            M[:, idx] = M[:, idx] @ Qloc
        for M in (H1f, H2f):
            M[idx, :] = Qloc.conj().T @ M[idx, :]
            M[:, idx] = M[:, idx] @ Qloc
    st.V, st.L, st.X_blocks = Vfull, Lfull, blocks + [X.copy()]
    st.W1, st.W3, st.W4, st.H1, st.H2 = W1f, W3f, W4f, H1f, H2f
    return l, False


def _refresh_aux_for(st: RecycleState):
    T, V = st.T, st.V
    st.W1 = T @ V
    st.W3 = T.conj().T @ st.W1
    st.W4 = T.conj().T @ V
    st.H1 = st.W1.conj().T @ st.W1
    st.H2 = st.W1.conj().T @ V
