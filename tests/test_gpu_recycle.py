"""Recycling path (Alg. 3 with Alg. 1 / Alg. 2 / Alg. SM1.2) against the
Jacobi-SVD oracle, plus algebraic facts that hold at any size:

* a full basis (k = n on a tiny matrix) makes the recycled Ritz value exact;
* every accepted Ritz value is an upper bound of sigma_min (Courant--Fischer);
* the counter identity mv_M = 3 r * (#updates) of Table 2;
* the per-phase times (recySing, refinement, values, updateRecy) are filled
  and add up to no more than the call.
"""
import numpy as np
import pytest

import oracle
from paper_2606_26785_b300 import workloads
from tests.parity import check_sigma

pytestmark = pytest.mark.gpu

EPS = workloads.EPS_LEVELS


@pytest.fixture(scope="module")
def grcar():
    W = workloads.make("grcar")
    ref, off = oracle.sigma_min_grid(W.C, W.z)
    return W, ref, off


def _run(W, precision, rtol, **kw):
    import paper_2606_26785_b300 as p

    h = p.Pseudo(W.T)
    opts = dict(mode=p.RECYCLE, precision=precision, rtol=rtol, r=4, p_max=4, grid_nx=W.nx, grid_ny=W.ny, batch_b=10)
    opts.update(kw)
    out = h.grid(W.z, EPS, **opts)
    st = h.stats()
    h.close()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}, st


@pytest.mark.parametrize("precision,rtol", [(0, 1e-10), (1, 1e-8)])
def test_grcar_recycle_full_grid(grcar, precision, rtol):
    W, ref, off = grcar
    out, st = _run(W, precision, rtol)
    rep = check_sigma(out["sigma"], ref, n=W.n, fro=np.linalg.norm(W.C), schur_err=W.schur_err, oracle_off=off,
                      rtol=rtol, eps_levels=EPS, member=out["member"])
    print(rep, st)
    assert rep["n_bad"] == 0, rep
    assert rep["member_mismatch"] == 0, rep
    assert st["n_accepted"] + st["n_refined"] == W.z.size
    assert st["mv_M"] == 3 * 4 * st["n_updates"]
    # per-phase device time in the paper's breakdown: every phase ran, and the
    # phases (disjoint stretches of the stream) fit inside the whole call
    phases = [st[k] for k in ("ms_recysing", "ms_refine", "ms_polish", "ms_update")]
    assert all(t > 0.0 for t in phases), st
    assert sum(phases) <= st["ms_total"] * 1.001 + 1e-3, st


@pytest.mark.parametrize("traversal", [1, 2])
@pytest.mark.parametrize("precision,rtol", [(0, 1e-10), (1, 1e-8)])
def test_grcar_recycle_hilbert_morton(grcar, traversal, precision, rtol):
    """The Hilbert (1) and Morton (2) grid orders that Sec. 5 names, on the
    full Grcar grid, every point against the oracle; the acceptance count of
    each order is printed (the recycled subspace follows the visiting order)."""
    W, ref, off = grcar
    out, st = _run(W, precision, rtol, traversal=traversal, lanes=1)
    rep = check_sigma(out["sigma"], ref, n=W.n, fro=np.linalg.norm(W.C), schur_err=W.schur_err, oracle_off=off,
                      rtol=rtol, eps_levels=EPS, member=out["member"])
    print("traversal", traversal, "precision", precision, "accepted", st["n_accepted"], "of", W.z.size, rep)
    assert rep["n_bad"] == 0, rep
    assert rep["member_mismatch"] == 0, rep
    assert st["n_accepted"] + st["n_refined"] == W.z.size
    assert st["mv_M"] == 3 * 4 * st["n_updates"]


def test_full_basis_makes_ritz_exact():
    # n = 8, r = 4, p_max = 2 -> k = 8 = n once two blocks are recycled
    rng = np.random.default_rng(5)
    n = 8
    C = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    T, _, err = workloads.schur(C)
    z = workloads.grid(-1, 1, -1, 1, 12, 12)
    W = workloads.Workload("tiny", C, T, z, 12, 12, err)
    ref, off = oracle.sigma_min_grid(C, z)
    out, st = _run(W, 0, 1e-10, p_max=2, lanes=1, batch_b=4, omega=1.0)
    rep = check_sigma(out["sigma"], ref, n=n, fro=np.linalg.norm(C), schur_err=err, oracle_off=off, rtol=1e-10)
    assert rep["n_bad"] == 0, rep
    assert st["n_accepted"] > 0.5 * z.size, st


def test_accepted_values_are_upper_bounds():
    """Paper-mode acceptance (eq. (tolC) only) on a banded Toeplitz matrix plus
    noise, where neighbouring singular subspaces are close: points must get
    accepted, and every accepted Ritz value is >= sigma_min.

    The acceptance rate depends on how accurate the recycled vectors are:
    eq. (tolC) at a neighbouring point needs a vector error of about
    eta * sigma / ||M(z)||, while LOBPCG-SVD stopped by eq. (tolSVD) only
    guarantees about eta.  With exact refinement the sequential method accepts
    about 25% of this grid, with refinement errors of 1e-6 about 23% and with
    1e-4 none; the GPU path with paper-mode LOBPCG lands in between (about
    4%), so the test asks for at least 1%."""
    n = 100
    C = workloads.toeplitz_noisy(n, 5)
    T, _, err = workloads.schur(C)
    z = workloads.grid(-1.5, 1.5, -1.0, 1.0, 40, 40)
    W = workloads.Workload("toeplitz100", C, T, z, 40, 40, err)
    ref, off = oracle.sigma_min_grid(C, z)
    out, st = _run(W, 0, 0.0, batch_b=20)
    acc = (out["flags"] & 1) != 0
    assert acc.sum() >= 0.01 * z.size, st
    assert np.all(out["sigma"][acc] >= ref[acc] * (1 - 1e-12) - 1e-14)
    # paper mode still meets the backward-stability bound eta at accepted points
    assert np.all(out["res"][acc] <= 1e-4 * (1 + 1e-9))


def test_update_invariants_from_exported_state():
    """After a recycle run the lane state satisfies the identities Alg. 2
    maintains: V^H V = I, W1 = T V, W3 = T^H T V, W4 = T^H V, H1 = W1^H W1,
    H2 = W1^H V, and L block lower triangular (updates with pruning and
    block-unitary restoration have happened on the way)."""
    import torch

    import paper_2606_26785_b300 as p

    n = 100
    C = workloads.toeplitz_noisy(n, 5)
    T, _, err = workloads.schur(C)
    z = workloads.grid(-1.5, 1.5, -1.0, 1.0, 12, 12)
    h = p.Pseudo(T)
    o = p.default_opts(mode=p.RECYCLE, precision=0, rtol=0.0, r=4, p_max=4, grid_nx=12, grid_ny=12, batch_b=6,
                       lanes=1)
    ws = torch.empty(h.workspace_bytes(z.size, o), dtype=torch.uint8, device="cuda")
    h.grid(z, (), opts=o, workspace=ws)
    st = h.stats()
    lane = h.recycle_state(z.size, o, ws)[0]
    V, W1, W3, W4, H1, H2, L = (lane[k] for k in ("V", "W1", "W3", "W4", "H1", "H2", "L"))
    k = V.shape[1]
    nt = np.linalg.norm(T, 2)
    errs = {
        "orth": np.linalg.norm(V.conj().T @ V - np.eye(k)),
        "W1": np.linalg.norm(W1 - T @ V) / nt,
        "W3": np.linalg.norm(W3 - T.conj().T @ (T @ V)) / nt ** 2,
        "W4": np.linalg.norm(W4 - T.conj().T @ V) / nt,
        "H1": np.linalg.norm(H1 - W1.conj().T @ W1) / nt ** 2,
        "H2": np.linalg.norm(H2 - W1.conj().T @ V) / nt,
    }
    r = 4
    upper = max([np.abs(L[a * r:(a + 1) * r, b * r:(b + 1) * r]).max() for a in range(k // r)
                 for b in range(a + 1, k // r)] + [0.0])
    print(k, st, errs, upper)
    assert k >= 4 and st["n_updates"] >= 2
    assert all(v < 1e-10 for v in errs.values()), errs
    assert upper < 1e-12
    assert st["mv_M"] == 3 * r * (st["n_updates"])
    h.close()
