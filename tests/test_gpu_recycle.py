"""Recycling path (Alg. 3 with Alg. 1 / Alg. 2 / Alg. SM1.2) against the
Jacobi-SVD oracle, plus algebraic facts that hold at any size:

* a full basis (k = n on a tiny matrix) makes the recycled Ritz value exact;
* every accepted Ritz value is an upper bound of sigma_min (Courant--Fischer);
* the counter identity mv_M = 3 r * (#updates) of Table 2.
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
    accepted, and every accepted Ritz value is >= sigma_min."""
    n = 100
    C = workloads.toeplitz_noisy(n, 5)
    T, _, err = workloads.schur(C)
    z = workloads.grid(-1.5, 1.5, -1.0, 1.0, 40, 40)
    W = workloads.Workload("toeplitz100", C, T, z, 40, 40, err)
    ref, off = oracle.sigma_min_grid(C, z)
    out, st = _run(W, 0, 0.0, batch_b=20)
    acc = (out["flags"] & 1) != 0
    assert acc.sum() > 0.05 * z.size, st
    assert np.all(out["sigma"][acc] >= ref[acc] * (1 - 1e-12) - 1e-14)
    # paper mode still meets the backward-stability bound eta at accepted points
    assert np.all(out["res"][acc] <= 1e-4 * (1 + 1e-9))
