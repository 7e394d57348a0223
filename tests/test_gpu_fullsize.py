"""Full-size parity on the dense complex Gaussian workload (n = 2000, seed 2,
200 x 200 grid over [-1.5, 1.5]^2) in the launch configuration bench.py
times, against stored oracle values at 32 sampled grid points
(tests/golden/gaussian2000_samples.json, written by the oracle alone), with
identical epsilon-membership there, plus
the strongly nonnormal triangular workload (n = 8000, seed 3) where the mixed
path is compared with the FP64 path at every point of a coarse sub-grid."""
import json
from pathlib import Path

import numpy as np
import pytest

from paper_2606_26785_b300 import workloads
from tests.parity import check_sigma

pytestmark = pytest.mark.gpu
GOLD = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def gauss():
    W = workloads.make("gaussian")
    g = json.loads((GOLD / "gaussian2000_samples.json").read_text())
    return W, g


@pytest.mark.parametrize("mode,precision,rtol", [("invlanc", 1, 1e-8), ("recycle", 1, 1e-8), ("invlanc", 0, 1e-10)])
def test_gaussian2000_full_grid(gauss, mode, precision, rtol):
    import paper_2606_26785_b300 as p

    W, g = gauss
    h = p.Pseudo(W.T)
    idx = np.array(g["index"])
    if mode == "invlanc":
        z = W.z if precision == 1 else W.z[idx]
        out = h.grid(z, workloads.EPS_LEVELS, mode=p.INVLANC, precision=precision, rtol=rtol)
        sig, mem = out["sigma"].cpu().numpy(), out["member"].cpu().numpy()
        if precision == 1:
            sig, mem = sig[idx], mem[idx]
    else:
        out = h.grid(W.z, workloads.EPS_LEVELS, mode=p.RECYCLE, precision=precision, rtol=rtol, r=4, p_max=4,
                     grid_nx=W.nx, grid_ny=W.ny, batch_b=20)
        sig, mem = out["sigma"].cpu().numpy()[idx], out["member"].cpu().numpy()[idx]
    rep = check_sigma(sig, np.array(g["sigma_ref"]), n=W.n, fro=g["fro_norm"], schur_err=W.schur_err,
                      oracle_off=np.array(g["oracle_off"]), rtol=rtol, eps_levels=workloads.EPS_LEVELS, member=mem)
    print(mode, precision, rep, h.stats())
    assert rep["n_bad"] == 0 and rep["member_mismatch"] == 0, rep
    h.close()


def test_triangular8000_mixed_matches_fp64():
    import paper_2606_26785_b300 as p

    T = workloads.triangular(8000, 3)
    z = workloads.grid(-1.5, 1.5, -1.5, 1.5, 300, 300)[:: 353]  # 255 points spread over the grid
    h = p.Pseudo(T)
    a = h.grid(z, (), mode=p.INVLANC, precision=p.FP64, rtol=1e-10)["sigma"].cpu().numpy()
    b = h.grid(z, (), mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)["sigma"].cpu().numpy()
    fro = float(np.linalg.norm(T))
    ok = a >= 1e-8 * fro
    err = np.abs(a - b)
    assert np.all(err[ok] <= 1e-8 * a[ok] + 4 * 8000 * 2.2e-16 * fro), float((err[ok] / a[ok]).max())
    h.close()


def test_triangular8000_stored_oracle_points():
    """The strongly nonnormal triangular workload (n = 8000, seed 3, 300 x 300
    grid) in the launch configuration bench.py times (strided batches of every
    20th grid point, mixed precision, rtol 1e-8) against the stored oracle
    values at the grid's rim (tests/golden/triangular8000_samples.json, written
    by tests/golden/make_triangular_samples.py), under the pass rule including
    the relative-only test above 1e-6 ||T||_F, with identical membership."""
    import paper_2606_26785_b300 as p

    g = json.loads((GOLD / "triangular8000_samples.json").read_text())
    T = workloads.triangular(g["n"], 3)
    z = workloads.grid(-1.5, 1.5, -1.5, 1.5, g["nx"], g["ny"])
    h = p.Pseudo(T)
    got, mem = {}, {}
    for b in sorted({i % 20 for i in g["index"]}):
        idx = np.arange(b, z.size, 20)
        out = h.grid(z[idx], workloads.EPS_LEVELS, mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
        sig, m = out["sigma"].cpu().numpy(), out["member"].cpu().numpy()
        for j, i in enumerate(idx):
            got[int(i)], mem[int(i)] = sig[j], m[j]
    sig = np.array([got[i] for i in g["index"]])
    member = np.array([mem[i] for i in g["index"]])
    rep = check_sigma(sig, np.array(g["sigma_ref"]), n=g["n"], fro=g["fro_norm"], schur_err=0.0,
                      oracle_off=np.array(g["oracle_off"]), rtol=1e-8, eps_levels=workloads.EPS_LEVELS,
                      member=member)
    print(rep)
    assert rep["n_bad"] == 0 and rep["member_mismatch"] == 0, rep
    assert rep["n_rel_only"] == len(g["index"]), rep
    h.close()


@pytest.mark.parametrize("mode,k", [("recycle", 8), ("recycle", 32), ("recycle", 64), ("invlanc", 0)])
def test_toeplitz1200_mixed(mode, k):
    """The banded Toeplitz + noise workload, reduced to n = 1200 on a 50 x 50
    grid over the full-size window, in mixed precision: the recycling path with
    recycled rank k (r = 4, p_max = k / 4) and the inverse-Lanczos path, against
    stored oracle values (tests/golden/toeplitz1200_samples.json, written by
    tests/golden/make_toeplitz_samples.py).  Outside the symbol's ellipse the
    smallest singular values of a large banded Toeplitz matrix crowd together,
    so at some points the iteration caps (64 Lanczos steps, 60 LOBPCG
    iterations) cannot separate sigma_min from its neighbours: those points must
    be reported as not converged, with an upper bound within 1e-3.  At k = 64
    the second Rayleigh--Ritz step keeps at most 16 of the r~ columns eq. (tau)
    asks for; how often that cap binds is printed (it costs acceptances, not
    accuracy: the returned pair comes from a subspace of span V and passes the
    same acceptance test)."""
    import paper_2606_26785_b300 as p

    g = json.loads((GOLD / "toeplitz1200_samples.json").read_text())
    C = workloads.toeplitz_noisy(g["n"], 5)
    T, _, err = workloads.schur(C)
    z = workloads.grid(-1.5, 1.5, -1.0, 1.0, g["nx"], g["ny"])
    idx = np.array(g["index"])
    assert np.allclose(z[idx], np.array([complex(a, b) for a, b in g["z"]]))
    h = p.Pseudo(T)
    if mode == "recycle":
        out = h.grid(z, workloads.EPS_LEVELS, mode=p.RECYCLE, precision=p.MIXED, rtol=1e-8, r=4, p_max=k // 4,
                     grid_nx=g["nx"], grid_ny=g["ny"], batch_b=20)
    else:
        out = h.grid(z, workloads.EPS_LEVELS, mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    sig = out["sigma"].cpu().numpy()[idx]
    flags = out["flags"].cpu().numpy()[idx]
    mem = out["member"].cpu().numpy()[idx]
    ref = np.array(g["sigma_ref"])
    unconv = (flags & p._abi.PT_NOT_CONVERGED) != 0
    rel = np.abs(sig - ref) / ref
    print(mode, k, h.stats(), [f"{r:.1e}{'*' if u else ''}" for r, u in zip(rel, unconv)])
    # every point meets the pass rule unless the library reports it as not
    # converged (a cluster of nearly equal singular values the iteration caps
    # cannot resolve); such estimates stay upper bounds and close to sigma_min
    rep = check_sigma(sig[~unconv], ref[~unconv], n=g["n"], fro=g["fro_norm"], schur_err=err,
                      oracle_off=np.array(g["oracle_off"])[~unconv], rtol=1e-8, eps_levels=workloads.EPS_LEVELS,
                      member=mem[~unconv])
    assert rep["n_bad"] == 0 and rep["member_mismatch"] == 0, rep
    assert np.all(sig[unconv] >= ref[unconv] * (1 - 1e-12)), rel[unconv]
    assert np.all(rel[unconv] <= 1e-3), rel[unconv]
    assert (~unconv).sum() >= len(ref) // 4, unconv
    h.close()
