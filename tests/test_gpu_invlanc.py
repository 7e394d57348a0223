"""Inverse-Lanczos grid path against the Jacobi-SVD oracle.

Grcar n = 100 on the full 50 x 50 grid over [-1, 3] x [-3.5, 3.5]: every one
of the 2,500 points is compared (FP64 at rtol 1e-10, mixed at 1e-8, under the
pass rule of tests/parity.py), with identical epsilon-membership."""
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


@pytest.mark.parametrize("precision,rtol", [(0, 1e-10), (1, 1e-8)])
def test_grcar_full_grid(grcar, precision, rtol):
    import paper_2606_26785_b300 as p

    W, ref, off = grcar
    h = p.Pseudo(W.T)
    out = h.grid(W.z, EPS, mode=p.INVLANC, precision=precision, rtol=rtol)
    sig = out["sigma"].cpu().numpy()
    rep = check_sigma(sig, ref, n=W.n, fro=np.linalg.norm(W.C), schur_err=W.schur_err, oracle_off=off, rtol=rtol,
                      eps_levels=EPS, member=out["member"].cpu().numpy())
    print(rep, h.stats())
    assert rep["n_bad"] == 0, rep
    assert rep["member_mismatch"] == 0, rep
    h.close()


def test_host_io_matches_device_io(grcar):
    import paper_2606_26785_b300 as p

    W, ref, off = grcar
    h = p.Pseudo(W.T)
    z = W.z[:300]
    a = h.grid(z, EPS, mode=p.INVLANC, precision=0)
    b = h.grid_host(z, EPS, mode=p.INVLANC, precision=0)
    assert np.array_equal(a["sigma"].cpu().numpy(), b["sigma"])
    assert np.array_equal(a["member"].cpu().numpy().astype(np.uint32), b["member"])
    h.close()


def test_small_waves_and_ragged_tail(grcar):
    import paper_2606_26785_b300 as p

    W, ref, off = grcar
    h = p.Pseudo(W.T)
    z = W.z[:203]
    a = h.grid(z, EPS, mode=p.INVLANC, precision=0, shift_batch=37)["sigma"].cpu().numpy()
    rep = check_sigma(a, ref[:203], n=W.n, fro=np.linalg.norm(W.C), schur_err=W.schur_err, oracle_off=off,
                      rtol=1e-10)
    assert rep["n_bad"] == 0, rep
    h.close()
