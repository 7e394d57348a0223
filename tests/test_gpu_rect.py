"""Rectangular input, m > n (SM2.2; a C with n < m < 2n is extended by zero
rows to 2n): FP64 inverse Lanczos on the 2n x n
pencil [T - zI; B] with one QR factorisation per point, against the oracle's
Jacobi SVD of the ORIGINAL rectangular C - zI (m x n, rectangular identity).

Workloads (seeded, paper_2606_26785_b300.workloads): a dense Gaussian
C (n = 150, m = 2n + 37), the m = 2n section of the banded Toeplitz
operator (superdiagonal 1, subdiagonal 0.25; a matrix folding, Sec. 1), and a
Gaussian with n < m < 2n (n = 120, m = 165, extended by zero rows), each on
a 40 x 40 grid with every point compared at rtol 1e-10 under the pass rule of
tests/parity.py, with identical epsilon-membership; a larger Gaussian
(n = 600) at sampled points; and the zero-bottom case that reduces to the
square path."""
import numpy as np
import pytest

import oracle
from paper_2606_26785_b300 import workloads
from tests.parity import check_sigma

pytestmark = pytest.mark.gpu

EPS = workloads.EPS_LEVELS


def _parity(W, sig, member, ref, off, rtol=1e-10):
    rep = check_sigma(sig, ref, n=W.n, fro=np.linalg.norm(W.C), schur_err=W.schur_err, oracle_off=off, rtol=rtol,
                      eps_levels=EPS if member is not None else (), member=member)
    print(rep)
    assert rep["n_bad"] == 0, rep
    if member is not None:
        assert rep["member_mismatch"] == 0, rep
    return rep


@pytest.mark.parametrize("name", ["rect_gaussian", "toeplitz_folding", "rect_gaussian_short"])
def test_rect_full_grid(name):
    import paper_2606_26785_b300 as p

    W = workloads.make(name)
    ref, off = oracle.sigma_min_grid(W.C, W.z)
    h = p.Pseudo(W.T)
    assert h.m == 2 * h.n
    out = h.grid(W.z, EPS, mode=p.INVLANC, precision=p.FP64, rtol=1e-10)
    _parity(W, out["sigma"].cpu().numpy(), out["member"].cpu().numpy(), ref, off)
    st = h.stats()
    assert st["n_points"] == W.z.size and st["n_not_converged"] == 0
    h.close()


def test_rect_waves_ragged_tail_and_host_loop():
    """Slots refilled mid-grid (shift_batch 37 over 203 points) rebuild their
    factor for every new point; the host-driven loop gives the same bits."""
    import paper_2606_26785_b300 as p

    W = workloads.make("toeplitz_folding")
    z = W.z[:203]
    ref, off = oracle.sigma_min_grid(W.C, z)
    h = p.Pseudo(W.T)
    kw = dict(mode=p.INVLANC, precision=p.FP64, rtol=1e-10, shift_batch=37)
    a = h.grid(z, EPS, device_loop=1, **kw)
    b = h.grid(z, EPS, device_loop=0, **kw)
    _parity(W, a["sigma"].cpu().numpy(), a["member"].cpu().numpy(), ref, off)
    for k in ("sigma", "res", "flags", "member"):
        assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), k
    h.close()


def test_rect_zero_bottom_block_is_the_square_problem():
    """C = [C_u; 0]: B = 0, every reflector is the identity, and sigma is that
    of the square C_u - zI, which the square (Schur) path computes too."""
    import paper_2606_26785_b300 as p

    n = 64
    Cu = workloads.gaussian(n, 21)
    C = np.vstack([Cu, np.zeros((n, n))])
    M, err = workloads.rect_reduce(C)
    assert np.all(M[n:] == 0)
    z = workloads.grid(-1.2, 1.2, -1.2, 1.2, 12, 12)
    hr = p.Pseudo(M)
    T, _, serr = workloads.schur(Cu)
    hs = p.Pseudo(T)
    a = hr.grid(z, EPS, mode=p.INVLANC, precision=p.FP64, rtol=1e-10)["sigma"].cpu().numpy()
    b = hs.grid(z, EPS, mode=p.INVLANC, precision=p.FP64, rtol=1e-10)["sigma"].cpu().numpy()
    ref, off = oracle.sigma_min_grid(C, z)
    W = workloads.Workload("zero_bottom", C, M, z, 12, 12, err)
    _parity(W, a, None, ref, off)
    assert np.max(np.abs(a - b) / b) <= 1e-10
    hr.close()
    hs.close()


def test_rect_larger_order_sampled():
    """n = 600 (m = 1237): factors of 180,300 packed entries per slot, solves
    with 38 KB of right-hand sides per CTA; 10 grid points against the oracle."""
    import paper_2606_26785_b300 as p

    W = workloads.make("rect_gaussian", n=600, nx=20, ny=20)
    idx = np.arange(0, W.z.size, 41)[:10]
    ref, off = oracle.sigma_min_grid(W.C, W.z[idx])
    h = p.Pseudo(W.T)
    out = h.grid(W.z, EPS, mode=p.INVLANC, precision=p.FP64, rtol=1e-10)
    _parity(W, out["sigma"].cpu().numpy()[idx], out["member"].cpu().numpy()[idx], ref, off)
    h.close()


def test_rect_refuses_other_modes():
    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import _abi

    W = workloads.make("toeplitz_folding", n=20, nx=4, ny=4)
    h = p.Pseudo(W.T)
    for kw in (dict(mode=p.INVLANC, precision=p.MIXED), dict(mode=p.RECYCLE, precision=p.FP64)):
        with pytest.raises(p.PseudoError) as ei:
            h.grid(W.z, EPS, **kw)
        assert ei.value.code == _abi.ERR_UNSUPPORTED
    h.close()
