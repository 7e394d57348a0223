"""Failure paths of the library on a GPU, each made on purpose in a form that
cannot fault or hang the device: a bounded wait whose limit is set to zero
(the tensor-core kernels give up, drain their copies and MMAs, release their
tensor memory and report PSEUDO_ERR_TIMEOUT), non-finite T or z
(PSEUDO_ERR_NONFINITE before any work), a workspace one byte short
(PSEUDO_ERR_WORKSPACE) and an iteration cap too small to converge
(PSEUDO_WARN_NOT_CONVERGED with flagged points and finite outputs).  After
every failure the handle must still give correct results."""
import numpy as np
import pytest

import oracle
from oracle import steps
from paper_2606_26785_b300 import workloads
from tests.parity import check_sigma

pytestmark = pytest.mark.gpu


def _tri(n, seed):
    rng = np.random.default_rng(seed)
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    T[np.arange(n), np.arange(n)] += 1.5 * np.exp(2j * np.pi * rng.random(n))
    return T, rng


@pytest.mark.parametrize("adjoint", [False, True])
def test_zero_wait_limit_times_out_and_handle_recovers(adjoint):
    import torch

    import paper_2606_26785_b300 as p

    n, ncols = 300, 40
    T, rng = _tri(n, 5)
    h = p.Pseudo(T)
    B = rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))
    z = 0.3 * (rng.standard_normal(ncols) + 1j * rng.standard_normal(ncols))
    h.set_wait_limit(0)
    # three 128-row panels: the second one's chunks wait for the first panel's
    # solve, which is never done at once, so the first wait gives up
    X = torch.from_numpy(B.copy()).cuda()
    with pytest.raises(p.PseudoError) as ei:
        h.solve(X, z, adjoint=adjoint, precision=p.MIXED)
    assert ei.value.code == p._abi.ERR_TIMEOUT
    # the slice product waits on its copies the same way; a copy that has
    # already landed when it is first tested needs no wait, so the product may
    # also finish: then its result must be right
    Xm = torch.from_numpy(B.copy()).cuda()
    try:
        Y = h.matvec(Xm, z=z, adjoint=adjoint, precision=p.MIXED)
        want = steps.shifted_matvec(T, z, B, adjoint=adjoint)
        rel = np.linalg.norm(Y.cpu().numpy() - want, axis=0) / np.linalg.norm(want, axis=0)
        assert rel.max() < 1e-12, rel.max()
    except p.PseudoError as err:
        assert err.code == p._abi.ERR_TIMEOUT
    torch.cuda.synchronize()
    # the default limit back: the same handle solves correctly
    h.set_wait_limit(10 ** 9)
    X = torch.from_numpy(B.copy()).cuda()
    h.solve(X, z, adjoint=adjoint, precision=p.MIXED)
    exact = steps.shifted_solve(T, z, B, adjoint=adjoint)
    rel = np.linalg.norm(X.cpu().numpy() - exact, axis=0) / np.linalg.norm(exact, axis=0)
    assert rel.max() < 1e-4, rel.max()
    h.close()


def test_zero_wait_limit_in_a_grid_call():
    import paper_2606_26785_b300 as p

    W = workloads.make("grcar", nx=10, ny=8, n=300)
    h = p.Pseudo(W.T)
    h.set_wait_limit(0)
    with pytest.raises(p.PseudoError) as ei:
        h.grid(W.z, workloads.EPS_LEVELS, mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    assert ei.value.code == p._abi.ERR_TIMEOUT
    h.set_wait_limit(10 ** 9)
    ref, off = oracle.sigma_min_grid(W.C, W.z)
    out = h.grid(W.z, workloads.EPS_LEVELS, mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    rep = check_sigma(out["sigma"].cpu().numpy(), ref, n=W.n, fro=np.linalg.norm(W.C), schur_err=W.schur_err,
                      oracle_off=off, rtol=1e-8)
    assert rep["n_bad"] == 0, rep
    h.close()


def test_non_finite_inputs():
    import torch

    import paper_2606_26785_b300 as p

    T, _ = _tri(64, 6)
    for bad in (np.nan, np.inf):
        Tb = T.copy()
        Tb[3, 40] = bad
        with pytest.raises(p.PseudoError) as ei:
            p.Pseudo(Tb)
        assert ei.value.code == p._abi.ERR_NONFINITE
    # below the diagonal nothing is read
    Tl = T.copy()
    Tl[40, 3] = np.nan
    h = p.Pseudo(Tl)
    z = np.array([0.1 + 0.1j, 0.2, -0.3j, 0.5 + 0.5j])
    good = h.grid(z, (), mode=p.INVLANC, precision=p.FP64)["sigma"].cpu().numpy()
    for zb in (complex(np.nan, 0.0), complex(0.0, np.inf)):
        zz = z.copy()
        zz[2] = zb
        for host in (False, True):
            with pytest.raises(p.PseudoError) as ei:
                if host:
                    h.grid_host(zz, (), mode=p.INVLANC, precision=p.FP64)
                else:
                    h.grid(torch.from_numpy(zz).cuda(), (), mode=p.INVLANC, precision=p.FP64)
            assert ei.value.code == p._abi.ERR_NONFINITE
    again = h.grid(z, (), mode=p.INVLANC, precision=p.FP64)["sigma"].cpu().numpy()
    assert np.array_equal(good, again)
    h.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_workspace_one_byte_short(mode):
    """Through the C ABI directly (the Python binding would allocate a big
    enough workspace itself): one byte short is refused before any launch,
    the exact size works."""
    import ctypes

    import torch

    import paper_2606_26785_b300 as p

    lib = p._abi.load()
    W = workloads.make("grcar", nx=6, ny=5, n=60)
    h = p.Pseudo(W.T)
    o = p.default_opts(mode=mode, precision=p.MIXED, rtol=1e-8, r=4, p_max=4, grid_nx=W.nx, grid_ny=W.ny, batch_b=5)
    need = h.workspace_bytes(W.z.size, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    z = torch.from_numpy(W.z).cuda()
    sig = torch.empty(W.z.size, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = ctypes.c_void_p

    def call(nbytes):
        return lib.pseudo_grid(h._h, vp(z.data_ptr()), W.z.size, None, 0, ctypes.byref(o), vp(sig.data_ptr()), None,
                               None, None, vp(ws.data_ptr()), nbytes, stream)

    before = lib.pseudo_launch_count()
    assert call(need - 1) == p._abi.ERR_WORKSPACE
    assert lib.pseudo_launch_count() == before
    assert b"workspace" in lib.pseudo_last_error()
    assert call(need) >= 0
    torch.cuda.synchronize()
    assert np.all(np.isfinite(sig.cpu().numpy()))
    h.close()


def test_iteration_cap_flags_points():
    import paper_2606_26785_b300 as p

    W = workloads.make("grcar", nx=10, ny=8, n=100)
    h = p.Pseudo(W.T)
    for prec in (p.FP64, p.MIXED):
        out = h.grid(W.z, workloads.EPS_LEVELS, mode=p.INVLANC, precision=prec, rtol=1e-10 if prec == p.FP64 else 1e-8,
                     maxiter_lanczos=1)
        assert out["status"] == p._abi.WARN_NOT_CONVERGED
        flags = out["flags"].cpu().numpy()
        sig, res = out["sigma"].cpu().numpy(), out["res"].cpu().numpy()
        assert ((flags & p._abi.PT_NOT_CONVERGED) != 0).sum() > 0
        assert np.all(np.isfinite(sig)) and np.all(np.isfinite(res)) and np.all(sig > 0)
        # an unconverged estimate is still the Rayleigh quotient of a vector: an upper bound
        ref, _ = oracle.sigma_min_grid(W.C, W.z)
        assert np.all(sig >= ref * (1 - 1e-10))
    h.close()
