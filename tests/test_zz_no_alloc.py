"""pseudo_solve_noalloc: the FP64 multi-shift solve for callers that cannot
allocate device memory (it runs on a fixed scratch array inside the library
instead of a caller workspace).  Checked through the C ABI against
pseudo_solve and against the oracle's textbook substitution on two calls in a
row, with different inputs, so that the second call runs on the scratch
contents the first one left behind.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from oracle import steps

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2606_26785_b300 import _abi

    lib = _abi.load()
    vp = ctypes.c_void_p
    lib.pseudo_solve_noalloc.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int, vp]
    lib.pseudo_solve_noalloc.restype = ctypes.c_int
    return lib


def _case(n, ncols, seed):
    rng = np.random.default_rng(seed)
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    T[np.arange(n), np.arange(n)] += 1.5 * np.exp(2j * np.pi * rng.random(n))
    return T, rng


@pytest.mark.parametrize("adjoint", [False, True])
def test_noalloc_solve_matches_workspace_solve_twice(adjoint):
    import torch

    import paper_2606_26785_b300 as p

    lib = _lib()
    n, ncols = 300, 37
    T, rng = _case(n, ncols, 42 + int(adjoint))
    h = p.Pseudo(T)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        B = rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))
        z = 0.5 * (rng.standard_normal(ncols) + 1j * rng.standard_normal(ncols))
        zt = torch.from_numpy(z).cuda()
        ref = torch.from_numpy(B.copy()).cuda()
        h.solve(ref, z, adjoint=adjoint, precision=p.FP64)
        X = torch.from_numpy(B.copy()).cuda()
        rc = lib.pseudo_solve_noalloc(h._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(zt.data_ptr()), ncols,
                                      int(adjoint), stream)
        assert rc == 0, lib.pseudo_last_error()
        torch.cuda.synchronize()
        got, want = X.cpu().numpy(), ref.cpu().numpy()
        rel = np.linalg.norm(got - want, axis=0) / np.linalg.norm(want, axis=0)
        assert rel.max() < 1e-12, (call, rel.max())
        exact = steps.shifted_solve(T, z, B, adjoint=adjoint)
        rel = np.linalg.norm(got - exact, axis=0) / np.linalg.norm(exact, axis=0)
        assert rel.max() < 1e-12, (call, rel.max())
    h.close()


def test_noalloc_rejects_oversized_calls():
    import torch

    import paper_2606_26785_b300 as p

    lib = _lib()
    n = 2000
    T, _ = _case(n, 1, 7)
    h = p.Pseudo(T)
    ncols = 4096  # needs 512 groups x 2048 rows x 8 > 2^20 scratch elements
    X = torch.zeros((n, ncols), dtype=torch.complex128, device="cuda")
    z = torch.zeros(ncols, dtype=torch.complex128, device="cuda")
    rc = lib.pseudo_solve_noalloc(h._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(z.data_ptr()), ncols, 0,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == p._abi.ERR_ARG
    assert b"scratch" in lib.pseudo_last_error()
    # a column count whose scratch size would overflow 64 bits is refused too,
    # before any launch (X and z are never touched)
    before = lib.pseudo_launch_count()
    rc = lib.pseudo_solve_noalloc(h._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                  (1 << 60) + 1000, 0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == p._abi.ERR_ARG and lib.pseudo_launch_count() == before
    # a successful call clears the message of the failed one
    rc = lib.pseudo_solve_noalloc(h._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(z.data_ptr()), 8, 0,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0 and lib.pseudo_last_error() == b""
    h.close()
