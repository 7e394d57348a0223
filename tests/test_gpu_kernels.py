"""Multi-shift triangular solve and FP64 triangular product against the
step-level oracle, on sizes that span several 64-row panels, ragged tails
and 1/2/3-row matrices, with column counts that leave partial CTA groups."""
import numpy as np
import pytest

from oracle import steps

pytestmark = pytest.mark.gpu


def _case(n, ncols, seed):
    rng = np.random.default_rng(seed)
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    T[np.arange(n), np.arange(n)] += 1.5 * np.exp(2j * np.pi * rng.random(n))
    z = 0.5 * (rng.standard_normal(ncols) + 1j * rng.standard_normal(ncols))
    B = rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))
    return T, z, B


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 100, 257])
@pytest.mark.parametrize("ncols", [1, 3, 37])
@pytest.mark.parametrize("adjoint", [False, True])
def test_solve_fp64_and_mixed(n, ncols, adjoint):
    import torch

    import paper_2606_26785_b300 as p

    T, z, B = _case(n, ncols, 1000 * n + ncols)
    h = p.Pseudo(T)
    ref = steps.shifted_solve(T, z, B, adjoint)
    X = torch.from_numpy(B.copy()).cuda()
    h.solve(X, z, adjoint=adjoint, precision=p.FP64)
    got = X.cpu().numpy()
    rel = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() < 1e-12, rel.max()
    for prec in (p.MIXED, p.MIXED_CUDACORE):
        X = torch.from_numpy(B.copy()).cuda()
        h.solve(X, z, adjoint=adjoint, precision=prec)
        got = X.cpu().numpy()
        rel = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert rel.max() < 2e-4, (prec, rel.max())
    h.close()


@pytest.mark.parametrize("n", [127, 128, 129, 300, 520])
@pytest.mark.parametrize("ncols", [1, 16, 45])
@pytest.mark.parametrize("adjoint", [False, True])
def test_solve_fp32_tensor_cores(n, ncols, adjoint):
    """The tcgen05 solve (3xTF32 off-diagonal blocks, 128-row panels) across
    several panels with a ragged last panel and partial 16-column groups: its
    error against the oracle stays within a few FP32 units of the condition
    number, like the CUDA-core FP32 solve."""
    import torch

    import paper_2606_26785_b300 as p

    T, z, B = _case(n, ncols, 7000 + 1000 * n + ncols)
    h = p.Pseudo(T)
    ref = steps.shifted_solve(T, z, B, adjoint)
    errs = {}
    for prec in (p.MIXED, p.MIXED_CUDACORE):
        X = torch.from_numpy(B.copy()).cuda()
        h.solve(X, z, adjoint=adjoint, precision=prec)
        got = X.cpu().numpy()
        errs[prec] = (np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max()
    h.close()
    assert errs[p.MIXED] < 2e-5, errs
    assert errs[p.MIXED] < 30 * errs[p.MIXED_CUDACORE] + 1e-6, errs


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 300, 520])
@pytest.mark.parametrize("ncols", [1, 7, 37, 300, 333])
@pytest.mark.parametrize("adjoint", [False, True])
def test_solve_double_single(n, ncols, adjoint):
    """The double-single solve (FP32 pairs on the CUDA cores, the solve of the
    points the FP32 solves cannot serve) against the oracle's substitution:
    about 2^-46 relative per operation, so within 1e-11 on these
    well-conditioned shifts (FP32 solves: 1e-4), across ragged 64-row panels
    and both the narrow (up to 296 columns) and the 8-column groups."""
    import torch

    import paper_2606_26785_b300 as p

    T, z, B = _case(n, ncols, 3000 + 1000 * n + ncols)
    h = p.Pseudo(T)
    ref = steps.shifted_solve(T, z, B, adjoint)
    X = torch.from_numpy(B.copy()).cuda()
    h.solve(X, z, adjoint=adjoint, precision=p.DOUBLE_SINGLE)
    got = X.cpu().numpy()
    rel = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    h.close()
    assert rel.max() < 1e-11, rel.max()


@pytest.mark.parametrize("n", [1, 3, 65, 130])
@pytest.mark.parametrize("adjoint", [False, True])
def test_matvec_fp64(n, adjoint):
    import torch

    import paper_2606_26785_b300 as p

    T, z, B = _case(n, 5, 7 + n)
    X = np.random.default_rng(n).standard_normal((n, 5)) + 0j
    h = p.Pseudo(T)
    Xt = torch.from_numpy(X).cuda()
    Y = h.matvec(Xt, z=z, adjoint=adjoint).cpu().numpy()
    ref = steps.shifted_matvec(T, z, X, adjoint)
    assert np.max(np.abs(Y - ref)) <= 1e-13 * np.max(np.abs(ref))
    Bt = torch.from_numpy(B).cuda()
    R = h.matvec(Xt, z=z, B=Bt, adjoint=adjoint).cpu().numpy()
    assert np.max(np.abs(R - (B - ref))) <= 1e-13 * np.max(np.abs(B - ref))
    h.close()


@pytest.mark.parametrize("n", [3, 65, 257, 300])
@pytest.mark.parametrize("ncols", [6, 64, 131])
@pytest.mark.parametrize("adjoint", [False, True])
def test_matvec_double_single(n, ncols, adjoint):
    """double-single accurate products: the tensor-core slicing (PSEUDO_MIXED)
    and the CUDA-core double-single kernel, relative error near 2^-46, far
    below FP32's, across several 64-row tiles, ragged tails, partial
    64-column tiles and a column scaled by 1e-9 (per-column exponents)."""
    import torch

    import paper_2606_26785_b300 as p

    T, z, B = _case(n, ncols, 11 + n + ncols)
    rng = np.random.default_rng(n + 1)
    X = rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))
    X[:, 0] *= 1e-9
    h = p.Pseudo(T)
    Xt, Bt = torch.from_numpy(X).cuda(), torch.from_numpy(B).cuda()
    ref = steps.shifted_matvec(T, z, X, adjoint)
    # per column: sum_k |T_ik| |x_k| bounds the rounding of any summation order
    Ta = np.abs(np.triu(T))
    bound = ((Ta.T if adjoint else Ta) @ np.abs(X)).max(axis=0) + np.abs(z) * np.abs(X).max(axis=0)
    for prec in (p.MIXED, p.MIXED_CUDACORE):
        Y = h.matvec(Xt, z=z, adjoint=adjoint, precision=prec).cpu().numpy()
        err = np.abs(Y - ref).max(axis=0) / bound
        assert err.max() <= 64 * 2.0 ** -46, (prec, err.max())
        R = h.matvec(Xt, z=z, B=Bt, adjoint=adjoint, precision=prec).cpu().numpy()
        err = np.abs(R - (B - ref)).max(axis=0) / bound
        assert err.max() <= 64 * 2.0 ** -46, (prec, err.max())
    h.close()
    h.close()


def test_norms():
    import paper_2606_26785_b300 as p

    T, _, _ = _case(150, 1, 5)
    h = p.Pseudo(T)
    info = h.info()
    assert abs(info["norm_fro"] - np.linalg.norm(T)) <= 1e-12 * np.linalg.norm(T)
    s2 = np.linalg.norm(T, 2)
    assert 0.9 * s2 <= info["norm2_est"] <= s2 * (1 + 1e-12)
    h.close()
