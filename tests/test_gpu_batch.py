"""Many matrices in one call against the Jacobi-SVD oracle.

A batch of independent complex Gaussian matrices N(0, 1/n) with sizes drawn
log-uniformly (the multi-matrix workload scaled down so that the oracle
finishes in seconds), each on its own grid over [-1.5, 1.5]^2 with a different
point count (one of them empty).  Every point of every matrix is compared with
the oracle under the pass rule of tests/parity.py, and every matrix's result
must equal what the single-matrix call returns for it."""
import numpy as np
import pytest

import oracle
from paper_2606_26785_b300 import workloads
from tests.parity import check_sigma

pytestmark = pytest.mark.gpu

EPS = workloads.EPS_LEVELS


@pytest.fixture(scope="module")
def batch():
    sizes = workloads.gaussian_batch_sizes(5, seed=11, lo=48, hi=320)
    mats = workloads.gaussian_batch(5, seed=11, lo=48, hi=320)
    shapes = [(7, 5), (12, 9), (0, 0), (6, 11), (10, 10)]
    probs = []
    for n, C, (nx, ny) in zip(sizes, mats, shapes):
        T, _, schur_err = workloads.schur(C)
        z = workloads.grid(-1.5, 1.5, -1.5, 1.5, nx, ny) if nx else np.zeros(0, np.complex128)
        ref, off = oracle.sigma_min_grid(C, z) if z.size else (np.zeros(0), np.zeros(0))
        probs.append((n, C, T, schur_err, z, ref, off))
    return probs


@pytest.mark.parametrize("precision,rtol", [(0, 1e-10), (1, 1e-8)])
def test_batch_matches_oracle_and_single_calls(batch, precision, rtol):
    import paper_2606_26785_b300 as p

    hs = [p.Pseudo(T) for (_, _, T, _, _, _, _) in batch]
    outs, rc = p.grid_batch(hs, [pr[4] for pr in batch], EPS, mode=p.INVLANC, precision=precision, rtol=rtol)
    assert rc in (0, 1)
    for h, out, (n, C, T, schur_err, z, ref, off) in zip(hs, outs, batch):
        sig = out["sigma"].cpu().numpy()
        assert sig.shape == z.shape
        if not z.size:
            continue
        rep = check_sigma(sig, ref, n=n, fro=np.linalg.norm(C), schur_err=schur_err, oracle_off=off, rtol=rtol,
                          eps_levels=EPS, member=out["member"].cpu().numpy())
        assert rep["n_bad"] == 0 and rep["member_mismatch"] == 0, (n, rep)
        single = h.grid(z, EPS, mode=p.INVLANC, precision=precision, rtol=rtol)["sigma"].cpu().numpy()
        assert np.array_equal(sig, single), n
    for h in hs:
        h.close()


def test_batch_rejects_repeated_handle(batch):
    import paper_2606_26785_b300 as p

    h = p.Pseudo(batch[0][2])
    z = batch[0][4]
    with pytest.raises(p.PseudoError):
        p.grid_batch([h, h], [z, z], mode=p.INVLANC)
    h.close()


def test_multi_matrix_workload_sampled():
    """The multi-matrix workload at full grid size (64 x 64 points per matrix)
    on the first 16 matrices of its sequence, in one batched call in mixed
    precision; stored oracle values (tests/golden/batch16_samples.json,
    written by tests/golden/make_batch_samples.py) at 24 points of the 8
    smallest matrices, and at every point the bound sigma_min(T - zI) <=
    min_i |t_ii - z| (the smallest singular value never exceeds the modulus
    of an eigenvalue)."""
    import json
    from pathlib import Path

    import paper_2606_26785_b300 as p

    g = json.loads((Path(__file__).parent / "golden" / "batch16_samples.json").read_text())
    sizes = workloads.gaussian_batch_sizes(64, 40)[: g["count"]]
    assert sizes == g["sizes"]
    mats = workloads.gaussian_batch(64, 40)[: g["count"]]
    z = workloads.grid(-1.5, 1.5, -1.5, 1.5, g["nx"], g["nx"])
    Ts, errs = [], []
    for C in mats:
        T, _, e = workloads.schur(C)
        Ts.append(T)
        errs.append(e)
    hs = [p.Pseudo(T) for T in Ts]
    outs, rc = p.grid_batch(hs, [z] * len(hs), EPS, mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    sig = [o["sigma"].cpu().numpy() for o in outs]
    for m, T in enumerate(Ts):
        d = np.min(np.abs(np.diag(T)[None, :] - z[:, None]), axis=1)
        assert np.all(sig[m] <= d * (1 + 1e-8) + 1e-12), m
        assert np.all(sig[m] >= 0.0)
    for smp in g["samples"]:
        m, i = smp["matrix"], smp["index"]
        rep = check_sigma(np.array([sig[m][i]]), np.array([smp["sigma_ref"]]), n=smp["n"], fro=smp["fro_norm"],
                          schur_err=errs[m], oracle_off=np.array([smp["oracle_off"]]), rtol=1e-8)
        assert rep["n_bad"] == 0, (smp, sig[m][i], rep)
    for h in hs:
        h.close()
