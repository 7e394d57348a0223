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


@pytest.mark.parametrize("solver", [1, 3, 4])
def test_grcar_mixed_every_fp32_solver(grcar, solver):
    """Mixed precision with each FP32 solver forced (CUDA cores; tensor cores
    with 16 or 32 right-hand sides per CTA, the column-group forms the tuned
    table chooses between): every grid point against the oracle at 1e-8,
    identical membership."""
    import paper_2606_26785_b300 as p

    W, ref, off = grcar
    h = p.Pseudo(W.T)
    out = h.grid(W.z, EPS, mode=p.INVLANC, precision=p.MIXED, rtol=1e-8, fp32_solver=solver)
    rep = check_sigma(out["sigma"].cpu().numpy(), ref, n=W.n, fro=np.linalg.norm(W.C), schur_err=W.schur_err,
                      oracle_off=off, rtol=1e-8, eps_levels=EPS, member=out["member"].cpu().numpy())
    print(solver, rep)
    assert rep["n_bad"] == 0 and rep["member_mismatch"] == 0, rep
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


@pytest.mark.parametrize("precision", [0, 1])
def test_device_loop_matches_host_loop(grcar, precision):
    """The graph-driven loop (conditional nodes decide every step, finish and
    stop on the device) runs the same kernels on the same columns as the
    host-driven loop: the results agree bit for bit, also with waves that
    finish mid-grid (shift_batch 37 on 2,500 points) and a ragged tail."""
    import paper_2606_26785_b300 as p

    W, ref, off = grcar
    h = p.Pseudo(W.T)
    kw = dict(mode=p.INVLANC, precision=precision, rtol=1e-10 if precision == 0 else 1e-8, shift_batch=37)
    h.reset_stats()
    a = h.grid(W.z, EPS, device_loop=1, **kw)
    sa = h.stats()
    h.reset_stats()
    b = h.grid(W.z, EPS, device_loop=0, **kw)
    sb = h.stats()
    assert sa["n_graph_launches"] >= 1 and sb["n_graph_launches"] == 0
    for k in ("sigma", "res", "flags", "member"):
        assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), k
    # the device-side counts of steps, solves and products equal the host loop's
    for k in ("lanczos_steps", "sv_R", "mv_M_fp64_refine", "n_fallback"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    h.close()


def test_device_loop_launch_count(grcar):
    """Kernels run by graph replays are counted (pseudo_launch_count): the
    device loop reports as many launches as the host loop, give or take the
    per-iteration control launches the host loop adds for its own reads."""
    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import _abi

    W, ref, off = grcar
    h = p.Pseudo(W.T)
    lib = _abi.load()
    kw = dict(mode=p.INVLANC, precision=1, rtol=1e-8, shift_batch=256)
    c0 = lib.pseudo_launch_count()
    h.grid(W.z, EPS, device_loop=1, **kw)
    c1 = lib.pseudo_launch_count()
    h.grid(W.z, EPS, device_loop=0, **kw)
    c2 = lib.pseudo_launch_count()
    assert c1 - c0 > 0
    assert abs((c1 - c0) - (c2 - c1)) <= 0.05 * (c2 - c1), (c1 - c0, c2 - c1)
    h.close()


def test_loop_graph_cache(grcar):
    """A repeated call with the same workspace, inputs and outputs replays the
    handle's cached loop graph (no new capture); other buffers get their own
    graph; results are the same bits every time."""
    import torch

    import paper_2606_26785_b300 as p

    W, ref, off = grcar
    h = p.Pseudo(W.T)
    o = p.default_opts(mode=p.INVLANC, precision=p.MIXED, rtol=1e-8)
    z = torch.from_numpy(W.z).cuda()
    ws = torch.empty(h.workspace_bytes(z.numel(), o), dtype=torch.uint8, device="cuda")
    h.reset_stats()
    a = h.grid(z, EPS, opts=o, workspace=ws)
    first = {k: v.clone() for k, v in a.items() if k != "status"}
    st1 = h.stats()  # the main pass's graph, and the FP64 pass's if points needed it
    assert 1 <= st1["n_graph_builds"] <= 2, st1
    for _ in range(3):
        h.grid(z, EPS, opts=o, workspace=ws, out=a)
    st = h.stats()
    assert st["n_graph_builds"] == st1["n_graph_builds"], st
    assert st["n_graph_launches"] >= st1["n_graph_launches"] + 3, st
    b = h.grid(z, EPS, opts=o, workspace=ws)  # fresh outputs: the main pass needs a new graph
    assert h.stats()["n_graph_builds"] == st1["n_graph_builds"] + 1
    for k in ("sigma", "res", "flags", "member"):
        assert torch.equal(first[k], a[k]) and torch.equal(first[k], b[k]), k
    h.close()
