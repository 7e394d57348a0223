"""B300 (sm_103a) pseudospectra library: sigma_min(C - zI) over a grid from
the complex Schur factor T of C, with hand-written CUDA kernels behind a C ABI
(include/pseudo.h).  This module is the thin Python binding: it marshals
arguments (device buffers come from PyTorch) and calls the library; every step
of the computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (  # noqa: F401
    DOUBLE_SINGLE, FP64, INVLANC, MIXED, MIXED_CUDACORE, RECYCLE, TRAVERSE_BATCH_ZIGZAG, TRAVERSE_HILBERT, TRAVERSE_MORTON, Opts,
    PseudoError, Stats, check)

__all__ = ["Pseudo", "grid_batch", "grid_batch_workspace_bytes", "traversal_order", "tuned_config", "default_opts", "FP64", "MIXED", "MIXED_CUDACORE",
           "DOUBLE_SINGLE", "INVLANC",
           "RECYCLE", "TRAVERSE_BATCH_ZIGZAG", "TRAVERSE_HILBERT", "TRAVERSE_MORTON", "PseudoError"]


def default_opts(**kw) -> Opts:
    o = Opts()
    _abi.load().pseudo_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _torch():
    import torch

    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Pseudo:
    """Handle on one Schur factor T (n x n, upper triangular, complex128), or
    on a rectangular pencil [T; B] (2n x n, both blocks upper triangular; see
    ``workloads.rect_reduce``, which takes any C with m > n rows)."""

    def __init__(self, T, stream=None):
        torch = _torch()
        lib = _abi.load()
        if isinstance(T, np.ndarray):
            Tt = torch.from_numpy(np.asfortranarray(T.astype(np.complex128)).T.copy()).cuda()
        else:
            Tt = T.to(device="cuda", dtype=torch.complex128).t().contiguous()
        # Tt holds T^T row-major == T column-major (m x n, leading dimension m)
        n, m = Tt.shape
        h = ctypes.c_void_p()
        check(lib.pseudo_create(_ptr(Tt), m, m, n, 0, _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.n = n
        self.m = m
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pseudo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n = ctypes.c_int64()
        f = ctypes.c_double()
        t = ctypes.c_double()
        check(self._lib.pseudo_info(self._h, ctypes.byref(n), ctypes.byref(f), ctypes.byref(t)))
        return {"n": n.value, "norm_fro": f.value, "norm2_est": t.value}

    def stats(self) -> dict:
        s = Stats()
        check(self._lib.pseudo_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def kernel_stats(self) -> dict:
        out = {}
        for i, name in enumerate(_abi.KCLASSES):
            k = _abi.KStat()
            check(self._lib.pseudo_kernel_stats(self._h, i, ctypes.byref(k)))
            out[name] = {"launches": k.launches, "ms": k.ms, "flops": k.flops, "bytes": k.bytes}
        return out

    def reset_stats(self):
        check(self._lib.pseudo_stats_reset(self._h))

    def set_wait_limit(self, ns: int):
        """Limit of the bounded waits of the tensor-core kernels (pseudo_set_wait_limit)."""
        check(self._lib.pseudo_set_wait_limit(self._h, ctypes.c_uint64(int(ns))))

    def workspace_bytes(self, npts: int, opts: Opts) -> int:
        b = ctypes.c_size_t()
        check(self._lib.pseudo_workspace_bytes(self._h, ctypes.byref(opts), int(npts), ctypes.byref(b)))
        return b.value

    def grid(self, z, eps_levels=(), opts: Opts | None = None, workspace=None, stream=None, out=None, **kw):
        """sigma_min(T - z I) for a 1-D complex128 CUDA tensor (or array) z.
        Returns dict of CUDA tensors: sigma, res, flags, member, plus 'status'.
        ``out``: a dict returned by an earlier call on as many points, whose
        tensors receive the results (with the same workspace, a repeated call
        then replays the library's cached loop graph)."""
        torch = _torch()
        o = Opts.from_buffer_copy(opts) if opts is not None else default_opts(**kw)
        o.io_host = 0  # the binding hands the library device tensors
        zt = torch.as_tensor(np.asarray(z, dtype=np.complex128)) if not torch.is_tensor(z) else z
        zt = zt.to(device="cuda", dtype=torch.complex128).contiguous()
        npts = zt.numel()
        if out is not None:
            sigma, res, flags, member = out["sigma"], out["res"], out["flags"], out["member"]
            assert all(t.numel() == npts and t.is_cuda for t in (sigma, res, flags, member))
            member.zero_()
        else:
            sigma = torch.empty(npts, dtype=torch.float64, device="cuda")
            res = torch.empty(npts, dtype=torch.float64, device="cuda")
            flags = torch.empty(npts, dtype=torch.int32, device="cuda")
            member = torch.zeros(npts, dtype=torch.int32, device="cuda")
        eps = np.ascontiguousarray(np.asarray(eps_levels, dtype=np.float64))
        need = self.workspace_bytes(npts, o)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        rc = check(self._lib.pseudo_grid(
            self._h, _ptr(zt), npts, eps.ctypes.data_as(ctypes.c_void_p) if eps.size else None, int(eps.size),
            ctypes.byref(o), _ptr(sigma), _ptr(res), _ptr(flags), _ptr(member), _ptr(workspace),
            workspace.numel(), _stream_ptr(stream)))
        return {"sigma": sigma, "res": res, "flags": flags, "member": member, "status": rc}

    def grid_host(self, z: np.ndarray, eps_levels=(), opts: Opts | None = None, workspace=None, stream=None,
                  out=None, **kw):
        """Same as grid() but z and the outputs are (pinned) host arrays: the
        library copies them to and from the device inside the call."""
        torch = _torch()
        o = Opts.from_buffer_copy(opts) if opts is not None else default_opts(**kw)
        o.io_host = 1  # a copy: the caller's options are left as they were
        z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
        npts = z.size
        if out is None:
            out = {
                "sigma": np.empty(npts, np.float64), "res": np.empty(npts, np.float64),
                "flags": np.empty(npts, np.int32), "member": np.empty(npts, np.uint32),
            }
        eps = np.ascontiguousarray(np.asarray(eps_levels, dtype=np.float64))
        need = self.workspace_bytes(npts, o)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        rc = check(self._lib.pseudo_grid(
            self._h, vp(z), npts, vp(eps) if eps.size else None, int(eps.size), ctypes.byref(o),
            vp(out["sigma"]), vp(out["res"]), vp(out["flags"]), vp(out["member"]), _ptr(workspace),
            workspace.numel(), _stream_ptr(stream)))
        out["status"] = rc
        return out

    def recycle_state(self, npts: int, opts: Opts, workspace):
        """After a recycle-mode grid() call with this workspace: the lanes'
        recycled subspaces as numpy arrays, one dict per lane with V, W1, W3,
        W4 (n x k), H1, H2, L (k x k) and p."""
        torch = _torch()
        out = (ctypes.c_int64 * 11)()
        check(self._lib.pseudo_recycle_state_layout(self._h, ctypes.byref(opts), int(npts), out))
        lanes, km, ld = out[0], out[1], out[2]
        ws = workspace.cpu().numpy()
        n = self.n

        def mat(off, rows, cols, ldm):
            a = ws[off:off + rows * ldm * 16].view(np.complex128).reshape(rows, ldm)
            return a[:, :cols]

        p_all = ws[out[10]:out[10] + 4 * lanes].view(np.int32)
        res = []
        for l in range(lanes):
            k = int(p_all[l]) * opts.r
            d = {"p": int(p_all[l])}
            for name, oi in (("V", 3), ("W1", 4), ("W3", 5), ("W4", 6)):
                d[name] = mat(out[oi], n, ld, ld)[:, l * km:l * km + k].copy()
            for name, oi in (("H1", 7), ("H2", 8), ("L", 9)):
                base = out[oi] + l * km * km * 16
                d[name] = ws[base:base + km * km * 16].view(np.complex128).reshape(km, km)[:k, :k].copy()
            res.append(d)
        del torch
        return res

    def solve(self, X, z, adjoint: bool = False, precision: int = FP64, stream=None):
        """In-place multi-shift triangular solve on a row-major (n, ncols)
        complex128 CUDA tensor X, column c shifted by z[c]."""
        torch = _torch()
        assert X.is_cuda and X.dtype == torch.complex128 and X.is_contiguous() and X.shape[0] == self.n
        ncols = X.shape[1]
        zt = torch.as_tensor(z).to(device="cuda", dtype=torch.complex128).contiguous()
        b = ctypes.c_size_t()
        check(self._lib.pseudo_solve_workspace_bytes(self._h, ncols, ctypes.byref(b)))
        ws = torch.empty(b.value, dtype=torch.uint8, device="cuda")
        check(self._lib.pseudo_solve(self._h, _ptr(X), _ptr(zt), ncols, int(adjoint), int(precision), _ptr(ws),
                                     b.value, _stream_ptr(stream)))
        return X

    def matvec(self, X, z=None, B=None, adjoint: bool = False, precision: int = FP64, stream=None):
        """Y = (T - zI)^{op} X, or B - (T - zI)^{op} X when B is given; FP64,
        double-single accurate on the tensor cores (precision=MIXED) or on the
        CUDA cores (precision=MIXED_CUDACORE)."""
        torch = _torch()
        ncols = X.shape[1]
        Y = torch.empty_like(X)
        zt = None if z is None else torch.as_tensor(z).to(device="cuda", dtype=torch.complex128).contiguous()
        b = ctypes.c_size_t()
        check(self._lib.pseudo_matvec_workspace_bytes(self._h, ncols, ctypes.byref(b)))
        ws = torch.empty(b.value, dtype=torch.uint8, device="cuda")
        check(self._lib.pseudo_matvec(self._h, _ptr(X), _ptr(B), _ptr(Y), _ptr(zt), ncols, int(adjoint),
                                      int(B is not None), int(precision), _ptr(ws), b.value, _stream_ptr(stream)))
        return Y


def grid_batch(handles, zs, eps_levels=(), opts: Opts | None = None, workspace=None, stream=None, out=None, **kw):
    """sigma_min for many matrices at once: handles[m] (distinct Pseudo
    objects) on the complex128 grid zs[m].  The matrices run concurrently on
    the device.  Returns (list of per-matrix dicts as Pseudo.grid, status).
    ``out``: the list an earlier call returned, whose tensors receive the
    results (as in Pseudo.grid)."""
    torch = _torch()
    lib = _abi.load()
    o = Opts.from_buffer_copy(opts) if opts is not None else default_opts(**kw)
    o.io_host = 0  # the binding hands the library device tensors
    nmat = len(handles)
    if nmat != len(zs) or nmat < 1:
        raise ValueError("need one grid per handle")
    zt = [(z if torch.is_tensor(z) else torch.as_tensor(np.asarray(z, dtype=np.complex128)))
          .to(device="cuda", dtype=torch.complex128).contiguous() for z in zs]
    if out is not None:
        outs = out
        assert len(outs) == nmat and all(o_["sigma"].numel() == z.numel() for o_, z in zip(outs, zt))
        for o_ in outs:
            o_["member"].zero_()
    else:
        outs = []
        for z in zt:
            k = z.numel()
            outs.append({"sigma": torch.empty(k, dtype=torch.float64, device="cuda"),
                         "res": torch.empty(k, dtype=torch.float64, device="cuda"),
                         "flags": torch.empty(k, dtype=torch.int32, device="cuda"),
                         "member": torch.zeros(k, dtype=torch.int32, device="cuda")})
    hs = (ctypes.c_void_p * nmat)(*[h._h.value for h in handles])
    npts = (ctypes.c_int64 * nmat)(*[z.numel() for z in zt])

    def ptrs(key):
        return (ctypes.c_void_p * nmat)(*[o_[key].data_ptr() for o_ in outs])

    zp = (ctypes.c_void_p * nmat)(*[z.data_ptr() for z in zt])
    eps = np.ascontiguousarray(np.asarray(eps_levels, dtype=np.float64))
    need = ctypes.c_size_t()
    check(lib.pseudo_grid_batch_workspace_bytes(hs, nmat, npts, ctypes.byref(o), ctypes.byref(need)))
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    rc = check(lib.pseudo_grid_batch(
        hs, nmat, zp, npts, eps.ctypes.data_as(ctypes.c_void_p) if eps.size else None, int(eps.size),
        ctypes.byref(o), ptrs("sigma"), ptrs("res"), ptrs("flags"), ptrs("member"), _ptr(workspace),
        workspace.numel(), _stream_ptr(stream)))
    return outs, rc


def grid_batch_workspace_bytes(handles, npts, opts: Opts) -> int:
    """Device workspace bytes grid_batch needs (pseudo_grid_batch_workspace_bytes)."""
    nmat = len(handles)
    hs = (ctypes.c_void_p * nmat)(*[h._h.value for h in handles])
    np_ = (ctypes.c_int64 * nmat)(*[int(k) for k in npts])
    o = Opts.from_buffer_copy(opts)
    o.io_host = 0
    need = ctypes.c_size_t()
    check(_abi.load().pseudo_grid_batch_workspace_bytes(hs, nmat, np_, ctypes.byref(o), ctypes.byref(need)))
    return need.value


def tuned_config(n: int) -> dict:
    """The library's tuned choices for order n (pseudo_tuned_config): the FP32
    solver kernel of fp32_solver = SOLVER_AUTO and the Lanczos slots of
    shift_batch = 0."""
    s, k = ctypes.c_int(), ctypes.c_int()
    check(_abi.load().pseudo_tuned_config(int(n), ctypes.byref(s), ctypes.byref(k)))
    return {"fp32_solver": s.value, "slots": k.value}


def traversal_order(grid_nx: int, grid_ny: int, batch_b: int = 20, traversal: int = TRAVERSE_BATCH_ZIGZAG,
                    npts: int | None = None) -> np.ndarray:
    """Point indices in the order the recycling path visits a grid_nx x
    grid_ny grid (z[iy * grid_nx + ix]): the batch-zigzag traversal of Sec.
    2.3 with column batches of batch_b points, or the Hilbert / Morton order
    of Sec. 5 (pseudo_traversal_order)."""
    n = grid_nx * grid_ny if npts is None else int(npts)
    out = np.empty(n, dtype=np.int32)
    check(_abi.load().pseudo_traversal_order(ctypes.c_int64(n), grid_nx, grid_ny, batch_b, traversal,
                                             out.ctypes.data_as(ctypes.c_void_p)))
    return out
