"""ctypes view of the C ABI in include/pseudo.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
from pathlib import Path

_LIB = Path(__file__).resolve().parent / "libpseudo_b300.so"

OK = 0
WARN_NOT_CONVERGED = 1
ERR_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_WORKSPACE, ERR_NONFINITE, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6
INVLANC, RECYCLE = 0, 1
FP64, MIXED, MIXED_CUDACORE, DOUBLE_SINGLE = 0, 1, 2, 3
TRAVERSE_BATCH_ZIGZAG, TRAVERSE_HILBERT, TRAVERSE_MORTON = 0, 1, 2
SOLVER_TENSOR_CORES, SOLVER_CUDA_CORES, SOLVER_AUTO, SOLVER_TC16, SOLVER_TC32 = 0, 1, 2, 3, 4
PT_ACCEPTED, PT_REFINED, PT_NOT_CONVERGED, PT_IR_FALLBACK, PT_SINGULAR = 1, 2, 4, 8, 16

EXPORTED = (
    "pseudo_opts_default", "pseudo_create", "pseudo_workspace_bytes", "pseudo_grid", "pseudo_stats",
    "pseudo_stats_reset", "pseudo_info", "pseudo_destroy", "pseudo_last_error", "pseudo_solve_workspace_bytes",
    "pseudo_solve", "pseudo_matvec", "pseudo_kernel_stats", "pseudo_launch_count", "pseudo_recycle_state_layout",
    "pseudo_grid_batch_workspace_bytes", "pseudo_grid_batch", "pseudo_matvec_workspace_bytes",
    "pseudo_traversal_order", "pseudo_set_wait_limit", "pseudo_solve_noalloc", "pseudo_tuned_config",
)


class Opts(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int), ("precision", ctypes.c_int), ("r", ctypes.c_int), ("p_max", ctypes.c_int),
        ("grid_nx", ctypes.c_int), ("grid_ny", ctypes.c_int), ("batch_b", ctypes.c_int), ("lanes", ctypes.c_int),
        ("shift_batch", ctypes.c_int), ("eps_shift_rel", ctypes.c_double), ("tau", ctypes.c_double),
        ("omega", ctypes.c_double), ("eta", ctypes.c_double), ("rtol", ctypes.c_double),
        ("maxiter_lanczos", ctypes.c_int), ("maxiter_lobpcg", ctypes.c_int), ("max_ir", ctypes.c_int),
        ("io_host", ctypes.c_int), ("seed", ctypes.c_uint64), ("profile", ctypes.c_int), ("fp32_solver", ctypes.c_int),
        ("traversal", ctypes.c_int), ("device_loop", ctypes.c_int),
    ]


class KStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


KCLASSES = ("trsv32", "trsv64", "trmv64", "trmv_ds", "recysing", "lanczos", "trsv_ds", "rect_qr")


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "sv_R", "mv_M", "mv_M_fp64_refine", "n_points", "n_accepted", "n_refined", "n_not_converged",
        "n_updates", "lanczos_steps", "lobpcg_iters", "n_fallback")] + [(k, ctypes.c_double) for k in (
        "ms_recysing", "ms_refine", "ms_update", "ms_polish", "ms_total")] + [("n_singular", ctypes.c_int64), ("n_rtilde_capped", ctypes.c_int64),
                                                       ("n_graph_launches", ctypes.c_int64),
                                                       ("n_graph_builds", ctypes.c_int64),
                                                       ("ms_graph_build", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib_path() -> Path:
    return _LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library; raises if it cannot be built or loaded (there is
    no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build
        _build.build()
    if not _LIB.exists():
        raise RuntimeError(f"CUDA library {_LIB} is missing; run python -m paper_2606_26785_b300.build")
    lib = ctypes.CDLL(str(_LIB))
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    po = ctypes.POINTER(Opts)
    lib.pseudo_opts_default.argtypes = [po]
    lib.pseudo_create.argtypes = [vp, i64, i64, i64, ci, vp, ctypes.POINTER(vp)]
    lib.pseudo_workspace_bytes.argtypes = [vp, po, i64, ctypes.POINTER(ctypes.c_size_t)]
    lib.pseudo_grid.argtypes = [vp, vp, i64, vp, ci, po, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.pseudo_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.pseudo_stats_reset.argtypes = [vp]
    lib.pseudo_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(cd), ctypes.POINTER(cd)]
    lib.pseudo_destroy.argtypes = [vp]
    lib.pseudo_destroy.restype = None
    lib.pseudo_last_error.restype = ctypes.c_char_p
    lib.pseudo_solve_workspace_bytes.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_size_t)]
    lib.pseudo_solve.argtypes = [vp, vp, vp, i64, ci, ci, vp, ctypes.c_size_t, vp]
    lib.pseudo_recycle_state_layout.argtypes = [vp, po, i64, ctypes.POINTER(i64)]
    lib.pseudo_launch_count.argtypes = []
    lib.pseudo_launch_count.restype = ctypes.c_int64
    lib.pseudo_kernel_stats.argtypes = [vp, ci, ctypes.POINTER(KStat)]
    lib.pseudo_matvec.argtypes = [vp, vp, vp, vp, vp, i64, ci, ci, ci, vp, ctypes.c_size_t, vp]
    lib.pseudo_matvec_workspace_bytes.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_size_t)]
    lib.pseudo_grid_batch_workspace_bytes.argtypes = [vp, ci, vp, po, ctypes.POINTER(ctypes.c_size_t)]
    lib.pseudo_grid_batch.argtypes = [vp, ci, vp, vp, vp, ci, po, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.pseudo_set_wait_limit.argtypes = [vp, ctypes.c_uint64]
    lib.pseudo_tuned_config.argtypes = [i64, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.pseudo_solve_noalloc.argtypes = [vp, vp, vp, i64, ci, vp]
    for name in EXPORTED:
        fn = getattr(lib, name)
        if name not in ("pseudo_destroy", "pseudo_last_error", "pseudo_launch_count"):
            fn.restype = ctypes.c_int
    _lib = lib
    return lib


class PseudoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pseudo error {code}: {msg}")
        self.code = code


def check(rc: int) -> int:
    if rc < 0:
        raise PseudoError(rc, load().pseudo_last_error().decode())
    return rc
