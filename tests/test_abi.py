"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function include/pseudo.h declares (no compute calls here)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    txt = (ROOT / "include" / "pseudo.h").read_text()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pseudo_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_all_declared_symbols():
    from paper_2606_26785_b300 import _abi

    lib = _abi.load()
    names = _declared()
    assert "pseudo_grid" in names and "pseudo_create" in names
    missing = [nm for nm in names if not hasattr(lib, nm)]
    assert not missing, missing
    assert set(_abi.EXPORTED) <= set(names)


def test_struct_layout_matches_header(tmp_path):
    import subprocess

    from paper_2606_26785_b300 import _abi

    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pseudo.h"\nint main(){printf("%zu %zu %zu %zu",'
                   'sizeof(pseudo_opts),sizeof(pseudo_stats_t),offsetof(pseudo_opts,profile),offsetof(pseudo_stats_t,ms_total));}')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()
    assert [int(v) for v in out] == [ctypes.sizeof(_abi.Opts), ctypes.sizeof(_abi.Stats), _abi.Opts.profile.offset,
                                     _abi.Stats.ms_total.offset]


def test_defaults_are_the_papers_parameters():
    import paper_2606_26785_b300 as p

    o = p.default_opts()
    assert (o.r, o.p_max, o.batch_b) == (6, 60, 20)
    assert (o.eta, o.tau, o.omega, o.eps_shift_rel) == (1e-4, 1e-10, 1.6, 1e-14)


def test_errors_without_handle():
    from paper_2606_26785_b300 import _abi

    lib = _abi.load()
    assert lib.pseudo_info(None, None, None, None) == _abi.ERR_ARG
    assert b"NULL" in lib.pseudo_last_error()
    lib.pseudo_destroy(None)  # NULL-safe


def test_argument_errors_are_reported_before_any_device_work():
    """Every entry point validates its host-side arguments first: these calls
    return their documented error codes on a machine without a GPU."""
    from paper_2606_26785_b300 import _abi

    lib = _abi.load()
    vp, c64 = ctypes.c_void_p, ctypes.c_int64
    buf = (ctypes.c_double * 8)()
    h = vp()
    # pseudo_create: NULL out, NULL T, rows neither n nor 2n, n out of range,
    # ldT < m (square and stacked pencil)
    assert lib.pseudo_create(buf, c64(2), c64(2), c64(2), 1, None, None) == _abi.ERR_ARG
    assert lib.pseudo_create(None, c64(2), c64(2), c64(2), 1, None, ctypes.byref(h)) == _abi.ERR_ARG
    for m in (1, 3, 5, 8):
        assert lib.pseudo_create(buf, c64(8), c64(m), c64(2), 1, None, ctypes.byref(h)) == _abi.ERR_UNSUPPORTED
        assert b"pencil" in lib.pseudo_last_error()
    assert lib.pseudo_create(buf, c64(0), c64(0), c64(0), 1, None, ctypes.byref(h)) == _abi.ERR_ARG
    assert lib.pseudo_create(buf, c64(1), c64(2), c64(2), 1, None, ctypes.byref(h)) == _abi.ERR_ARG
    assert lib.pseudo_create(buf, c64(3), c64(4), c64(2), 1, None, ctypes.byref(h)) == _abi.ERR_ARG
    assert h.value is None
    o = _abi.Opts()
    assert lib.pseudo_opts_default(None) == _abi.ERR_ARG
    assert lib.pseudo_opts_default(ctypes.byref(o)) == 0
    size = ctypes.c_size_t()
    assert lib.pseudo_workspace_bytes(None, ctypes.byref(o), c64(4), ctypes.byref(size)) == _abi.ERR_ARG
    assert lib.pseudo_grid(None, buf, c64(4), None, 0, ctypes.byref(o), buf, None, None, None, buf,
                           ctypes.c_size_t(64), None) == _abi.ERR_ARG
    n1 = (ctypes.c_int64 * 1)(4)
    assert lib.pseudo_grid_batch_workspace_bytes(None, 1, n1, ctypes.byref(o), ctypes.byref(size)) == _abi.ERR_ARG
    assert lib.pseudo_grid_batch(None, 0, None, n1, None, 0, ctypes.byref(o), None, None, None, None, None,
                                 ctypes.c_size_t(0), None) == _abi.ERR_ARG
    assert lib.pseudo_solve(None, buf, buf, c64(1), 0, 0, buf, ctypes.c_size_t(64), None) == _abi.ERR_ARG
    assert lib.pseudo_matvec(None, buf, None, buf, buf, c64(1), 0, 0, 0, buf, ctypes.c_size_t(64),
                             None) == _abi.ERR_ARG
    assert lib.pseudo_stats(None, None) == _abi.ERR_ARG
    assert lib.pseudo_set_wait_limit(None, ctypes.c_uint64(0)) == _abi.ERR_ARG
    assert lib.pseudo_solve_noalloc(None, buf, buf, c64(1), 0, None) == _abi.ERR_ARG
    assert lib.pseudo_tuned_config(c64(0), None, None) == _abi.ERR_ARG


def test_misaligned_device_arrays_are_refused():
    """Device arrays are read with their natural vector widths, so a
    misaligned pointer would fault on the device: the host refuses it first
    (complex arrays 16 bytes, sigma/res 8, flags/member 4), before looking at
    the handle.  Host arrays (io_host = 1) are only copied and need no such
    alignment."""
    from paper_2606_26785_b300 import _abi

    lib = _abi.load()
    raw = (ctypes.c_char * 256)()
    a = ctypes.addressof(raw)
    assert a % 8 == 0
    good = a if a % 16 == 0 else a + 8
    odd = good + 8
    vp, c64 = ctypes.c_void_p, ctypes.c_int64
    assert lib.pseudo_solve(None, vp(odd), vp(good), c64(1), 0, 0, vp(good), ctypes.c_size_t(64), None) == _abi.ERR_ARG
    assert b"aligned" in lib.pseudo_last_error()
    assert lib.pseudo_solve(None, vp(good), vp(odd), c64(1), 0, 0, vp(good), ctypes.c_size_t(64), None) == _abi.ERR_ARG
    assert b"aligned" in lib.pseudo_last_error()
    assert lib.pseudo_matvec(None, vp(good), None, vp(odd), None, c64(1), 0, 0, 0, None, ctypes.c_size_t(0),
                             None) == _abi.ERR_ARG
    assert b"aligned" in lib.pseudo_last_error()
    assert lib.pseudo_solve_noalloc(None, vp(odd), vp(good), c64(1), 0, None) == _abi.ERR_ARG
    assert b"aligned" in lib.pseudo_last_error()
    o = _abi.Opts()
    assert lib.pseudo_opts_default(ctypes.byref(o)) == 0
    for z, sig, flags in ((odd, good, None), (good, good + 4, None), (good, good, good + 2)):
        assert lib.pseudo_grid(None, vp(z), c64(4), None, 0, ctypes.byref(o), vp(sig), None, vp(flags), None,
                               vp(good), ctypes.c_size_t(64), None) == _abi.ERR_ARG
        assert b"aligned" in lib.pseudo_last_error()
    # aligned arrays get as far as the handle check
    assert lib.pseudo_grid(None, vp(good), c64(4), None, 0, ctypes.byref(o), vp(good), None, None, None,
                           vp(good), ctypes.c_size_t(64), None) == _abi.ERR_ARG
    assert b"handle" in lib.pseudo_last_error()
    # host arrays are not checked for alignment
    o.io_host = 1
    assert lib.pseudo_grid(None, vp(odd), c64(4), None, 0, ctypes.byref(o), vp(odd), None, None, None,
                           vp(good), ctypes.c_size_t(64), None) == _abi.ERR_ARG
    assert b"handle" in lib.pseudo_last_error()


def test_tuned_table_covers_every_order():
    """The tuned table (pseudo_tuned_config, host-only) gives a valid solver
    kernel and a positive slot count for every order, piecewise constant over
    buckets, and the default options ask for it."""
    import paper_2606_26785_b300 as p
    from paper_2606_26785_b300 import _abi

    assert p.default_opts().fp32_solver == _abi.SOLVER_AUTO
    prev = None
    changes = 0
    for n in list(range(1, 4100, 7)) + [8000, 16000, 1 << 20]:
        c = p.tuned_config(n)
        assert c["fp32_solver"] in (0, 1, 3, 4) and c["slots"] >= 1
        changes += prev is not None and c != prev
        prev = c
    assert changes <= 16


def test_last_error_is_per_thread():
    import threading

    from paper_2606_26785_b300 import _abi

    lib = _abi.load()
    assert lib.pseudo_info(None, None, None, None) == _abi.ERR_ARG
    mine = lib.pseudo_last_error()
    seen = {}

    def other():
        buf = (ctypes.c_double * 8)()
        h = ctypes.c_void_p()
        seen["rc"] = lib.pseudo_create(buf, ctypes.c_int64(4), ctypes.c_int64(3), ctypes.c_int64(2), 1, None,
                                       ctypes.byref(h))
        seen["msg"] = lib.pseudo_last_error()

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["rc"] == _abi.ERR_UNSUPPORTED and b"pencil" in seen["msg"]
    assert lib.pseudo_last_error() == mine and b"NULL" in mine
