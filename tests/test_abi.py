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
