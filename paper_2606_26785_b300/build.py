"""Build the CUDA library libpseudo_b300.so for sm_103a (in-tree).

    python -m paper_2606_26785_b300.build
    python -m paper_2606_26785_b300.build --define TC_WIDE_MIN_NPAD=0 --out /tmp/wide/libpseudo_b300.so

``--define`` passes compile-time tuning constants of the kernels (for example
``TC_WIDE_MIN_NPAD``, the padded order from which the tensor-core solve runs
32 columns per CTA); such builds go to ``--out`` for side-by-side timing
(``probe/solve_sweep.py --lib``) and never replace the in-tree library.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIB = PKG / "libpseudo_b300.so"
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = list(CSRC.glob("*")) + [ROOT / "include" / "pseudo.h"]
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose: bool = False, defines=(), out: Path | None = None) -> Path:
    lib = LIB if out is None else Path(out).resolve()
    if lib == LIB and defines:
        raise ValueError("builds with --define go to their own --out path")
    if lib == LIB and not force and not _stale():
        return LIB
    objdir = PKG / "_build" if lib == LIB else lib.parent / "_build"
    objdir.mkdir(parents=True, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(ROOT / "include"),
                    "--expt-relaxed-constexpr"] + ["-D" + d for d in defines]
    if verbose:
        flags += ["-Xptxas", "-v"]
    objs = []
    procs = []
    for src in sources():
        obj = objdir / (src.stem + ".o")
        objs.append(obj)
        cmd = [NVCC, "-c", str(src), "-o", str(obj)] + flags
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed = True
    if failed:
        raise RuntimeError("nvcc failed")
    tmp = lib.with_suffix(".so.tmp")
    subprocess.run([NVCC, "-shared", *ARCH, "-o", str(tmp), *map(str, objs), "-lcudart"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", dest="verbose", action="store_true")
    ap.add_argument("--define", action="append", default=[], help="NAME=VALUE, a compile-time tuning constant")
    ap.add_argument("--out", type=Path, default=None, help="library path of a build with --define")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose, defines=a.define, out=a.out))
