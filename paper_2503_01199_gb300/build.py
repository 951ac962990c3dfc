"""Compile the CUDA sources of csrc/ into the in-tree shared libraries
paper_2503_01199_gb300/_build/liblgs.so (release) and
paper_2503_01199_gb300/_build/debug/liblgs_debug.so (the same sources with
-DLGS_DEBUG: the kernels' bounds checks, see lgs_get_debug_error), sm_103a
only.

Each translation unit is compiled by its own nvcc process in parallel and
the objects are linked with nvcc -shared. A rebuild happens only when a
source or header is newer than the library.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
SRC = PKG / "csrc"
INC = PKG.parent / "include"
OUT_DIR = PKG / "_build"
LIB = OUT_DIR / "liblgs.so"
DEBUG_DIR = OUT_DIR / "debug"
DEBUG_LIB = DEBUG_DIR / "liblgs_debug.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + str(INC), "-I" + str(SRC)]


def sources() -> list[Path]:
    return sorted(SRC.glob("*.cu"))


def _deps() -> list[Path]:
    return sources() + sorted(SRC.glob("*.cuh")) + sorted(INC.glob("*.h"))


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe is None:
        cand = Path(os.environ.get("CUDA_HOME", "/usr/local/cuda")) / "bin" / "nvcc"
        if cand.exists():
            exe = str(cand)
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblgs")
    return exe


def up_to_date(lib: Path = LIB) -> bool:
    machine = lib.parent / "machine.txt"
    if not lib.exists() or not machine.exists():
        return False
    if machine.read_text().strip() != platform.machine():
        return False
    t = lib.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _deps())


def _build_one(lib: Path, extra: list[str], verbose: bool, pool: ThreadPoolExecutor) -> Path:
    out = lib.parent
    out.mkdir(parents=True, exist_ok=True)
    cc = nvcc()

    def one(src: Path) -> Path:
        obj = out / (src.stem + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    objs = list(pool.map(one, sources()))
    tmp = lib.with_suffix(f".{os.getpid()}.tmp")
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {lib.name} failed:\n" + r.stderr)
    os.replace(tmp, lib)
    (out / "machine.txt").write_text(platform.machine())
    return lib


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> Path:
    """Builds the release library (and, with debug, the bounds-checked one);
    returns the release library's path."""
    todo = [(LIB, [])]
    if debug:
        todo.append((DEBUG_LIB, ["-DLGS_DEBUG"]))
    todo = [(lib, extra) for lib, extra in todo if force or not up_to_date(lib)]
    if todo:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as pool:
            list(ThreadPoolExecutor(max_workers=len(todo)).map(
                lambda t: _build_one(t[0], t[1], verbose, pool), todo))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
