"""Compile the CUDA sources of csrc/ into the in-tree shared library
paper_2503_01199_gb300/_build/liblgs.so (sm_103a only).

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


MACHINE = OUT_DIR / "machine.txt"


def up_to_date() -> bool:
    if not LIB.exists() or not MACHINE.exists():
        return False
    if MACHINE.read_text().strip() != platform.machine():
        return False
    t = LIB.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and up_to_date():
        return LIB
    OUT_DIR.mkdir(exist_ok=True)
    cc = nvcc()
    objs = []

    def one(src: Path) -> Path:
        obj = OUT_DIR / (src.stem + ".o")
        cmd = [cc, *ARCH, *FLAGS, "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(one, sources()))
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link of liblgs.so failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    MACHINE.write_text(platform.machine())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
