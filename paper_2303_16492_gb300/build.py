"""Build the CUDA library libtrsgd.so in-tree (sm_103a only).

Each translation unit under csrc/ is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and linked into
``_lib/libtrsgd.so`` against the shared CUDA runtime (the one PyTorch loads).
``debug=True`` builds the same sources with ``-DTRSGD_DEBUG`` (index checks
that report ``TRSGD_EBADINDEX``) into ``_lib/libtrsgd_debug.so``; the library
loader picks it when the environment sets ``TRSGD_DEBUG=1``.
Usage: ``python -m paper_2303_16492_gb300.build [--force] [--debug]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libtrsgd.so")
DEBUG_OUT = os.path.join(OUT, "debug")
DEBUG_LIB = os.path.join(OUT, "libtrsgd_debug.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtrsgd")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "trsgd.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra, out: str = OUT) -> str:
    obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile every .cu under csrc/ and link libtrsgd.so (or, debug,
    libtrsgd_debug.so); returns its path."""
    lib, out = (DEBUG_LIB, DEBUG_OUT) if debug else (LIB, OUT)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    extra = list(extra) + (["-Xptxas", "-v"] if verbose else []) + (["-DTRSGD_DEBUG"] if debug else [])
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, out), srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
