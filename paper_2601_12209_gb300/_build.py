"""In-tree build of libgbfft.so (CUDA, sm_103a only).

Each translation unit under csrc/ is compiled by nvcc in parallel, then the
objects are linked into ``paper_2601_12209_gb300/lib/libgbfft.so``. An object
is rebuilt when its source or any header is newer than it.
"""
from __future__ import annotations

import glob
import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "gbfft-" + platform.machine())
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libgbfft.so")
STAMP = os.path.join(LIBDIR, "libgbfft.machine")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbfft")


def _headers() -> list[str]:
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link libgbfft.so if anything changed; return its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    newest_header = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    todo = []
    objs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if (not os.path.exists(obj) or os.path.getmtime(obj) < os.path.getmtime(src)
                or os.path.getmtime(obj) < newest_header):
            todo.append((src, obj))

    def compile_one(pair):
        src, obj = pair
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc] + NVCC_FLAGS + ["-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, obj)
        if verbose:
            print(f"[gbfft build] compiled {os.path.basename(src)}", file=sys.stderr)

    if todo:
        workers = jobs or max(1, min(len(todo), os.cpu_count() or 1))
        # largest units first so the long poles start early
        todo.sort(key=lambda p: -os.path.getsize(p[0]))
        with ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(compile_one, todo))
    stale_machine = not os.path.exists(STAMP) or open(STAMP).read().strip() != platform.machine()
    if todo or stale_machine or not os.path.exists(LIB) or \
            os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libgbfft.so failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(STAMP, "w") as fh:
            fh.write(platform.machine())
        if verbose:
            print(f"[gbfft build] linked {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
