"""Build libkchol.so (sm_103a) in-tree with nvcc: one object per .cu file,
compiled in parallel, then linked into a shared library with a static CUDA
runtime.  Output: paper_1706_02205_gb300/_lib/libkchol.so."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
SO = os.path.join(OUT, "libkchol.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(SRC, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(SRC, "*.cuh"))) + [os.path.join(HERE, "..", "include", "kchol.h")]
    objs = [os.path.join(OUT, os.path.basename(s)[:-3] + ".o") for s in srcs]
    cc = nvcc()
    flags = ARCH + FLAGS + (extra or [])

    def one(pair):
        src, obj = pair
        if not force and not _stale(obj, [src] + hdrs):
            return obj, ""
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [cc] + flags + ["-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        os.replace(tmp, obj)
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        for obj, err in ex.map(one, zip(srcs, objs)):
            if verbose and err:
                print(err, file=sys.stderr)
    if force or _stale(SO, objs):
        tmp = SO + f".tmp{os.getpid()}"
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
