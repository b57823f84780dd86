"""Builds libmpkrylov.so (sm_103a) in-tree with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked into
one shared library against the shared CUDA runtime (so the process has a
single runtime shared with PyTorch).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmpkrylov.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def cuda_lib_dir() -> str:
    base = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        p = os.path.join(base, sub)
        if os.path.isdir(p):
            return p
    return os.path.join(base, "lib64")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_mtime():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(INCLUDE, "mpkrylov.h"))
    return max(os.path.getmtime(h) for h in hs)


# Translation units compiled once per word count W = p/32 (-DMPK_W=W) and
# once for their host entry points (-DMPK_W=0), in parallel.
SPLIT = {"solvers.cu", "batch.cu"}
WORDS = (0, 4, 8, 16, 32)


def units():
    out = []
    for s in sources():
        out += [(s, w) for w in WORDS] if s in SPLIT else [(s, None)]
    return out


def _compile(unit, verbose_ptxas: bool) -> str:
    src, w = unit
    obj = os.path.join(BUILD, src.replace(".cu", ".o" if w is None else f"_w{w}.o"))
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, "-c",
           os.path.join(CSRC, src), "-o", obj]
    if w is not None:
        cmd.insert(1, f"-DMPK_W={w}")
    if verbose_ptxas:
        cmd[1:1] = ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} (MPK_W={w}):\n{r.stderr[-6000:]}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    newest = max([_headers_mtime()] + [os.path.getmtime(os.path.join(CSRC, s)) for s in srcs])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    todo = units()
    # the longest units first: the W = 32 builds dominate
    todo.sort(key=lambda u: -(u[1] if u[1] is not None else 6))
    jobs = jobs or min(len(todo), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda u: _compile(u, verbose_ptxas), todo))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "--cudart", "shared", *objs, "-o", tmp,
           "-Xlinker", f"-rpath,{cuda_lib_dir()}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time

    t = time.time()
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv), f"{time.time() - t:.1f}s")
