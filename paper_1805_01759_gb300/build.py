"""Build libbpdn.so (the CUDA kernels and the C ABI of include/bpdn.h) for sm_103a.

The library is compiled in-tree into ``paper_1805_01759_gb300/_build/`` with nvcc:
one object per translation unit (compiled in parallel), then a shared link with the
static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbpdn.so")
SOURCES = ["api.cu", "operator.cu", "rbpg.cu", "refit.cu", "backward.cu", "ragged.cu", "noalloc.cu", "select.cu", "rbpg_block.cu", "peaks.cu", "preclass.cu", "rbpg_px.cu", "rbpg_split.cu"]
HEADERS = ["bpdn_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
# The refit's FP32 phase only finds the support that its FP64 phase then finishes and
# checks, so it takes the approximate FP32 divide and square root (these flags change
# no FP64 operation).
FILE_FLAGS = {"refit.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbpdn")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libbpdn.so."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    header_deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", h)
                                                                  for h in ("bpdn.h", "bpdn_bench.h")]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + header_deps):
            jobs.append([nvcc, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), "-I", os.path.join(ROOT, "include"),
                         "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
