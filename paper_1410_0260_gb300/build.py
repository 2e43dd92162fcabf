"""Build libaskit.so in-tree for sm_103a (nvcc, translation units in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libaskit.so")

SOURCES = ["capi.cu", "setup_sort.cu", "setup_tree.cu", "setup_skel.cu", "eval_lists.cu",
           "weights.cu", "eval_simt.cu", "eval_tc.cu", "eval_tc_wide.cu", "eval_tc16.cu", "eval_g16.cu", "prune_stats.cu"]
# setup stages are bit-exact FP64: no contraction into fused multiply-adds anywhere
NO_FMAD = {"setup_tree.cu", "setup_skel.cu", "prune_stats.cu"}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(src: str) -> list[str]:
    f = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if src in NO_FMAD:
        f += ["-fmad=false"]
    return f


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    # every header of csrc/ (askit_impl.cuh, tc_ptx.cuh, ...) and the public header
    deps = [src, os.path.join(ROOT, "include", "askit.h"), __file__]
    deps += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()

    def compile_one(name: str) -> str:
        src = os.path.join(CSRC, name)
        obj = os.path.join(OUT, name.replace(".cu", ".o"))
        if _stale(obj, src):
            cmd = [cc, *_flags(name), "-c", src, "-o", obj + ".tmp"]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {name}:\n{r.stderr}")
            os.replace(obj + ".tmp", obj)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [cc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs,
               "-cudart", "shared", "-lcuda"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
