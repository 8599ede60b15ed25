"""In-tree build of libfa.so for sm_103a (nvcc, one translation unit per
.cu file, compiled in parallel, linked against the shared CUDA runtime).

    python -m paper_2404_01249_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libfa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# ptxas reports register use (-v) and any double-precision instruction in a
# kernel (none may run on the GPU: tests/test_abi.py checks the log)
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-Xptxas", "-v",
                     "-Xptxas", "--warn-on-double-precision-use", "-I", INCLUDE, "-I", CSRC]
_lock = threading.Lock()


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(src: str) -> tuple[str, str]:
    obj = os.path.join(OUT, "obj", os.path.basename(src) + ".o")
    cmd = [_nvcc()] + NVCC_FLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, jobs: int | None = None) -> str:
    """Compile every kernel source and link libfa.so; returns its path."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
        srcs = sources()
        jobs = jobs or min(len(srcs), os.cpu_count() or 4)
        logs = []
        with cf.ThreadPoolExecutor(jobs) as ex:
            objs = []
            for obj, log in ex.map(_compile, srcs):
                objs.append(obj)
                logs.append(log)
        with open(os.path.join(OUT, "ptxas.log"), "w") as f:
            f.write("\n".join(logs))
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
