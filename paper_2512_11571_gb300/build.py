"""Build libcemtamp.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  Portable flags only: the same command builds on
the x86 development host and on the Arm (Grace) GPU host.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libcemtamp.so")
BUILD = os.path.join(HERE, "_build")
# the debug build: the same sources with the kernels' bounds checks compiled in
# (-DCEM_DEBUG; see cem_debug_status), in its own object folder and library
DEBUG_OUT = os.path.join(HERE, "libcemtamp_debug.so")
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
SOURCES = ["capi.cu", "sample.cu", "rollout.cu", "refit.cu", "batch.cu", "surrogate.cu", "mlp_tc.cu", "gemm_tc.cu", "solve_static.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-O3"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcemtamp")
    return p


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(HERE, "..", "include", "cemtamp.h"))
    return hdrs


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, debug: bool = False) -> str:
    out, folder = (DEBUG_OUT, DEBUG_BUILD) if debug else (OUT, BUILD)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    paths = [os.path.join(CSRC, s) for s in srcs]
    newest = max(os.path.getmtime(p) for p in paths + _deps() + [__file__])
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    os.makedirs(folder, exist_ok=True)
    cc = nvcc()
    extra = (extra or []) + (["-DCEM_DEBUG"] if debug else [])

    def compile_one(src):
        obj = os.path.join(folder, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(paths))) as ex:
        objs = list(ex.map(compile_one, paths))
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None, debug="--debug" in sys.argv))
