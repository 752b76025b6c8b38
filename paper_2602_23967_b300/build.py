"""Build libpdhcg.so for sm_103a with nvcc (in-tree, no JIT cache).

Usage: python -m paper_2602_23967_b300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpdhcg.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels_f64.cu", "kernels_f32.cu", "kernels_mixed.cu", "kernels_dfloat.cu", "pdhcg_api.cu",
              "pdhcg_server.cu", "selftest.cu", "autotune.cu"]
CPP_SOURCES = ["host_prep.cpp"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "pdhcg.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(src, out_dir=None, defines=()):
    obj = os.path.join(out_dir or OUT_DIR, os.path.basename(src) + ".o")
    if src.endswith(".cu"):
        cmd = [NVCC, "-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", *defines,
               "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    else:
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-I", INCLUDE, "-I", CSRC,
               "-I", "/usr/local/cuda/include", "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, lib_path: str | None = None,
          defines=()) -> str:
    """Compile every source and link libpdhcg.so (``defines``: extra -D flags, used
    with ``lib_path`` to build tuning variants next to the default library)."""
    lib = lib_path or LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps():
        return lib
    out_dir = OUT_DIR if not defines else OUT_DIR + "_" + "_".join(d.strip("-D").replace("=", "") for d in defines)
    os.makedirs(out_dir, exist_ok=True)
    srcs = [s for s in CU_SOURCES + CPP_SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, out_dir, defines), srcs))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
