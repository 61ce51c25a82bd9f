"""Builds libdamf.so in-tree from csrc/*.cu for sm_103a (nvcc, one -gencode, parallel).

build(check=True) builds libdamf_check.so instead: the same sources with DAMF_CHECK defined,
which turns on device bounds checks (a failed check sets DAMF_ERR_BOUNDS and skips the access);
load it with DAMF_LIB_VARIANT=check.
"""

import concurrent.futures
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdamf.so")


def _paths(check: bool):
    if check:
        return os.path.join(HERE, "_build_check"), os.path.join(HERE, "libdamf_check.so"), ["-DDAMF_CHECK"]
    return BUILD, LIB, []


def _compile(src: str, verbose: bool, build_dir: str, extra) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    deps = [src, os.path.join(INCLUDE, "damf.h")] + glob.glob(os.path.join(CSRC, "*.cuh"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [NVCC] + ARCH + FLAGS + extra + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    subprocess.run(cmd, check=True)
    return obj


def build(verbose: bool = False, check: bool = False) -> str:
    build_dir, lib, extra = _paths(check)
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, build_dir, extra), srcs))
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, check="--check" in sys.argv))
