"""Build the sm_103a shared library ``_lib/libnmpc_gb300.so`` with nvcc.

One translation unit (the C ABI plus the kernels it launches), compiled
in-tree; the output is git-ignored.  ``build()`` rebuilds only when a source
is newer than the library.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libnmpc_gb300.so")
SOURCES = [os.path.join(HERE, "csrc", "nmpc_capi.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", "nmpc_kernels.cuh"),
                  os.path.join(ROOT, "include", "nmpc.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = LIB_PATH + ".tmp"
    cmd = [nvcc_path(), "-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
           "-shared", "-o", tmp] + SOURCES
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
