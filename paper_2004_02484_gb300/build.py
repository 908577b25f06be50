"""Build the sm_103a shared library ``_lib/libnmpc_gb300.so`` with nvcc.

Four translation units (the solver's C ABI with its kernels, the learned
warm start's network, the pinned-actuator solver of the paper's plate and
the second-order-in-time solver), compiled in parallel in-tree and linked
into one library; the outputs are git-ignored.  ``build()`` rebuilds only when a
source is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libnmpc_gb300.so")
SOURCES = [os.path.join(HERE, "csrc", "nmpc_capi.cu"), os.path.join(HERE, "csrc", "mlp_capi.cu"),
           os.path.join(HERE, "csrc", "plate_capi.cu"), os.path.join(HERE, "csrc", "wave_capi.cu")]
# every source and header the library is built from
DEPS = SOURCES + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh")) +
                        glob.glob(os.path.join(ROOT, "include", "*.h")))
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
    nvcc = nvcc_path()
    flags = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC"]
    if verbose:
        flags.append("-Xptxas=-v")
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(LIB_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc] + flags + ["-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd)))
    for cmd, p in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, cmd)
    tmp = LIB_PATH + ".tmp"
    subprocess.run([nvcc, ARCH, "-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
