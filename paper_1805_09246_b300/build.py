"""Builds libsse.so (the CUDA library behind include/sse.h) in place, for sm_103a."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsse.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
    "-Xcompiler", "-fvisibility=hidden", "-Xcompiler", "-ffp-contract=off",
]


# translation units: the API with every estimator kernel, and the roof microbenchmarks
UNITS = ["sse_api.cu", "microbench.cu"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def build(force: bool = False, verbose: bool = False, nvtx: bool | None = None, out: str | None = None) -> str:
    """Compile the translation units (sse_api.cu includes the kernels) into libsse.so if stale.
    nvtx (default: the SSE_NVTX environment variable) compiles in NVTX ranges around the
    entry points; out builds into another path (always rebuilt)."""
    if nvtx is None:
        nvtx = os.environ.get("SSE_NVTX", "0") not in ("", "0")
    lib = out or LIB
    newest = max(os.path.getmtime(s) for s in sources())
    if out is None and not force and not nvtx and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    cmd = [NVCC, *FLAGS, "-I", INCLUDE, "-o", lib + ".tmp", *[os.path.join(CSRC, u) for u in UNITS]]
    if nvtx:
        cmd.insert(1, "-DSSE_NVTX")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
