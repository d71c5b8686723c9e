"""Builds libvpm.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

    python -m paper_2509_16079_b300.build [--verbose] [--debug-bounds]

--debug-bounds builds libvpm_debug.so instead, with the device-side bounds checks on
(VPM_DEBUG_BOUNDS); the Python binding loads it when VPM_DEBUG_BOUNDS=1 is set.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libvpm.so")
LIB_DEBUG = os.path.join(HERE, "libvpm_debug.so")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    # binary32 denormals flush to zero: the pair kernels never produce them in a meaningful
    # way (r^4 + r_core^4 >= r_core^4), and without the flush rsqrtf needs a fix-up sequence
    "-ftz=true",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-shared",
    "-cudart", "static",
    "-I", os.path.join(ROOT, "include"),
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "vpm.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    """Compiles every .cu file under csrc/ into libvpm.so (libvpm_debug.so with the device-side
    bounds checks) if a source is newer."""
    out = LIB_DEBUG if debug_bounds else LIB
    if not force and not _stale(out):
        return out
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [nvcc] + NVCC_FLAGS + (["-DVPM_DEBUG_BOUNDS=1"] if debug_bounds else []) + \
          (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp] + sources()
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
