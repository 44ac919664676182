"""Builds the sm_103a shared library ``libsurflbm.so`` in-tree with nvcc.

Usage: ``python -m paper_2609_26332_b300.build [--verbose]``.  The library holds
the CUDA kernels and the C ABI declared in ``include/surflbm.h`` and
``include/surflbm_ws.h`` and ``include/surflbm3d.h``.
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libsurflbm.so")
SOURCES = ["surflbm_api.cu", "surflbm_batch.cu", "surflbm_exact.cu", "surflbm3d.cu", "ws_net.cu"]
HEADERS = ["surflbm_device.cuh", "surflbm_step.cuh", "surflbm_step_tile.inc", "surflbm_internal.cuh", "ws_tc.cuh", "ws_conv.cuh", "ws_conv_tma.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 denormals flushed, approximate FP32 division and square root: the few divisions and
# roots of the step are not on the conserved paths (moments are float-float sums and the
# exchange is fixed point), and every result stays within the oracle tolerances
FLOAT_FLAGS = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", h) for h in ("surflbm.h", "surflbm_ws.h", "surflbm3d.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(verbose=False, force=False):
    if not force and not needs_build():
        return LIB
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, *FLOAT_FLAGS, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-o", LIB + ".tmp"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, f) for f in SOURCES]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed building libsurflbm.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, force=True)
    print(LIB)
