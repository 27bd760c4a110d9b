"""Build libclaire.so in-tree for sm_103a with nvcc (no JIT cache, no torch extension).

    python -m paper_2401_17493_b300.build
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libclaire.so")
SOURCES = ["kernels.cu", "mixed.cu", "claire_api.cu", "noalloc.cu", "unet.cu", "precond.cu"]
HEADERS = ["common.cuh", "internal.h", "sl_brick.cuh", "sl_tma.cuh", "sl_window.cuh", "fd8_march.cuh",
           "reduce.cuh",
           "device_setup.h", "tc_sm100.cuh"]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-shared",
    "--threads", "0",
]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "claire.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False, ptxas_info=False):
    """Compile the CUDA sources into paper_2401_17493_b300/libclaire.so."""
    if not force and not _stale():
        return LIB
    cmd = [_nvcc()] + NVCC_FLAGS
    if ptxas_info:
        cmd += ["-Xptxas", "-v"]
    cmd += ["-o", LIB + ".tmp"] + [os.path.join(CSRC, f) for f in SOURCES] + ["-lcufft"]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose and (res.stdout or res.stderr):
        print(res.stdout + res.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="-v" in sys.argv)
