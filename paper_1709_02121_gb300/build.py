"""Build the CUDA library libwbrw.so for sm_103a (GB300), in tree.

Eleven translation units (the kernels of each precision and phase-space model,
the resampling kernels, the C ABI and the Philox rate probe) are compiled in parallel with nvcc and
linked into
``paper_1709_02121_gb300/_build/libwbrw.so`` against the shared CUDA runtime
(the process shares one runtime with PyTorch).  No CMake, one -gencode.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libwbrw.so")
SOURCES = ["wbrw_fp32.cu", "wbrw_fp32_lean.cu", "wbrw_fp32_lean_batch.cu", "wbrw_fp64.cu",
           "wbrw_fp32_4d.cu", "wbrw_fp64_4d.cu",
           "wbrw_fp32_grad.cu", "wbrw_fp32_grad_lean.cu", "wbrw_fp64_grad.cu",
           "wbrw_common.cu", "wbrw_api.cu", "wbrw_probe.cu"]
HEADERS = ["wbrw_device.cuh", "wbrw_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(INCLUDE, "wbrw.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # host code: no contraction into fused multiply-adds, so that host-side
    # constants round as written on either host architecture
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-Xcompiler", "-ffp-contract=off",
                    "-I", INCLUDE, "-I", CSRC, "-Xptxas", "-v" if verbose else "-O3"]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out)
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    link = [nvcc(), "-shared"] + ARCH + objs + ["-o", tmp, "-cudart", "shared",
                                              "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("link failed: " + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
