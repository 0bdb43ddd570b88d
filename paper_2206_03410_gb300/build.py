"""Builds libnrr.so (the C-ABI registration library) in-tree for sm_103a.

Sources are compiled in parallel (nvcc for .cu, g++ for .cpp) into
``_build/`` next to this file and linked with nvcc into ``_build/libnrr.so``.
A rebuild happens only when a source or header is newer than the library.
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
LIB = os.path.join(BUILD, "libnrr.so")

CU_SOURCES = ["kernels_nn.cu", "kernels_system.cu", "kernels_solve.cu", "kernels_aa.cu", "kernels_unroll.cu", "kernels_lbfgs.cu",
              "graph_gpu.cu", "nrr_api.cu", "noalloc.cu"]
CPP_SOURCES = ["graph_build.cpp", "geodesic.cpp"]
HEADERS = ["nrr_internal.h", "nrr_device.cuh", "nrr_rotation.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I", INCLUDE, "-I", CSRC]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INCLUDE,
             "-I", CSRC, "-I", "/usr/local/cuda/include"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    deps += [os.path.join(INCLUDE, "nrr.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compiles the library if needed and returns the path of libnrr.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, f), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((f, cmd))
        objs.append(obj)
    for f in CPP_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append((f, ["g++", *CXX_FLAGS, "-c", os.path.join(CSRC, f), "-o", obj]))
        objs.append(obj)
    procs = [(f, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
             for f, cmd in jobs]
    failed = []
    for f, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((f, text))
        elif verbose and text.strip():
            sys.stderr.write(f"--- {f}\n{text}\n")
    if failed:
        msg = "\n".join(f"--- {f}\n{t}" for f, t in failed)
        raise RuntimeError(f"libnrr build failed:\n{msg}")
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libnrr link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
