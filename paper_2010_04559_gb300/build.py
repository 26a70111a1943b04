"""Builds libamgt.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel and linked into one shared
library under paper_2010_04559_gb300/_build/.  Re-running only recompiles
sources newer than their objects.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libamgt.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU = ["capi.cu", "kernels_transport.cu", "kernels_gemm.cu", "kernels_blas.cu",
      "kernels_gs.cu", "kernels_gs_rows.cu", "kernels_gs_tc.cu", "kernels_tc.cu", "kernels_adjoint.cu",
      "kernels_split64.cu", "kernels_tc3.cu", "kernels_setup.cu"]
CPP = ["setup.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "amgt.h"))
    jobs = []
    objs = []
    for f in CU + CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if not _stale(obj, [src] + headers):
            continue
        if f.endswith(".cu"):
            cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-c", src, "-o", obj]
        else:
            cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-I", INCLUDE, "-c", src, "-o", obj]
        jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stdout.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("compilation failed: " + os.path.basename(cmd[-3]))
    if jobs or not os.path.exists(LIB):
        cmd = [nvcc, "-shared", *ARCH, "-o", LIB, *objs, "-lcudart", "-lcuda"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stdout.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
