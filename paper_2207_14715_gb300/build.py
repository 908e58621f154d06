"""Builds the VB-QMC CUDA library in-tree: paper_2207_14715_gb300/_lib/libvbqmc.so (sm_103a).

Each translation unit is compiled in parallel (nvcc for .cu, g++ for host .cpp), then linked
with nvcc into one shared library exporting the C ABI of include/vbqmc.h.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libvbqmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")

CU_SOURCES = ["kernels.cu", "eval_jastrow.cu", "eval_orbitals.cu", "eval_det.cu", "eval_dettab.cu", "eval_forces.cu",
              "dmc.cu", "gradient.cu", "linmethod.cu", "linmethod_noalloc.cu", "api.cu", "batch_api.cu", "peaks.cu", "batch_fused.cu"]
CPP_SOURCES = ["system_host.cpp", "host_linalg.cpp"]


def _headers():
    out = []
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                out.append(os.path.join(d, f))
    return out


def _stale(obj, src, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + deps)


def _compile(src, obj, extra=()):
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", src, "-o", obj, *extra]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-c", src, "-o", obj]
    subprocess.check_call(cmd)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    deps = _headers()
    jobs = []
    objs = []
    for src in CU_SOURCES + CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJDIR, src + ".o")
        objs.append(o)
        if force or verbose_ptxas or _stale(o, s, deps):
            jobs.append((s, o))
    if jobs:
        extra = ["-Xptxas", "-v"] if verbose_ptxas else []
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(_compile, s, o, extra if s.endswith(".cu") else ()) for s, o in jobs]
            for f in futs:
                f.result()
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv))
