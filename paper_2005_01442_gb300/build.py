"""Builds libvrc.so (the CUDA kernels and the C ABI) in-tree with nvcc for sm_103a.

Translation units compile in parallel to objects under ``_build/`` and link into
``_build/libvrc.so``; a unit is recompiled only when it or a header is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libvrc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit multiply-add contraction, so the same source expression rounds
# the same way in every kernel (the adjoint replays the forward's transmittances bit for bit);
# every fused multiply-add in the kernels is written out with fmaf.
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-I",
              INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
# Units with device-side kernel launches: relocatable device code, linked on the device with
# the device runtime (cudadevrt) before the shared library is linked.
RDC_UNITS = {"k_serve_dl.cu"}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvrc")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = _headers_mtime()
    cc = nvcc()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            rdc = ["-rdc=true"] if os.path.basename(s) in RDC_UNITS else []
            jobs.append([cc, *ARCH, *NVCC_FLAGS, *rdc, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    if jobs or not os.path.exists(LIB):
        rdc_objs = [o for s, o in zip(srcs, objs) if os.path.basename(s) in RDC_UNITS]
        dlink = os.path.join(BUILD, "device_link.o")
        run([cc, *ARCH, "-Xcompiler", "-fPIC", "-dlink", *rdc_objs, "-o", dlink, "-lcudadevrt"])
        tmp = LIB + f".tmp{os.getpid()}"
        run([cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, dlink, "-lcudadevrt"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
