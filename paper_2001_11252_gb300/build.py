"""Build the CUDA library in-tree for GB300 (sm_103a).

Five objects compiled in parallel -- the kernels twice with nvcc (H(a,x) by
Tasitsiomi's form, and by the Faddeeva function with -DRG_FADDEEVA=1), the
allocation-free entry point and the issue-rate probes with nvcc, the C-ABI host
code with g++ against the CUDA runtime -- linked into
``paper_2001_11252_gb300/_build/librascas_gb300.so``.  No CMake.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librascas_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [
        os.path.join(ROOT, "include", "rascas_gb300.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False, ptxas_v=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cu = cuda_home()
    nvcc = os.path.join(cu, "bin", "nvcc")
    inc = ["-I", os.path.join(cu, "include"), "-I", CSRC, "-I", os.path.join(ROOT, "include")]
    k_obj = os.path.join(BUILD, "kernels.o")
    f_obj = os.path.join(BUILD, "kernels_fad.o")
    h_obj = os.path.join(BUILD, "host.o")
    n_obj = os.path.join(BUILD, "noalloc.o")
    p_obj = os.path.join(BUILD, "probe_rates.o")
    kcmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
            os.path.join(CSRC, "kernels.cu"), "-o", k_obj, *inc]
    fcmd = [c if c != k_obj else f_obj for c in kcmd] + ["-DRG_FADDEEVA=1"]
    if ptxas_v:
        kcmd.insert(1, "-Xptxas=-v")
        fcmd.insert(1, "-Xptxas=-v")
    # no contraction into fused multiply-adds: the host's image-plane basis and
    # line constants are evaluated exactly as written, on x86 and on Arm
    hcmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-c", os.path.join(CSRC, "host.cpp"), "-o",
            h_obj, *inc]
    ncmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-c", os.path.join(CSRC, "noalloc.cu"),
            "-o", n_obj, *inc]
    pcmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-c", os.path.join(CSRC, "probe_rates.cu"),
            "-o", p_obj, *inc]
    cmds = (kcmd, fcmd, hcmd, ncmd, pcmd)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in cmds]
    outs = [p.communicate()[0].decode() for p in procs]
    for p, o, c in zip(procs, outs, cmds):
        if p.returncode != 0:
            raise RuntimeError("build failed: %s\n%s" % (" ".join(c), o))
        if verbose and o.strip():
            print(o)
    tmp = LIB + ".tmp%d" % os.getpid()
    lcmd = [nvcc, *ARCH, "-shared", "-o", tmp, k_obj, f_obj, h_obj, n_obj, p_obj, "-lcudart"]
    r = subprocess.run(lcmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(lcmd), r.stdout.decode()))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv)
    print(LIB)
