"""Build the CUDA library in-tree (sm_103a) with nvcc.

Produces ``paper_2511_15624_gb300/_lib/libibp_gb300.so``.  Translation units are
compiled in parallel and linked once; nothing outside the package is written.
``build(check=True)`` makes the checked library ``libibp_gb300_check.so``
(-DIBP_CHECK: index guards that record an error instead of accessing out of
bounds), which the binding loads when IBP_LIB=check is set.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libibp_gb300.so")
LIB_CHECK = os.path.join(OUT_DIR, "libibp_gb300_check.so")
SOURCES = ["ibp_abi.cu", "abi_linear.cu", "abi_multi.cu", "kernels_aux.cu", "kernel_ctg.cu",
           "kernel_screen.cu", "kernels_bwd.cu", "noalloc.cu", "kernel_linear.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA library cannot be built")
    return cand


def _flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
            "-I" + os.path.join(PKG, "..", "include"), "--expt-relaxed-constexpr", *extra]


def build(force: bool = False, verbose: bool = False, extra_flags=(), check: bool = False) -> str:
    lib_path = LIB_CHECK if check else LIB
    if check:
        extra_flags = (*extra_flags, "-DIBP_CHECK")
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(PKG, "..", "include", "ibp.h"))
    if not force and os.path.exists(lib_path):
        t = os.path.getmtime(lib_path)
        if all(os.path.getmtime(d) <= t for d in deps):
            return lib_path
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src) + (".check.o" if check else ".o"))
        cmd = [nvcc, *_flags(extra_flags), "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        for obj, log in ex.map(compile_one, srcs):
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = lib_path + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcusolver", "-lcublas", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    for o in objs:
        os.remove(o)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
