"""Build libnufftjac.so in-tree with nvcc for sm_103a (one -gencode, TUs compiled in parallel)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libnufftjac.so")
SOURCES = ["kernels_fft2_fwd_mid.cu", "kernels_fft2_fwd_first.cu", "kernels_fft2_inv_mid.cu", "kernels_fft2_inv_last.cu",
           "kernels_gather_d3.cu", "kernels_gather_d2.cu", "kernels_gather_d1.cu", "nufft_api.cu", "kernels_sort.cu",
           "kernels_fft.cu", "kernels_spread.cu", "kernels_strip.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--extended-lambda",
         "-Xcompiler", "-Wall", "-diag-suppress", "177"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def build(verbose=False, force=False):
    """Compile every CUDA translation unit and link the shared library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in ("common.cuh", "internal.h", "interp.cuh", "fft_dft.cuh", "fft_twostep.cuh")] + \
        [os.path.join(ROOT, "include", "nufftjac.h"), os.path.join(CSRC, "exports.map")]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in deps + [os.path.abspath(__file__)])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [exe] + ARCH + FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs + [
        "-Xlinker", "--version-script=" + os.path.join(CSRC, "exports.map"),
        "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
