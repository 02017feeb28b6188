"""Build libdg.so in-tree with nvcc for sm_103a (host C++ and CUDA sources)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libdg.so")
BUILD = os.environ.get("DG_BUILD_DIR", os.path.join(ROOT, "_build"))
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
EXTRA = os.environ.get("DG_NVCC_FLAGS", "").split()   # extra nvcc flags (variant builds)
SOURCES = ["refelem.cpp", "setup.cpp", "api.cpp", "kernels.cu", "kernels_gen2.cu", "kernels_tc.cu", "kernels_prec.cu", "noalloc.cu", "mrlsrk.cu", "batch.cpp", "adjoint.cu", "source.cu", "tune.cpp"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    objs, cmds = [], []
    for s in SOURCES:
        src = os.path.join(SRC, s)
        obj = os.path.join(BUILD, s + ".o")
        deps = [src] + [os.path.join(SRC, h) for h in os.listdir(SRC) if h.endswith((".h", ".cuh"))]
        deps.append(os.path.join(ROOT, "include", "dg.h"))
        if not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(d) for d in deps):
            cmds.append([nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-fopenmp"] + EXTRA + [
                        "-I", os.path.join(ROOT, "include"), "-I", SRC, "-c", src, "-o", obj])
        objs.append(obj)
    # the translation units compile independently: run them side by side, the largest first
    cmds.sort(key=lambda c: -os.path.getsize(c[-3]))
    with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as pool:
        for c in cmds:
            if verbose:
                print(" ".join(c), flush=True)
        for r in pool.map(lambda c: subprocess.run(c), cmds):
            if r.returncode != 0:
                raise subprocess.CalledProcessError(r.returncode, r.args)
    cmd = [nvcc(), ARCH, "-shared", "-o", OUT] + objs + ["-lcudart", "-lgomp"]
    subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
