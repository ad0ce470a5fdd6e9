"""Build libocg.so in-tree with nvcc for sm_103a (B300)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libocg.so")
SOURCES = ["ocg_api.cu", "octree_host.cpp"]
DEPS = SOURCES + ["kernels.cuh", "octet.cuh", "batch.cuh", "batch_host.cuh", "octree_host.h"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def needs_build():
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    paths = [os.path.join(CSRC, f) for f in DEPS] + [os.path.join(HERE, "..", "include", "ocg.h")]
    return any(os.path.getmtime(p) > t for p in paths)


def build(verbose=False, force=False):
    if not force and not needs_build():
        return OUT
    cmd = [_nvcc(), "-O3", "-std=c++17", "-shared", "-lineinfo",
           "-gencode", "arch=compute_103a,code=sm_103a",
           "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off",
           "-Xptxas", "-v" if verbose else "-O3",
           "-o", OUT] + [os.path.join(CSRC, f) for f in SOURCES] + ["-lgomp"]
    if verbose:
        print(" ".join(cmd))
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building libocg.so")
    if verbose:
        sys.stderr.write(res.stderr)
    return OUT


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, force=True)
    print(OUT)
