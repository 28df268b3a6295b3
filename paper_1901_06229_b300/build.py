"""Build libgeodock.so (the CUDA library) in-tree for sm_103a with nvcc."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", f) for f in ("gd_api.cu", "gd_search.cu", "gd_select.cu", "gd_features.cu",
                                                "gd_noalloc.cu", "gd_mlp.cu", "gd_peak.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("gd_internal.h", "gd_mlp.h", "gd_pack.h", "gd_peak.h")] + \
    [os.path.join(ROOT, "include", f) for f in ("geodock.h", "geodock_mlp.h")]
LIB = os.path.join(HERE, "libgeodock.so")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or stale():
        nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-o", tmp, *SRC]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
