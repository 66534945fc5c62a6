"""Build libstereo.so in-tree for sm_103a (nvcc + g++, three translation units in parallel)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libstereo.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    return [os.path.join(CSRC, f) for f in ("kernels.cu", "retess.cu", "noalloc.cu", "mesh.cpp", "engine.cpp",
                                              "internal.h")] + \
           [os.path.join(ROOT, "include", "stereo.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources() if os.path.exists(s))


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + os.path.join(cuda, "include"), "-I" + os.path.join(ROOT, "include")]
    tmp = os.path.join(OUT_DIR, f"obj.{os.getpid()}")
    os.makedirs(tmp, exist_ok=True)
    jobs = {
        "kernels.o": [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                      "-Xptxas", "-warn-spills", *inc, "-c", os.path.join(CSRC, "kernels.cu")],
        # the plane solve uses explicitly rounded fp64 operations (no contraction)
        "retess.o": [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-warn-spills", *inc, "-c", os.path.join(CSRC, "retess.cu")],
        "noalloc.o": [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                      "-c", os.path.join(CSRC, "noalloc.cu")],
        # the plane solve is a fixed fp64 expression: no contraction into FMAs
        "mesh.o": ["g++", "-O3", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", *inc,
                   "-c", os.path.join(CSRC, "mesh.cpp")],
        "engine.o": ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", *inc, "-c", os.path.join(CSRC, "engine.cpp")],
    }
    procs = {}
    for obj, cmd in jobs.items():
        procs[obj] = subprocess.Popen(cmd + ["-o", os.path.join(tmp, obj)], stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True)
    try:
        failed = []
        for obj, p in procs.items():
            out, _ = p.communicate()
            if verbose or p.returncode != 0:
                sys.stderr.write(out)
            if p.returncode != 0:
                failed.append(obj)
        if failed:
            raise RuntimeError(f"libstereo build failed: {failed}")
        lib_tmp = LIB + f".{os.getpid()}.tmp"
        link = [nvcc, *ARCH, "-shared", "-o", lib_tmp, *[os.path.join(tmp, o) for o in jobs],
                "-cudart", "shared", "-Xlinker", "-rpath," + os.path.join(cuda, "lib64"), "-lpthread"]
        subprocess.check_call(link)
        os.replace(lib_tmp, LIB)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
