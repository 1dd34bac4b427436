"""Compile libhz.so (C ABI of the solver) in-tree for sm_103a.

Each translation unit is compiled in parallel into ``_build/``; the library is
linked with nvcc.  A rebuild only happens when a source is newer than the
library.
"""
import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhz.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["setup.cpp", "symbolic.cpp", "kernels.cu", "capi.cu", "noalloc.cu", "server.cpp", "recycle.cpp"]
HEADERS = ["host.h", "dev.h", "engine.h", "small_la.h"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _cmd(src, obj):
    path = os.path.join(CSRC, src)
    inc = ["-I" + os.path.join(ROOT, "include")]
    if src.endswith(".cu"):
        return [_nvcc(), "-c", path, "-o", obj, "-O3", "-lineinfo", "-std=c++17", *ARCH,
                "-Xcompiler", "-fPIC,-fopenmp", *inc]
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "include")
    return ["g++", "-c", path, "-o", obj, "-O3", "-std=c++17", "-fPIC", "-fopenmp",
            "-I" + cuda_inc, *inc]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "hz.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile the library; returns its path.  Raises on a compiler error."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = [os.path.join(BUILD, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    cmds = [_cmd(s, o) for s, o in zip(SOURCES, objs)]

    def run(cmd):
        if verbose:
            print(" ".join(cmd))
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + p.stdout + p.stderr)
        return p.stderr

    with concurrent.futures.ThreadPoolExecutor(len(cmds)) as ex:
        for out in ex.map(run, cmds):
            if verbose and out:
                print(out)
    tmp = LIB + ".tmp"
    run([_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
