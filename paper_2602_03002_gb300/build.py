"""Builds librpl.so in-tree with nvcc for sm_103a (host code with the system C++ compiler via nvcc).

Translation units are compiled in parallel and linked with the static CUDA runtime, so the library
loads next to PyTorch without depending on where libcudart lives.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librpl.so")
# bounds-checked build (every node and triangle index tested before it is read; see render.cu)
LIB_CHECKED = os.path.join(HERE, "librpl_checked.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["render.cu", "rpl_api.cpp", "bvh_build.cpp", "bvh8.cpp", "bvh4.cpp", "noalloc.cu", "server.cpp"]
HEADERS = ["bvh.h", "bvh8.h", "bvh4.h", "render.h", "scene_access.h"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librpl.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "rpl.h"),
                                                                  os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, checked: bool = False) -> str:
    """Compile and link librpl.so (or, with checked, librpl_checked.so, whose kernels test every node
    and triangle index against its array) unless it is up to date. Returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    out_dir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(out_dir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden,-ffp-contract=off",
              "-I", os.path.join(ROOT, "include")] + (["-DRPL_CHECKED"] if checked else [])

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, src + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + common
        if src.endswith(".cu"):
            cmd += ARCH + ["-lineinfo"]
            if ptxas_v:
                cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compiling %s failed:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose or ptxas_v:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("linking librpl.so failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv))
