"""Build libpyro.so in-tree: host C++ (parser, emitter, runtime) with g++, CUDA
sources with nvcc for sm_103a, linked against the static CUDA runtime and NVRTC.

Usage: python -m paper_2503_24286_gb300.build   (or build() from Python).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "_lib", "libpyro.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _embed_devmath() -> str:
    src = open(os.path.join(CSRC, "pyro_device_math.cuh")).read()
    out = os.path.join(BUILD, "pyro_devmath_src.cpp")
    text = ('// generated from pyro_device_math.cuh\nnamespace pyro {\n'
            'extern const char* kDeviceMathSource;\n'
            'const char* kDeviceMathSource = R"PYRODM(' + src + ')PYRODM";\n}\n')
    if not os.path.exists(out) or open(out).read() != text:
        with open(out, "w") as f:
            f.write(text)
    return out


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp"))) + [_embed_devmath()]
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = []
    for s in cpp:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function", "-I", INCLUDE, "-I", CSRC,
               "-I", os.path.join(CUDA, "include"), "-c", s, "-o", o]
        jobs.append((o, cmd, [s] + headers))
    for s in cu:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        cmd = [os.path.join(CUDA, "bin", "nvcc"), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-I", CSRC, "-c", s, "-o", o]
        jobs.append((o, cmd, [s] + headers))
    todo = [(o, c) for o, c, d in jobs if _stale(o, d)]

    def run(item):
        o, c = item
        if verbose:
            print(" ".join(c))
        r = subprocess.run(c, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(c), r.stdout, r.stderr))
        return o
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, len(todo)))) as ex:
        list(ex.map(run, todo))
    objs = [o for o, _, _ in jobs]
    if todo or not os.path.exists(LIB) or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-shared", "-o", tmp, *objs, "-L", os.path.join(CUDA, "lib64"), "-lcudart_static", "-lnvrtc",
               "-ldl", "-lpthread", "-lrt", "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-Wl,--no-undefined"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
