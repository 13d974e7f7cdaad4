"""Builds the checker's shared library in-tree: ``libdrfcheck.so`` next to
this file.  CUDA sources are compiled for sm_103a only (B300); host sources
with g++.  Incremental: a source is recompiled when it or any header under
``csrc/`` or ``include/`` is newer than its object."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdrfcheck.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXXFLAGS = ["-std=c++17", "-O3", "-fPIC", "-Wall"]


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "**", "*.cu"), recursive=True))
    cpp = sorted(glob.glob(os.path.join(CSRC, "**", "*.cpp"), recursive=True))
    return cu, cpp


def _headers():
    hs = glob.glob(os.path.join(CSRC, "**", "*.h"), recursive=True)
    hs += glob.glob(os.path.join(CSRC, "**", "*.cuh"), recursive=True)
    hs += glob.glob(os.path.join(ROOT, "include", "*.h"))
    return hs


# Headers the per-protocol kernels compiled at run time inline as text.
JIT_HEADERS = (("kJitDevprogH", "devprog.h"), ("kJitBatchArgsH", "batch_args.h"),
               ("kJitIntmathCuh", os.path.join("cuda", "intmath.cuh")),
               ("kJitOwnerCuh", os.path.join("cuda", "owner.cuh")))
GEN = os.path.join(BUILD, "gen")


def _gen_jit_headers():
    """Writes _build/gen/jit_headers.inc (the headers as C++ raw strings)
    when it is missing or older than one of them."""
    os.makedirs(GEN, exist_ok=True)
    out = os.path.join(GEN, "jit_headers.inc")
    srcs = [os.path.join(CSRC, rel) for _, rel in JIT_HEADERS]
    if os.path.exists(out) and os.path.getmtime(out) >= max(os.path.getmtime(x) for x in srcs):
        return out
    parts = ["// Generated by build.py from the shared headers; do not edit.\n"]
    for (name, _), path in zip(JIT_HEADERS, srcs):
        text = open(path).read()
        if ")DRFH\"" in text:
            raise RuntimeError(f"{path} contains the raw-string delimiter")
        parts.append(f'static const char {name}[] = R"DRFH({text})DRFH";\n')
    tmp = out + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write("".join(parts))
    os.replace(tmp, out)
    return out


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compiles what is out of date and links the library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp = _sources()
    gen = _gen_jit_headers()
    newest_header = max([os.path.getmtime(h) for h in _headers()] + [os.path.getmtime(gen)])
    objs = []
    for src in cu + cpp:
        rel = os.path.relpath(src, CSRC).replace(os.sep, "_")
        obj = os.path.join(BUILD, rel + ".o")
        objs.append(obj)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header):
            continue
        if src.endswith(".cu"):
            cmd = [NVCC, "-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        else:
            cmd = ["g++", *CXXFLAGS, "-I", "/usr/local/cuda/include", "-I", os.path.join(ROOT, "include"),
                   "-I", GEN, "-c", src, "-o", obj]
        _run(cmd, verbose)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([NVCC, "-shared", *ARCH, "-Xcompiler", "-fPIC", "-o", tmp, *objs,
              "-cudart", "static", "-lpthread", "-ldl"], verbose)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
