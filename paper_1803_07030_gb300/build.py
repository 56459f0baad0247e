"""Builds the CUDA library (libvegas.so) in-tree for sm_103a with nvcc and g++.

The translation units compile in parallel; the CUDA runtime is linked statically, so
the library needs only the NVIDIA driver at run time.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libvegas.so")
LIB_DEBUG = os.path.join(OUT_DIR, "libvegas_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["vegas_kernels.cu", "vegas_staged.cu", "vegas_policy32.cu", "vegas_r32_renorm.cu", "vegas_wave.cu", "vegas_analysis.cu", "vegas_ising.cu", "vegas_capi.cu", "vegas_noalloc.cu", "vegas_loader.cpp"]
HEADERS = ["vegas_internal.h", "vegas_device.cuh", "vegas_staged.cuh", "vegas_r32.cuh", os.path.join("..", "..", "include", "vegas.h")]


def _nvcc() -> str:
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    return "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every translation unit and link libvegas.so; returns its path.

    debug=True builds libvegas_debug.so instead, whose staged sweep kernel checks every
    index and address it computes (a failed check is reported as a device error)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, src + f".{os.getpid()}{'.dbg' if debug else ''}.o")
        path = os.path.join(CSRC, src)
        if src.endswith(".cu"):
            # -ftz=true: FP32 subnormals flush to zero (spins, fields and energy changes are O(1);
            # the special-function instructions then need no subnormal fix-ups); FP64 is unaffected
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC", "-diag-suppress",
                   "1444", "-c", path, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            if debug:
                cmd.insert(1, "-DVEGAS_DEBUG_CHECKS")
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I/usr/local/cuda/include", "-c", path, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("compilation failed: " + "; ".join(failed))
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
