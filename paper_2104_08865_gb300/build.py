"""Builds libhalftime.so and its checked twin in-tree with nvcc for sm_103a.

Every translation unit under csrc/ compiles in parallel to an object under
_build/ (and, with -DHT_CHECK, under _build_check/), then nvcc links them
(static CUDA runtime) into paper_2104_08865_gb300/libhalftime.so and
libhalftime_check.so (the debug library whose kernels range-check every
global access).  Rebuilds only when a source or header is newer than a
library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhalftime.so")
BUILD_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(PKG, "libhalftime_check.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    targets = [(lib, d, flags) for lib, d, flags in ((LIB, BUILD, []), (LIB_CHECK, BUILD_CHECK, ["-DHT_CHECK"]))
               if force or stale(lib)]
    if not targets:
        return LIB
    nvcc = _nvcc()
    procs = []
    links = []
    for lib, bdir, extra in targets:
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in sources():
            obj = os.path.join(bdir, os.path.basename(src) + ".o")
            objs.append(obj)
            cmd = [nvcc] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [nvcc] + NVCC_FLAGS + extra + ["-x", "c++", "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        links.append((lib, objs))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join("%s:\n%s" % f for f in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    for lib, objs in links:
        tmp = lib + ".tmp.%d" % os.getpid()
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
