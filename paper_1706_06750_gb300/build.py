"""In-tree build of libkaze.so for sm_103a (GB300).

Each CUDA translation unit under ``csrc/`` is compiled by nvcc in parallel
into ``_build/`` and linked into ``_build/libkaze.so`` (CUDA runtime linked
statically, only the C ABI of ``include/kaze.h`` exported).  A rebuild
happens only when a source or header is newer than the library.

    python -m paper_1706_06750_gb300.build
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libkaze.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-fvisibility=hidden", "-Xptxas", "-v"]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkaze.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(INCLUDE, "*.h"))


def is_fresh() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ and link libkaze.so; returns its path."""
    with _lock:
        if not force and is_fresh():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        cc = nvcc()
        procs = []
        objs = []
        for src in sources():
            obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
            log = obj + ".log"
            cmd = [cc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
            f = open(log, "w")
            procs.append((subprocess.Popen(cmd, stdout=f, stderr=subprocess.STDOUT), f, log, src))
            objs.append(obj)
        failed = []
        for p, f, log, src in procs:
            rc = p.wait()
            f.close()
            if rc != 0 or verbose:
                with open(log) as fh:
                    text = fh.read()
                if rc != 0:
                    failed.append(f"{os.path.basename(src)}:\n{text}")
                elif verbose:
                    sys.stdout.write(text)
        if failed:
            raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"])
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
