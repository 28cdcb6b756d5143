"""Build the CUDA shared library in-tree (nvcc, sm_103a only).

``python -m paper_2402_17580_gb300.build`` or ``build()`` compiles every
``csrc/*.cu`` translation unit in parallel and links ``_build/libms_gb300.so``
(CUDA runtime linked statically, no torch dependency).  Rebuilds only when a
source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libms_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(
        os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]


STAMP = os.path.join(BUILD, "flags.txt")


def _extra_flags():
    """Extra nvcc flags from MS_NVCC_FLAGS (tuning builds, e.g. -DMS_TRACK_MINB=8)."""
    return os.environ.get("MS_NVCC_FLAGS", "").split()


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return False
    if open(STAMP).read() != " ".join(_extra_flags()):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs, objs = [], []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        log = obj + ".log"
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *_extra_flags(), "-c", src, "-o", obj]
        procs.append((subprocess.Popen(cmd, stdout=open(log, "w"), stderr=subprocess.STDOUT), src, log))
        objs.append(obj)
    failed = []
    for p, src, log in procs:
        if p.wait() != 0:
            failed.append((src, log))
    for src, log in failed:
        sys.stderr.write(open(log).read())
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(s) for s, _ in failed))
    if verbose:
        for _, _, log in procs:
            sys.stdout.write(open(log).read())
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(" ".join(_extra_flags()))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
