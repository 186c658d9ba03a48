"""In-tree build of libgfopt.so with nvcc for sm_103a (no cmake, no setuptools).

Each .cu translation unit is compiled in parallel, then linked into
paper_2202_05388_gb300/_lib/libgfopt.so.  A stamp file keyed on the sources, flags and the
host machine type makes repeated calls cheap and forces a rebuild on another architecture.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libgfopt.so")
STAMP = os.path.join(LIBDIR, "build.stamp")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fno-strict-aliasing", "--expt-relaxed-constexpr",
                     "-I", INCLUDE]


# Translation units that compile the shared stage bodies (csrc/gf_stage_bodies.cuh) contract a
# multiply and an add into one FMA only where the source writes fma(): otherwise the compiler's
# contraction choices differ between the kernels that inline the same body, and the batched, the
# persistent and the single-problem kernels would disagree in the last bits.
SHARED_BODY_FLAGS = ["-fmad=false"]


def _flags_for(src: str):
    with open(os.path.join(CSRC, src)) as fh:
        return SHARED_BODY_FLAGS if '#include "gf_stage_bodies.cuh"' in fh.read() else []


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgfopt")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    hdr = sorted(f for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    return cu, hdr


def _digest(extra_flags) -> str:
    cu, hdr = _sources()
    h = hashlib.sha256()
    for f in cu + hdr:
        h.update(f.encode())
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(INCLUDE, "gfopt.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + SHARED_BODY_FLAGS + list(extra_flags)).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(verbose: bool = False, extra_flags=(), force: bool = False) -> str:
    """Compile and link libgfopt.so if the sources changed; return its path."""
    digest = _digest(extra_flags)
    if not force and os.path.exists(LIB) and os.path.exists(STAMP):
        with open(STAMP) as fh:
            if fh.read().strip() == digest:
                return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cu, _ = _sources()
    objs = [os.path.join(BUILD, f[:-3] + ".o") for f in cu]

    def compile_one(args):
        src, obj = args
        cmd = [nvcc] + NVCC_FLAGS + _flags_for(src) + list(extra_flags) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    workers = min(len(cu), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for out in ex.map(compile_one, zip(cu, objs)):
            if verbose and out:
                sys.stderr.write(out)
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
