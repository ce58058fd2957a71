"""Build the decoder library (CUDA, sm_103a) in-tree with nvcc.

Produces ``paper_2507_03509_gb300/libldpc_gb300.so`` exporting the C ABI of
``include/ldpc.h``.  Rebuilds only when a source is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libldpc_gb300.so")
LIB_CHECKED = os.path.join(PKG, "libldpc_gb300_checked.so")  # index-checking build (-DLDPC_BOUNDS_CHECK)
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is needed to build the decoder")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + [os.path.join(ROOT, "include", "ldpc.h")])


def nvcc_flags() -> list[str]:
    # -ftz=true: single-precision denormals flush to zero (sign kept), which drops the
    # denormal fix-ups around the MUFU intrinsics; the decoder's values never get there.
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC,-O2", "-Xcompiler",
            "-fvisibility=hidden", "-I" + os.path.join(ROOT, "include")]


UNITS = ("ldpc_api.cu", "wbp_api.cu")  # translation units, compiled in parallel


def checked_requested() -> bool:
    """The binding loads the index-checking build when LDPC_GB300_CHECKED is set."""
    return os.environ.get("LDPC_GB300_CHECKED", "0") not in ("", "0")


def build(force: bool = False, verbose: bool = False, checked: bool | None = None) -> str:
    """Build the library (the index-checking variant when `checked`, by default
    when LDPC_GB300_CHECKED is set) unless it is newer than every source."""
    if checked is None:
        checked = checked_requested()
    lib = LIB_CHECKED if checked else LIB
    newest = max(os.path.getmtime(s) for s in sources())
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    out = os.path.join(PKG, "_build")
    os.makedirs(out, exist_ok=True)
    tag = f"{os.getpid()}{'c' if checked else ''}"
    objs = [os.path.join(out, f"{os.path.splitext(u)[0]}.{tag}.o") for u in UNITS]
    procs = []
    for unit, obj in zip(UNITS, objs):
        cmd = [nvcc_path(), *nvcc_flags(), *(["-DLDPC_BOUNDS_CHECK"] if checked else []), "-c", "-o", obj,
               os.path.join(CSRC, unit)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
    failed = [u for u, pr in zip(UNITS, procs) if pr.wait() != 0]
    if failed:
        raise RuntimeError(f"nvcc failed on {', '.join(failed)}")
    tmp = lib + f".{tag}.tmp"
    subprocess.run([nvcc_path(), ARCH, "-shared", "-o", tmp, *objs], check=True)
    for obj in objs:
        os.remove(obj)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
