"""Build ``libdies.so`` (the CUDA library behind include/dies.h) in-tree.

nvcc compiles each translation unit for sm_103a only, in parallel, and links
one shared library next to this file.  No CMake, no PyTorch extension
machinery: the library has a plain C ABI and the Python side loads it with
ctypes.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdies.so")
# the check build: device bounds checks that set status flags (-DDIES_CHECK), for debugging
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libdies_check.so")
SOURCES = ("dies_api.cu", "dies_tables.cu", "dies_transport.cu", "dies_peaks.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdies.so")


def _flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v",
            f"-I{os.path.join(HERE, '..', 'include')}", *extra]


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    with open(obj + ".log", "w") as f:
        f.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{p.stderr[-4000:]}")
    return obj


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "dies.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, extra=(), check: bool = False) -> str:
    """Compile and link libdies.so (with ``check``: libdies_check.so, the
    device-bounds-check build) if any source is newer than it; return its path."""
    lib, bdir = (LIB_CHECK, BUILD_CHECK) if check else (LIB, BUILD)
    extra = tuple(extra) + (("-DDIES_CHECK",) if check else ())
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, bdir), SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr[-4000:]}")
    os.replace(tmp, lib)
    return lib


def ptxas_report() -> str:
    """Register / spill / shared-memory lines of the last build (from -Xptxas -v)."""
    out = []
    for s in SOURCES:
        log = os.path.join(BUILD, os.path.splitext(s)[0] + ".o.log")
        if os.path.exists(log):
            out += [l for l in open(log) if "registers" in l or "spill" in l or "Compiling entry" in l]
    return "".join(out)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(ptxas_report())
