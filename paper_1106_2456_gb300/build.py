"""Build libmsd (the CUDA path) in-tree for sm_103a with nvcc.

The library is plain C ABI (``include/msd.h``); nothing here links against PyTorch.
Each translation unit is compiled in parallel, then linked into
``paper_1106_2456_gb300/_lib/libmsd.so`` with the CUDA runtime linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from typing import List, Optional

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "_lib")
BUILDDIR = os.path.join(PKG, "_build")
SOURCES = ["msd_kernels.cu", "msd_backward.cu", "msd_vmc.cu", "msd_tc.cu", "msd_api.cu"]
# host-only translation units keep libstdc++ bounds assertions on (an out-of-range index
# aborts with a message instead of corrupting the heap)
HOST_CHECKED = {"msd_api.cu": ["-Xcompiler", "-D_GLIBCXX_ASSERTIONS"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def library_path() -> str:
    return os.path.join(LIBDIR, "libmsd.so")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmsd")


def _inputs() -> List[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".h", ".cuh"))]
    files.append(os.path.join(INCLUDE, "msd.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in _inputs())


def compile_flags(extra: Optional[List[str]] = None) -> List[str]:
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC,
             "--expt-relaxed-constexpr"]
    if extra:
        flags += extra
    return flags


def build(force: bool = False, verbose: bool = False, extra_flags: Optional[List[str]] = None) -> str:
    """Compile and link libmsd if any source changed; return the library path."""
    out = library_path()
    if not force and not _stale(out):
        return out
    os.makedirs(LIBDIR, exist_ok=True)
    os.makedirs(BUILDDIR, exist_ok=True)
    cc = nvcc()
    flags = compile_flags(extra_flags)

    def one(src: str) -> str:
        obj = os.path.join(BUILDDIR, os.path.splitext(src)[0] + ".o")
        extra = HOST_CHECKED.get(src, [])
        cmd = [cc, *flags, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"nvcc failed on {src}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or r.returncode:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode:
        raise RuntimeError("link of libmsd failed")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
