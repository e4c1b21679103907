"""Builds the CUDA library libbdra.so in-tree for sm_103a.

The translation units compile in parallel: the float32 and float64
instantiations of the parent / replica kernels (the replica kernels twice:
without and with the Eq. 5 diagnostics) and of the adjoint kernels
(with -fmad=false, so every fused multiply-add is the explicit one written
in the source), the support kernels, the C ABI, the allocation-free
event compaction and the Philox-round throughput probe. Only nvcc is needed; no CMake.
"""
from __future__ import annotations

import concurrent.futures as cf
import contextlib
import fcntl
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libbdra.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
UNITS = [("bd_window_f32.cu", ["-fmad=false"]), ("bd_window_f64.cu", ["-fmad=false"]),
         ("bd_window_f32c.cu", ["-fmad=false"]), ("bd_window_f64c.cu", ["-fmad=false"]),
         ("bd_hi_f32.cu", ["-fmad=false"]), ("bd_hi_f64.cu", ["-fmad=false"]),
         ("bd_window_f32b.cu", ["-fmad=false"]),
         ("bd_adjoint_f32.cu", ["-fmad=false"]), ("bd_adjoint_f64.cu", ["-fmad=false"]),
         ("bd_support.cu", []), ("bd_api.cu", []), ("bd_noalloc.cu", []), ("bd_probe.cu", [])]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _sources():
    out = []
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    out.append(os.path.join(ROOT, "include", "bdra.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


@contextlib.contextmanager
def _locked(objdir: str):
    """One build at a time per object directory (test processes that start
    together would otherwise write the same objects and library)."""
    os.makedirs(objdir, exist_ok=True)
    with open(os.path.join(objdir, ".lock"), "w") as fh:
        fcntl.flock(fh, fcntl.LOCK_EX)
        try:
            yield
        finally:
            fcntl.flock(fh, fcntl.LOCK_UN)


def build(force: bool = False, verbose: bool = False, out: str = None,
          defines=(), csrc: str = None) -> str:
    """Compile csrc/ (or another source directory) into libbdra.so (or `out`),
    with optional -D defines."""
    lib = out or LIB
    src_dir = csrc or CSRC
    default = out is None and not defines and csrc is None
    if not force and default and up_to_date():
        return LIB
    objdir = os.path.join(os.path.dirname(lib), "_build") if out else os.path.join(PKG, "_build")
    with _locked(objdir):
        if not force and default and up_to_date():     # built by another process meanwhile
            return LIB
        return _build(lib, src_dir, objdir, defines, verbose)


def _build(lib: str, src_dir: str, objdir: str, defines, verbose: bool) -> str:
    nvcc = _nvcc()

    def compile_unit(unit):
        src, extra = unit
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *[f"-D{d}" for d in defines], *extra, "-c",
               os.path.join(src_dir, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
