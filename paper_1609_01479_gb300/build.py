"""Build the CUDA library libld.so in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel and linked
into paper_1609_01479_gb300/_lib/libld.so (CUDA runtime linked statically).
Rebuilds only when a source or header is newer than the library.

build(debug=True) makes _lib/libld_debug.so from the same sources with
-DLD_DEBUG_BOUNDS: the step kernels check every site index against the
lattice before a global access and report a bad one through ld_check instead
of faulting (slower; for tests).
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(PKG, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libld.so")
DEBUG_LIB_PATH = os.path.join(LIB_DIR, "libld_debug.so")
OBJ_DIR = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libld.so")
    return exe


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return False
    t = os.path.getmtime(path)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link libld.so (libld_debug.so with
    debug=True); returns its path."""
    lib_path = DEBUG_LIB_PATH if debug else LIB_PATH
    obj_dir = os.path.join(OBJ_DIR, "debug") if debug else OBJ_DIR
    flags = [*extra_flags, *(["-DLD_DEBUG_BOUNDS"] if debug else [])]
    if not force and up_to_date(lib_path):
        return lib_path
    os.makedirs(LIB_DIR, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        # the FP64 unit rounds every operation separately (no FMA contraction)
        per_file = ["-fmad=false"] if src.endswith("_f64.cu") else []
        cmd = [exe, *ARCH, *NVCC_FLAGS, *per_file, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking {os.path.basename(lib_path)} failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


def build_all(force: bool = False) -> None:
    """The release and the debug library, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        for f in [ex.submit(build, force), ex.submit(build, force, debug=True)]:
            f.result()


if __name__ == "__main__":
    print(build(force=True, verbose=True))
