"""Compile the CUDA sources of the package into an in-tree shared library (sm_103a).

    python -m paper_1412_3228_gb300._build_lib

builds paper_1412_3228_gb300/_build/libhom.so with nvcc: each translation unit is compiled in
parallel for `-gencode arch=compute_103a,code=sm_103a` and linked with the static CUDA runtime.
The build is skipped when the library is newer than every source file.  build(debug=True) makes
the bounds-checked variant (-DHOM_DEBUG) in paper_1412_3228_gb300/_build_debug/libhom.so.
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
LIB = os.path.join(BUILD, "libhom.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libhom.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["hom_capi.cu", "hom_filter.cu", "hom_solver.cu", "hom_fast2d.cu", "hom_fast3d.cu", "hom_noalloc.cu", "hom_backward.cu", "hom_extrap.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhom.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build libhom.so (or its bounds-checked variant) if needed and return its path."""
    build_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE] + ARCH
    if debug:
        common.append("-DHOM_DEBUG")
    if os.environ.get("HOM_PTXAS_VERBOSE"):
        common += ["-Xptxas", "-v"]
    if os.environ.get("HOM_THREADS"):  # threads per CTA of the solver passes (tuning)
        common += ["-DHOM_THREADS=%d" % int(os.environ["HOM_THREADS"])]
    if os.environ.get("HOM_GREEN_TW2"):  # Green pass with a scalar twiddle table (tuning)
        common += ["-DHOM_GREEN_TW2=%d" % int(os.environ["HOM_GREEN_TW2"])]
    if os.environ.get("HOM_ROW_TW2"):  # row pass with a scalar twiddle table (tuning)
        common += ["-DHOM_ROW_TW2=%d" % int(os.environ["HOM_ROW_TW2"])]
    if os.environ.get("HOM_FAST3D_THREADS"):  # threads per CTA of the specialised 3D passes (tuning)
        common += ["-DHOM_FAST3D_THREADS=%d" % int(os.environ["HOM_FAST3D_THREADS"])]
    if os.environ.get("HOM_FAST_THREADS"):  # threads per CTA of the specialised 2D passes (tuning)
        common += ["-DHOM_FAST_THREADS=%d" % int(os.environ["HOM_FAST_THREADS"])]
    for d in os.environ.get("HOM_EXTRA_DEFINES", "").split():  # other build-time tunables (-DNAME=VALUE)
        if d.startswith("-D"):
            common.append(d)

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
