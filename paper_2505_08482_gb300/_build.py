"""Compile the CUDA library ``libpat.so`` in-tree for sm_103a with nvcc.

Each ``csrc/*.cu`` translation unit is compiled in parallel into
``_build/`` and linked into ``paper_2505_08482_gb300/_lib/libpat.so``.  The
library is rebuilt when a source or header is newer than it.

``build(debug=True)`` builds the same sources with ``-DPAT_DEBUG_BOUNDS``
into ``_build_debug/`` and ``_lib/libpat_debug.so``: device-side bounds
checks on the indices that come from run-time data, reported through the
status word (PAT_STATUS_BOUNDS).  The binding loads it instead of
``libpat.so`` when the environment has ``PAT_DEBUG_BOUNDS=1``.
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
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libpat.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(LIBDIR, "libpat_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpat.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))) + \
        [os.path.join(ROOT, "include", "pat.h")]


def is_stale(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None, debug: bool = False) -> str:
    """Build libpat.so (debug: libpat_debug.so with the bounds checks) if needed and return its path.

    Processes that build at the same time (the ranks of a multi-process launch) take turns on a
    lock file; the first one builds and the others then find the library up to date.
    """
    import fcntl
    lib = LIB_DEBUG if debug else LIB
    if not force and not is_stale(debug):
        return lib
    os.makedirs(LIBDIR, exist_ok=True)
    with open(os.path.join(LIBDIR, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and not is_stale(debug):
                return lib
            return _compile(lib, BUILD_DEBUG if debug else BUILD, verbose, extra_flags, debug)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _compile(lib: str, bdir: str, verbose: bool, extra_flags, debug: bool) -> str:
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--cudart", "shared",
                    "-I", os.path.join(ROOT, "include")] + (["-DPAT_DEBUG_BOUNDS"] if debug else []) + \
        list(extra_flags or [])
    objs = []
    cmds = []
    for src in _sources():
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        objs.append(obj)
        cmds.append([nvcc] + flags + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        for out in ex.map(run, cmds):
            if verbose and out.strip():
                print(out)
    link = [nvcc] + ARCH + ["-shared", "--cudart", "shared", "-o", lib + ".tmp"] + objs + \
        ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    run(link)
    os.replace(lib + ".tmp", lib)
    return lib
