"""Compile tests/c/pat_c_caller.c with gcc against include/pat.h, libpat.so and the CUDA runtime."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def build_c_caller(out_path: str) -> str:
    """Build the caller; returns the compiler's diagnostics (empty on a clean build), raises on failure."""
    libdir = os.path.join(ROOT, "paper_2505_08482_gb300", "_lib")
    cudalib = os.path.join(CUDA, "lib64")
    cmd = ["gcc", "-std=c99", "-O1", "-Wall", "-Wextra", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(HERE, "pat_c_caller.c"), "-o", out_path,
           "-L", libdir, "-lpat", "-L", cudalib, "-lcudart", f"-Wl,-rpath,{libdir}:{cudalib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr
