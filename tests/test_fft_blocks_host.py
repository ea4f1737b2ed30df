"""The register FFT building blocks of the fixed-size passes, run on the CPU.

The two- and three-level transforms (fft2l.cuh) and their register DFTs are
__host__ __device__ code: `tests/host/fft2l_host.cu` compiles the same header
for the host and runs, for every factorisation N = N1 x N2 of the compiled grid
sides (108, 144, 180, 200, 240, 300, in both orders), the three-level
factorisations N = NA x NM x NB of the compiled sides and a few others, the
forward transform through the A (and M) and B layouts, its inverse through the
B (and M) and A layouts, and the plain register DFTs of the outer lengths.  The results are
compared with numpy's FFT in FP64 (the DFT's definition up to rounding): a
wrong twiddle exponent, sign or index, or a mis-ordered output, fails here
without a GPU.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2505_08482_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "host", "fft2l_host.cu")
CASES = [(12, 9), (9, 12), (12, 12), (12, 15), (15, 12), (20, 10), (10, 20), (16, 15), (15, 16),
         (20, 15), (15, 20), (2, 3), (4, 5), (8, 25)]
CASES3 = [(5, 10, 6), (5, 12, 5), (5, 6, 10), (4, 3, 9), (3, 4, 5), (2, 3, 2)]


@pytest.fixture(scope="module")
def host_binary(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("fft2l") / "fft2l_host")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, SRC, "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _run(binary, xs):
    """xs: ((n1, n2) or (na, nm, nb), x); returns (X, y, d, e) per case."""
    blob = [struct.pack("<i", len(xs))]
    for f, x in xs:
        blob.append(struct.pack("<iii", *(tuple(f) + (0,) * (3 - len(f)))))
        blob.append(np.stack([x.real, x.imag], -1).astype("<f4").tobytes())
    r = subprocess.run([binary], input=b"".join(blob), capture_output=True)
    assert r.returncode == 0, r.stderr.decode()
    out = np.frombuffer(r.stdout, dtype="<f4")
    res, o = [], 0
    for f, _ in xs:
        N = int(np.prod(f))
        parts = []
        for m in (N, N, f[0], f[-1]):
            parts.append(out[o:o + 2 * m].astype(np.float64).view(np.complex128))
            o += 2 * m
        res.append(parts)
    assert o == out.size
    return res


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_two_level_transforms_match_the_dft_definition(host_binary):
    rng = np.random.default_rng(2505)
    xs = []
    for n1, n2 in CASES:
        x = (rng.standard_normal(n1 * n2) + 1j * rng.standard_normal(n1 * n2)).astype(np.complex64)
        xs.append(((n1, n2), x))
    for ((n1, n2), x), (X, y, d, e) in zip(xs, _run(host_binary, xs)):
        x64 = x.astype(np.complex128)
        N = n1 * n2
        tol = 2e-6 * max(1.0, np.log2(N) / 4)
        assert _rel(X, np.fft.fft(x64)) < tol, (n1, n2, "forward")
        assert _rel(y, N * x64) < tol, (n1, n2, "inverse of forward")
        assert _rel(d, np.fft.fft(x64[:n1])) < tol, (n1, "register DFT")
        assert _rel(e, np.fft.fft(x64[:n2])) < tol, (n2, "register DFT")


def test_single_modes_land_on_their_bins(host_binary):
    """A pure exponential exp(2 pi i j n / N) transforms to N at bin j and ~0 elsewhere."""
    xs = []
    for n1, n2 in [(20, 15), (15, 20), (16, 15)]:
        N = n1 * n2
        for j in (1, n1, n2 + 1, N // 2, N - 1):
            xs.append(((n1, n2), np.exp(2j * np.pi * j * np.arange(N) / N).astype(np.complex64)))
    for ((n1, n2), x), (X, y, _, _) in zip(xs, _run(host_binary, xs)):
        N = n1 * n2
        j = int(np.argmax(np.abs(X)))
        ref = np.zeros(N, complex)
        ref[int(round(np.angle(x[1]) / (2 * np.pi) * N)) % N] = N
        assert np.abs(X - ref).max() < 1e-4 * N, (n1, n2, j)


def test_three_level_transforms_match_the_dft_definition(host_binary):
    rng = np.random.default_rng(2506)
    xs = []
    for f in CASES3:
        N = int(np.prod(f))
        x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
        xs.append((f, x))
    for (f, x), (X, y, d, e) in zip(xs, _run(host_binary, xs)):
        x64 = x.astype(np.complex128)
        N = int(np.prod(f))
        tol = 2e-6 * max(1.0, np.log2(N) / 4)
        assert _rel(X, np.fft.fft(x64)) < tol, (f, "forward")
        assert _rel(y, N * x64) < tol, (f, "inverse of forward")
        assert _rel(d, np.fft.fft(x64[:f[0]])) < tol, (f, "register DFT")
        assert _rel(e, np.fft.fft(x64[:f[-1]])) < tol, (f, "register DFT")


def test_three_level_single_modes_land_on_their_bins(host_binary):
    xs = []
    for f in [(5, 10, 6), (5, 12, 5)]:
        N = int(np.prod(f))
        for j in (1, f[0], f[0] * f[1] + 1, N // 2, N - 1):
            xs.append((f, np.exp(2j * np.pi * j * np.arange(N) / N).astype(np.complex64)))
    for (f, x), (X, _, _, _) in zip(xs, _run(host_binary, xs)):
        N = int(np.prod(f))
        ref = np.zeros(N, complex)
        ref[int(round(np.angle(x[1]) / (2 * np.pi) * N)) % N] = N
        assert np.abs(X - ref).max() < 1e-4 * N, f
