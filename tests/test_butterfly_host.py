"""The register butterflies (DFT_2 .. DFT_32 of the Stockham passes, Sec. V-B:
radix-2 DIT steps over the split-radix DFT_8, constant roots fused into the
combine in tangent form) and the twiddle-mode-1 derivation of a pass's
twiddle powers from the table rows it reads, compiled for the host and checked
against numpy's FFT and the exact roots, without a GPU.  butterfly.cuh is plain FP32 arithmetic; a host compiler
treats its device functions as ordinary ones, and fmaf rounds once on both
sides, so the host build performs the same operations as the device build.

Pins: every radix and both signs against numpy (relative L2 per vector within
FP32 rounding of a depth-log2(R) transform); the impulse at 0 maps to ones and
the constant to R at bin 0 exactly (every product then has a zero operand);
the sign convention (the tone e^{+2 pi i f n / R} lands in bin f under the
forward kernel, and its conjugate in bin f under the inverse kernel); every
derived power W^{jk} within a few FP32 ulps of the exact root (the products
are at most three deep), for every radix and many (k, table length).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2603_27569_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include "butterfly.cuh"
using namespace fftgb;

template <int R, int D>
static int run(long count) {
  for (long i = 0; i < count; ++i) {
    float2 a[R];
    if (fread(a, sizeof(float2), R, stdin) != (size_t)R) return 3;
    Dft<R, D>::run(a);
    fwrite(a, sizeof(float2), R, stdout);
  }
  return 0;
}

// Twiddle mode 1: the rows tw_loaded<R> names come in (FP32, rounded from
// the exact roots), derive_twiddles forms the others; all R - 1 go out.
template <int R>
static int derive(long count) {
  for (long i = 0; i < count; ++i) {
    float2 in[R], w[R];
    if (fread(in, sizeof(float2), R, stdin) != (size_t)R) return 3;
    for (int j = 0; j < R; ++j) w[j] = make_float2(0.f, 0.f);
    for (int j = 1; j < R; ++j)
      if (tw_loaded<R>(j)) w[j] = in[j];
    derive_twiddles<R>(w);
    fwrite(w + 1, sizeof(float2), R - 1, stdout);
  }
  return 0;
}

int main(int argc, char **argv) {
  if (argc != 4) return 2;
  const int R = atoi(argv[1]), D = atoi(argv[2]);
  const long count = atol(argv[3]);
#define CASE(r)                                                               \
  if (R == r) return D == 0 ? derive<r>(count) : D < 0 ? run<r, -1>(count) : run<r, 1>(count);
  CASE(2) CASE(4) CASE(8) CASE(16) CASE(32)
  return 2;
}
"""

RADICES = (2, 4, 8, 16, 32)


@pytest.fixture(scope="module")
def dft_host(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("butterfly_host")
    src, exe = d / "dft.cpp", d / "dft"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-O1", "-ffp-contract=off", "-w", f"-I{CUDA_INC}",
                    f"-I{CSRC}", str(src), "-o", str(exe)], check=True)

    def run(x, direction):
        """direction -1 / +1: DFT_R of each row; 0: derive_twiddles of each row."""
        x = np.ascontiguousarray(x, dtype=np.complex64)
        count, R = x.shape
        out = subprocess.run([str(exe), str(R), str(direction), str(count)],
                             input=x.tobytes(), capture_output=True, check=True).stdout
        return np.frombuffer(out, np.complex64).reshape(count, R if direction else R - 1)

    return run


@pytest.mark.parametrize("R", RADICES)
@pytest.mark.parametrize("direction", [-1, 1])
def test_dft_matches_numpy(dft_host, R, direction):
    rng = np.random.default_rng(R * 10 + (direction > 0))
    x = (rng.standard_normal((64, R)) + 1j * rng.standard_normal((64, R))).astype(np.complex64)
    y = dft_host(x, direction)
    xd = x.astype(np.complex128)
    ref = np.fft.fft(xd, axis=1) if direction < 0 else np.fft.ifft(xd, axis=1) * R
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-7 * np.log2(R) + 1e-7, err.max()


@pytest.mark.parametrize("R", RADICES)
def test_impulse_and_constant_are_exact(dft_host, R):
    for direction in (-1, 1):
        imp = np.zeros((1, R), np.complex64)
        imp[0, 0] = 1
        assert np.array_equal(dft_host(imp, direction), np.ones((1, R), np.complex64))
        const = np.ones((1, R), np.complex64)
        want = np.zeros((1, R), np.complex64)
        want[0, 0] = R
        assert np.array_equal(dft_host(const, direction), want)


@pytest.mark.parametrize("R", (8, 16, 32))
def test_sign_convention(dft_host, R):
    n = np.arange(R)
    for f in (1, 3, R // 2 - 1):
        tone = np.exp(2j * np.pi * f * n / R).astype(np.complex64)[None]
        fwd = dft_host(tone, -1)[0]       # sum_n e^{+2 pi i f n/R} e^{-2 pi i k n/R}: bin f
        inv = dft_host(tone.conj(), 1)[0]  # the conjugate tone under e^{+...}: bin f as well
        for y in (fwd, inv):
            assert np.argmax(np.abs(y)) == f
            assert abs(y[f] - R) <= 1e-5 * R
            assert np.max(np.abs(np.delete(y, f))) <= 1e-5 * R


@pytest.mark.parametrize("R", RADICES)
def test_twiddle_mode_1_derivation(dft_host, R):
    # Pass twiddles W_M^{j k}, j = 1..R-1, for table lengths M = p R and every k < p
    # of a few strides p (the Stockham pass tables), from the rows the kernel reads.
    rows = []
    for p in (1, 2, 16, 32, 512, 1024):
        M = p * R
        for k in range(p):
            j = np.arange(R)
            e = (j * k) % M                       # exact integer exponent
            rows.append(np.exp(-2j * np.pi * e / M))
    exact = np.array(rows)
    got = dft_host(exact.astype(np.complex64), 0)
    err = np.abs(got - exact[:, 1:])
    assert err.max() <= 4 * 2.0 ** -23, err.max()   # a few FP32 ulps of a unit root
