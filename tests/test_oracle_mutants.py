"""Planted mistakes: each mutant of the C oracle must fail at least one pin.

Every mutation is a plausible slip (a flipped sign, an off-by-one twiddle
index, a dropped normalisation, a transposed re/im operand, a wrong stride).
The mutant is compiled on the CPU into a temporary directory and run through a
small battery of the same facts the main pin file checks: the textbook N=4 DFT,
the pure tone, the definition as an explicit matrix, FFT = naive DFT, and the
inverse round trip.  The unmutated source must pass the battery.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "fft_oracle.c")

MUTANTS = {
    "angle_sign": ("double theta = (double)sign * kTwoPi",
                   "double theta = -(double)sign * kTwoPi"),
    "butterfly_sign": ("y[2 * (k + h)] = er - tr;", "y[2 * (k + h)] = er + tr;"),
    "twiddle_index": ("unit_root(N, k, sign, &wr, &wi);", "unit_root(N, k + 1, sign, &wr, &wi);"),
    "cmul_sign": ("double tr = wr * orr - wi * oi;", "double tr = wr * orr + wi * oi;"),
    "leaf_transposed": ("y[0] = x[0];\n        y[1] = x[1];", "y[0] = x[1];\n        y[1] = x[0];"),
    "odd_stride": ("fft_rec(h, x + 2 * stride, 2 * stride", "fft_rec(h, x + 4 * stride, 2 * stride"),
    "fft_no_inverse_scale": ("fft_rec(N, x, 1, tmp, direction);\n    double s = (direction == 1) ? 1.0 / (double)N : 1.0;",
                             "fft_rec(N, x, 1, tmp, direction);\n    double s = 1.0;"),
    "dft_exponent": ("(__int128)n * (__int128)k) % N", "(__int128)n * (__int128)(k + 1)) % N"),
    "dft_accum_sign": ("si += xr * wi + xi * wr;", "si += xr * wi - xi * wr;"),
}


def _compile(src_text: str, tmp_path, tag: str):
    c = tmp_path / f"{tag}.c"
    so = tmp_path / f"lib{tag}.so"
    c.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-std=gnu99", "-fPIC", "-shared", str(c), "-o", str(so),
                    "-lm", "-lpthread"], check=True)
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    for name in ("oracle_dft", "oracle_fft"):
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int]
        f.restype = ctypes.c_int
    return lib


def _call(lib, name, x, inverse=False):
    x = np.ascontiguousarray(x, np.complex128)
    y = np.empty_like(x)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = getattr(lib, name)(x.shape[0], x.ctypes.data_as(dp), y.ctypes.data_as(dp),
                            1 if inverse else -1)
    assert rc == 0
    return y


def _battery(lib):
    """Return the list of failed checks (empty if the library passes)."""
    failed = []
    rng = np.random.Generator(np.random.PCG64(0))
    # textbook N=4
    for name in ("oracle_dft", "oracle_fft"):
        X = _call(lib, name, np.array([1, 2, 3, 4], np.complex128))
        if not np.allclose(X, [10, -2 + 2j, -2, -2 - 2j], atol=1e-12):
            failed.append(f"textbook:{name}")
    # pure tone, N=16, f=3
    n = np.arange(16)
    tone = np.exp(2j * np.pi * ((3 * n) % 16) / 16)
    want = np.zeros(16, np.complex128)
    want[3] = 16
    for name in ("oracle_dft", "oracle_fft"):
        if not np.allclose(_call(lib, name, tone), want, atol=1e-10):
            failed.append(f"tone:{name}")
    # the definition as a matrix (N = 8)
    x8 = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    k = np.arange(8)
    F = np.exp(-2j * np.pi * (np.outer(k, k) % 8) / 8)
    if not np.allclose(_call(lib, "oracle_dft", x8), F @ x8, atol=1e-12):
        failed.append("matrix:forward")
    if not np.allclose(_call(lib, "oracle_dft", x8, True), np.conj(F) @ x8 / 8, atol=1e-12):
        failed.append("matrix:inverse")
    # FFT equals the naive DFT, both directions, N = 32
    x = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    for inv in (False, True):
        if not np.allclose(_call(lib, "oracle_fft", x, inv), _call(lib, "oracle_dft", x, inv), atol=1e-11):
            failed.append(f"fft_vs_dft:{inv}")
    # round trip
    if not np.allclose(_call(lib, "oracle_fft", _call(lib, "oracle_fft", x), True), x, atol=1e-12):
        failed.append("round_trip")
    return failed


def test_unmutated_oracle_passes_battery(tmp_path):
    src = open(ORACLE_SRC).read()
    assert _battery(_compile(src, tmp_path, "clean")) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(ORACLE_SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique in the oracle"
    lib = _compile(src.replace(old, new), tmp_path, name)
    assert _battery(lib), f"mutant {name} survived every pin"
