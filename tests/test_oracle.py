"""Pins for the FP64 oracle against facts fixed by the mathematics.

The DFT definition (paper Sec. II-A): X[k] = sum_n x[n] W_N^{nk}, W_N = e^{-2 pi i/N},
forward unnormalised; the inverse is read as (1/N) times the conjugate-sign sum.
Every check below holds independently of any FFT implementation: closed forms,
invariants of the DFT, brute force on tiny inputs and an independent library.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_27569_gb300 import synth

POW2_SMALL = [1, 2, 4, 8, 16, 32, 64]
POW2_LARGE = [128, 256, 1024, 4096, 16384]


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# --------------------------------------------------------------------------
# Closed forms of the definition (these also pin oracle.dft itself)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("impl", ["dft", "fft"])
def test_textbook_n4(impl):
    # X[k] = sum_{n<4} x[n] (-i)^{nk} for x = [1, 2, 3, 4]
    f = getattr(oracle, impl)
    X = f(np.array([1, 2, 3, 4], dtype=np.complex128))
    np.testing.assert_allclose(X, [10, -2 + 2j, -2, -2 - 2j], atol=1e-13)


@pytest.mark.parametrize("impl", ["dft", "fft"])
def test_textbook_n8_box(impl):
    # x = [1,1,1,1,0,0,0,0]: geometric sum (1 - W^{4k}) / (1 - W^k), W = e^{-i pi/4}
    f = getattr(oracle, impl)
    X = f(np.array([1, 1, 1, 1, 0, 0, 0, 0], dtype=np.complex128))
    r2 = math.sqrt(2.0)
    want = [4, 1 - (1 + r2) * 1j, 0, 1 - (r2 - 1) * 1j, 0, 1 + (r2 - 1) * 1j, 0,
            1 + (1 + r2) * 1j]
    np.testing.assert_allclose(X, want, atol=1e-13)


@pytest.mark.parametrize("impl", ["dft", "fft"])
@pytest.mark.parametrize("N", [2, 8, 64, 1024])
def test_impulse_and_constant(impl, N):
    if impl == "dft" and N > 64:
        pytest.skip("naive DFT only on small N")
    f = getattr(oracle, impl)
    d = np.zeros(N, np.complex128)
    d[0] = 1
    np.testing.assert_allclose(f(d), np.ones(N), atol=1e-12)           # delta -> ones
    c = np.ones(N, np.complex128)
    want = np.zeros(N, np.complex128)
    want[0] = N
    np.testing.assert_allclose(f(c), want, atol=1e-9 * N)               # ones -> N delta
    # inverse: ones -> delta (1/N scaling), delta -> 1/N
    np.testing.assert_allclose(f(c, inverse=True), d, atol=1e-12)
    np.testing.assert_allclose(f(d, inverse=True), np.full(N, 1.0 / N), atol=1e-15)


@pytest.mark.parametrize("impl", ["dft", "fft"])
@pytest.mark.parametrize("N,freq", [(8, 1), (16, 3), (64, 17), (4096, 1234), (16384, 16383)])
def test_pure_tone(impl, N, freq):
    # x[n] = e^{+2 pi i f n / N}  ->  X[k] = N delta[k - f]  (sign convention check)
    if impl == "dft" and N > 64:
        pytest.skip("naive DFT only on small N")
    f = getattr(oracle, impl)
    n = np.arange(N)
    x = np.exp(2j * np.pi * ((freq * n) % N) / N)
    X = f(x)
    want = np.zeros(N, np.complex128)
    want[freq] = N
    assert np.max(np.abs(X - want)) <= 1e-10 * N
    # a shifted index or a flipped sign would put the peak at -f
    assert abs(X[(-freq) % N]) < 1e-6 or freq == (-freq) % N


# --------------------------------------------------------------------------
# Brute force: the recursive FFT equals the definition on small N
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", POW2_SMALL + [128, 256])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft_matches_naive_dft(N, inverse):
    x = synth.gaussian((3, N), seed=N).astype(np.complex128)
    got = oracle.fft(x, inverse=inverse)
    want = oracle.dft(x, inverse=inverse)
    l1 = np.sum(np.abs(x), axis=1, keepdims=True)
    scale = l1 / (N if inverse else 1)
    assert np.all(np.abs(got - want) <= 1e-12 * np.maximum(scale, 1e-300))


def test_naive_dft_matches_matrix_product():
    # the definition as an explicit matrix, built here from W_N^{nk} with exact (nk mod N)
    N = 12  # the naive DFT is not restricted to powers of two
    x = synth.gaussian(N, seed=5).astype(np.complex128)
    n = np.arange(N)
    F = np.exp(-2j * np.pi * (np.outer(n, n) % N) / N)
    np.testing.assert_allclose(oracle.dft(x), F @ x, atol=1e-12)
    np.testing.assert_allclose(oracle.dft(x, inverse=True), np.conj(F) @ x / N, atol=1e-13)


# --------------------------------------------------------------------------
# Invariants (any N, including the sizes the GPU path covers)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", POW2_LARGE)
def test_linearity(N):
    x = synth.gaussian(N, seed=1).astype(np.complex128)
    y = synth.uniform(N, seed=2).astype(np.complex128)
    a, b = 0.75 - 1.25j, -2.0 + 0.5j
    lhs = oracle.fft(a * x + b * y)
    rhs = a * oracle.fft(x) + b * oracle.fft(y)
    assert rel_l2(lhs, rhs) < 1e-13


@pytest.mark.parametrize("N,m", [(256, 1), (1024, 37), (16384, 5000)])
def test_shift_theorem(N, m):
    # x[n - m] <-> X[k] W_N^{k m}
    x = synth.gaussian(N, seed=3).astype(np.complex128)
    X = oracle.fft(x)
    k = np.arange(N)
    want = X * np.exp(-2j * np.pi * ((k * m) % N) / N)
    assert rel_l2(oracle.fft(np.roll(x, m)), want) < 1e-12


@pytest.mark.parametrize("N", POW2_LARGE)
def test_parseval(N):
    x = synth.gaussian(N, seed=4).astype(np.complex128)
    X = oracle.fft(x)
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(X) ** 2) / N) <= 1e-12 * np.sum(np.abs(x) ** 2)


@pytest.mark.parametrize("N", POW2_LARGE)
def test_hermitian_symmetry_of_real_input(N):
    x = synth.gaussian(N, seed=6).real.astype(np.complex128)
    X = oracle.fft(x)
    k = np.arange(N)
    assert rel_l2(X[(-k) % N], np.conj(X)) < 1e-13


@pytest.mark.parametrize("N", POW2_LARGE)
def test_round_trip(N):
    x = synth.gaussian((2, N), seed=7).astype(np.complex128)
    assert rel_l2(oracle.ifft(oracle.fft(x)), x) < 1e-14


@pytest.mark.parametrize("N", [2, 64, 1024, 16384])
def test_adjoint_dot_product(N):
    # <F x, y> = <x, F^H y> with F^H = N * inverse
    x = synth.gaussian(N, seed=8).astype(np.complex128)
    y = synth.gaussian(N, seed=9).astype(np.complex128)
    lhs = np.vdot(y, oracle.fft(x))
    rhs = np.vdot(N * oracle.ifft(y), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-9


@pytest.mark.parametrize("N", [1, 2, 4, 256, 4096, 16384])
def test_agrees_with_numpy_fft(N):
    # an independent library implementation (not the oracle, only a cross-check)
    x = synth.gaussian((2, N), seed=10).astype(np.complex128)
    assert rel_l2(oracle.fft(x), np.fft.fft(x)) < 1e-13
    assert rel_l2(oracle.fft(x, inverse=True), np.fft.ifft(x)) < 1e-13


def test_complex64_input_is_widened_exactly():
    x = synth.gaussian((3, 512), seed=11)
    a = oracle.fft(x)                          # float32 path inside the C code
    b = oracle.fft(x.astype(np.complex128))    # double path
    assert np.array_equal(a, b)


def test_batch_threads_do_not_change_results():
    x = synth.gaussian((37, 256), seed=12).astype(np.complex128)
    assert np.array_equal(oracle.fft(x, nthreads=1), oracle.fft(x, nthreads=5))


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12, np.complex128))


# --------------------------------------------------------------------------
# Spectral filter: analytic gradient against FP64 central differences.
# --------------------------------------------------------------------------
def _sar_slice(rows=4, N=256, seed=0):
    x, pulse = synth.sar_echoes(rows, N, Np=64, seed=seed)
    H = np.conj(oracle.fft(pulse))
    m = synth.real_mask((rows, N), seed=2)
    return x.astype(np.complex128), H, m.astype(np.float64)


def test_spectral_filter_grad_H_central_differences():
    x, H, m = _sar_slice()
    gx, gH = oracle.spectral_filter_grads(x, H, m)
    h = 1e-6
    N = H.shape[0]
    fd = np.zeros(N, np.complex128)
    for j in range(N):
        for part, unit in ((0, 1.0), (1, 1j)):
            Hp = H.copy()
            Hm = H.copy()
            Hp[j] += h * unit
            Hm[j] -= h * unit
            d = (oracle.spectral_filter_loss(x, Hp, m) - oracle.spectral_filter_loss(x, Hm, m)) / (2 * h)
            if part == 0:
                fd[j] += d
            else:
                fd[j] += 1j * d
    assert rel_l2(gH, fd) < 1e-5


def test_spectral_filter_grad_x_central_differences():
    x, H, m = _sar_slice(seed=3)
    gx, _ = oracle.spectral_filter_grads(x, H, m)
    rng = np.random.Generator(np.random.PCG64(42))
    idx = rng.choice(x.size, size=64, replace=False)
    h = 1e-6
    flat = x.reshape(-1)
    got, want = [], []
    for q in idx:
        for unit in (1.0, 1j):
            xp = flat.copy()
            xm = flat.copy()
            xp[q] += h * unit
            xm[q] -= h * unit
            d = (oracle.spectral_filter_loss(xp.reshape(x.shape), H, m)
                 - oracle.spectral_filter_loss(xm.reshape(x.shape), H, m)) / (2 * h)
            want.append(d)
            g = gx.reshape(-1)[q]
            got.append(g.real if unit == 1.0 else g.imag)
    got = np.array(got)
    want = np.array(want)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5
