"""FP64 CPU oracle for the batched C2C FFT and the spectral-filter layer.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the product path
(``paper_2603_27569_gb300``) never does and shares no code with it.

Contents
  build()              compile ``fft_oracle.c`` with gcc into ``_build/``.
  dft(x, inverse)      the DFT definition, O(N^2)  (paper Sec. II-A).
  fft(x, inverse)      recursive radix-2 DIT FFT in FP64 (Eq. 1 with N1 = 2).
  spectral_filter_*    y = IFFT(FFT(x) * H), loss = sum m |y|^2, and its
                       analytic gradient written from the chain rule.

Conventions: the forward transform is unnormalised with W_N = exp(-2 pi i/N)
(Sec. II-A); the inverse is scaled by 1/N (the paper leaves it undefined; this
reading makes inverse(forward(x)) = x).  Arrays are complex with the transform
along the last axis; results are complex128.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain C99 + libm + pthreads) and return its path."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        i64 = ctypes.c_int64
        for name in ("oracle_dft", "oracle_fft"):
            f = getattr(lib, name)
            f.argtypes = [i64, dp, dp, ctypes.c_int]
            f.restype = ctypes.c_int
        lib.oracle_fft_batch.argtypes = [i64, i64, dp, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_fft_batch.restype = ctypes.c_int
        lib.oracle_fft_batch_f32.argtypes = [i64, i64, fp, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_fft_batch_f32.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def dft(x, inverse: bool = False) -> np.ndarray:
    """Naive O(N^2) DFT of each row (the definition of Sec. II-A)."""
    lib = _load()
    x = _as_c128(x)
    shape = x.shape
    N = shape[-1]
    rows = x.reshape(-1, N)
    out = np.empty_like(rows)
    d = 1 if inverse else -1
    for r in range(rows.shape[0]):
        src = np.ascontiguousarray(rows[r])
        dst = out[r]
        if lib.oracle_dft(N, _dptr(src), _dptr(dst), d) != 0:
            raise ValueError(f"oracle_dft rejected N={N}")
    return out.reshape(shape)


def fft(x, inverse: bool = False, nthreads: int = 1) -> np.ndarray:
    """Recursive radix-2 FP64 FFT of each row; N must be a power of two.

    complex64 input is widened exactly to FP64 inside the C code.
    """
    lib = _load()
    x = np.asarray(x)
    shape = x.shape
    N = shape[-1]
    d = 1 if inverse else -1
    if x.dtype == np.complex64:
        src = np.ascontiguousarray(x).reshape(-1, N)
        out = np.empty(src.shape, dtype=np.complex128)
        rc = lib.oracle_fft_batch_f32(
            N, src.shape[0],
            src.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
            _dptr(out), d, nthreads)
    else:
        src = _as_c128(x).reshape(-1, N)
        out = np.empty_like(src)
        rc = lib.oracle_fft_batch(N, src.shape[0], _dptr(src), _dptr(out), d, nthreads)
    if rc != 0:
        raise ValueError(f"oracle_fft rejected N={N}")
    return out.reshape(shape)


def ifft(x, nthreads: int = 1) -> np.ndarray:
    return fft(x, inverse=True, nthreads=nthreads)


# --------------------------------------------------------------------------
# Spectral filter (SAR range compression), paper Sec. II-D / IX-A context.
#   z = FFT(x) * H      (H broadcast over rows)
#   y = IFFT(z)
#   L = sum m * |y|^2   (m real, same shape as y)
# Gradients use the convention grad(z) = dL/dRe z + i dL/dIm z.
# With G = IFFT = (1/N) F^H:  G^H = (1/N) F  and  F^H = N G.
#   g_y    = 2 m y
#   g_z    = G^H g_y = (1/N) FFT(g_y)
#   grad_H = sum_rows conj(FFT(x)) * g_z
#   grad_x = F^H (conj(H) * g_z) = N * IFFT(conj(H) * g_z)
# --------------------------------------------------------------------------
# nthreads only spreads rows over threads; the arithmetic is the same.
def spectral_filter_forward(x, H, nthreads: int = 1):
    X = fft(x, nthreads=nthreads)
    z = X * _as_c128(H)
    return ifft(z, nthreads=nthreads)


def spectral_filter_loss(x, H, m, nthreads: int = 1) -> float:
    y = spectral_filter_forward(x, H, nthreads=nthreads)
    return float(np.sum(np.asarray(m, dtype=np.float64) * (y.real ** 2 + y.imag ** 2)))


def spectral_filter_grads(x, H, m, nthreads: int = 1):
    x = _as_c128(x)
    H = _as_c128(H)
    m = np.asarray(m, dtype=np.float64)
    N = x.shape[-1]
    X = fft(x, nthreads=nthreads)
    y = ifft(X * H, nthreads=nthreads)
    g_y = 2.0 * m * y
    g_z = fft(g_y, nthreads=nthreads) / N
    grad_H = np.sum(np.conj(X) * g_z, axis=tuple(range(x.ndim - 1)))
    grad_x = N * ifft(np.conj(H) * g_z, nthreads=nthreads)
    return grad_x, grad_H
