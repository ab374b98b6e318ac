"""A NumPy model of the cluster-split kernel's index algebra (cluster.cuh),
for every compiled cluster configuration, no GPU.

The four-step split with N1 = K (Sec. IV-B, Eq. 3): n = r + K n2,
k = k2 + H k1, H = N / K.  The model restates the kernel's indices:

- scatter (K >= 4 path): CTA r reads its contiguous slice x[r H .. (r+1) H)
  as pairs j = lt + m T (T = H / P threads) and sends elements e = r H + 2 j
  and e + 1 to CTA e mod K at position e div K, computed as q0 = (2 lt) mod K,
  base = r H / K + (2 lt) div K, position base + m (2 T / K);
- every CTA then holds its stride-K subsequence x[r + K n2] in natural order
  (the K = 2 path loads exactly that subsequence directly);
- A_r = FFT_H of it, B_r[k2] = A_r[k2] W_N^{r k2} (table laid out [r-1][k2]);
- CTA r combines k2 = r H / K + lt + u T (u < P / K) with a K-point DFT over
  the CTAs and stores X[k2 + H k1].

Checked: every scatter target in bounds and written exactly once, each CTA's
buffer equal to its subsequence, every output written exactly once, and the
result equal to numpy's FFT (forward) and N x its inverse FFT.
"""
import numpy as np
import pytest

import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import build as fbuild


def cluster_configs():
    fbuild.build()
    out = set()
    for N in (8192, 16384, 32768, 65536, 131072):
        for c in fg.fft_list_configs(N):
            if c["cluster_split"]:
                out.add((N, c["cluster_split"], c["points_per_thread"]))
    return sorted(out)


def split_model(x, K, P, direction):
    N = len(x)
    H = N // K
    T = H // P
    assert H % K == 0 and P % K == 0 and (2 * T) % K == 0
    f = np.fft.fft if direction < 0 else (lambda v: np.fft.ifft(v) * len(v))
    smem = np.full((K, H), np.nan, np.complex128)
    hits = np.zeros((K, H), int)
    for r in range(K):
        for lt in range(T):
            q0 = (2 * lt) % K
            base = r * (H // K) + (2 * lt) // K
            for m in range(P // 2):
                pos = base + m * (2 * T // K)
                assert 0 <= pos < H
                e = r * H + 2 * (lt + m * T)
                for s, q in ((0, q0), (1, q0 + 1)):
                    assert (e + s) % K == q and (e + s) // K == pos
                    smem[q, pos] = x[e + s]
                    hits[q, pos] += 1
    assert (hits == 1).all(), "scatter target written twice or never"
    for r in range(K):
        assert np.array_equal(smem[r], x[r::K])
    A = np.array([f(smem[r]) for r in range(K)])
    tw = np.exp(direction * 2j * np.pi * np.outer(np.arange(1, K), np.arange(H)) / N)
    B = A.copy()
    B[1:] *= tw
    out = np.full(N, np.nan, np.complex128)
    hits = np.zeros(N, int)
    for r in range(K):
        for lt in range(T):
            for u in range(P // K):
                k2 = r * (H // K) + lt + u * T
                b = f(B[:, k2])
                for k1 in range(K):
                    out[k2 + k1 * H] = b[k1]
                    hits[k2 + k1 * H] += 1
    assert (hits == 1).all(), "output written twice or never"
    return out


@pytest.mark.parametrize("N,K,P", cluster_configs())
def test_cluster_split_index_algebra(N, K, P):
    rng = np.random.default_rng(N + K)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = np.fft.fft(x)
    for direction in (-1, 1):
        want = X if direction < 0 else np.fft.ifft(x) * N
        y = split_model(x, K, P, direction)
        assert np.abs(y - want).max() <= 1e-12 * np.abs(X).max()
