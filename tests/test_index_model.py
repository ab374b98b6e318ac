"""A NumPy model of the Stockham kernels' index algebra, for every compiled
single-CTA schedule (taken from the library's configuration list, no GPU).

The model restates what stockham.cuh does with indices (Sec. II-B, Stockham
autosort): thread lt holds points lt + m T (T = N / P) of pass 0; in pass s
(radix r, stride p = product of the earlier radices, Q = P / r butterflies per
thread) butterfly i = lt + q T (the paired last pass: i = 2 lt + q) takes
register q + j Q as its point j, multiplies it by W_{p r}^{j k} (k = i mod p),
runs DFT_r and writes output j to (i - k) r + k + j p of the exchange buffer
through the swizzle swz<p, r> (butterfly.cuh); the next pass reads point
lt + m T (or, paired, the 16-byte pair at 2 lt + j N / r), and the last pass
stores register m at its final index.  The DFTs and twiddles are numpy's, so
what is checked is the index algebra alone:

- the model's output equals numpy's FFT (forward) and N x its inverse FFT, for
  every schedule, with and without the paired last pass where it applies;
- every exchange layout is a permutation of the row, and a paired read's two
  points are adjacent and 16-byte aligned;
- every exchange access is free of shared-memory bank conflicts: the 16 lanes
  of a half-warp hit 16 distinct 8-byte bank pairs (8-byte accesses), the 8
  lanes of a quarter-warp 8 distinct 16-byte bank quads (paired reads).
"""
import numpy as np
import pytest

import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import build as fbuild

SIZES = (256, 512, 1024, 2048, 4096, 8192, 16384)


def ilog2(v):
    return int(v).bit_length() - 1


def swz(idx, p, r):
    """The exchange layout of a pass with stride p and radix r (butterfly.cuh)."""
    if p >= 16:
        return idx
    sh, mask, tsh = ilog2(p * r), 16 // p - 1, ilog2(p)
    return idx ^ (((idx >> sh) & mask) << tsh)


def max_ways(words, lanes_per_group):
    """Largest number of lanes of one access group on one bank group."""
    worst = 1
    for h in range(0, len(words) - lanes_per_group + 1, lanes_per_group):
        worst = max(worst, int(np.bincount(words[h:h + lanes_per_group] % lanes_per_group).max()))
    return worst


def stockham_model(x, P, radices, direction, paired, ways):
    N = len(x)
    T = N // P
    npass = len(radices)
    lt = np.arange(T)
    a = x[lt[:, None] + np.arange(P)[None, :] * T].astype(np.complex128)
    p = 1
    for s, r in enumerate(radices):
        Q = P // r
        last = s == npass - 1
        q = np.arange(Q)
        i = (2 * lt[:, None] + q[None, :]) if (paired and last) else (lt[:, None] + q[None, :] * T)
        k = i % p
        reg = q[:, None] + np.arange(r)[None, :] * Q
        v = a[:, reg] * np.exp(direction * 2j * np.pi * np.arange(r)[None, None, :]
                               * k[:, :, None] / (p * r))
        V = np.fft.fft(v, axis=2) if direction < 0 else np.fft.ifft(v, axis=2) * r
        a = np.empty_like(a)
        a[:, reg] = V
        if last:
            break
        phys = swz(((i - k) * r + k)[:, :, None] + np.arange(r)[None, None, :] * p, p, r)
        assert np.unique(phys).size == N, "exchange layout is not a permutation"
        buf = np.empty(N, np.complex128)
        buf[phys] = V
        for qq in range(Q):
            for j in range(r):
                ways.append(max_ways(phys[:, qq, j], 16))
        rn = radices[s + 1]
        if paired and s + 2 == npass:
            src = 2 * lt[:, None] + np.arange(P // 2)[None, :] * (N // rn)
            ph0, ph1 = swz(src, p, r), swz(src + 1, p, r)
            assert (ph0 % 2 == 0).all() and (ph1 == ph0 + 1).all(), "pair split or misaligned"
            a = np.empty((T, P), np.complex128)
            a[:, 0::2], a[:, 1::2] = buf[ph0], buf[ph1]
            for j in range(P // 2):
                ways.append(max_ways(ph0[:, j] // 2, 8))
        else:
            src = swz(lt[:, None] + np.arange(P)[None, :] * T, p, r)
            a = buf[src]
            for m in range(P):
                ways.append(max_ways(src[:, m], 16))
        p *= r
    r = radices[-1]
    Q = P // r
    y = np.empty(N, np.complex128)
    if paired:
        out = 2 * lt[:, None] + np.arange(P // 2)[None, :] * (N // r)
        y[out], y[out + 1] = a[:, 0::2], a[:, 1::2]
    else:
        m = np.arange(P)
        y[lt[:, None] + (m % Q)[None, :] * T + (m // Q)[None, :] * (N // r)] = a
    return y


def schedules():
    fbuild.build()
    out = []
    for N in SIZES:
        seen = set()
        for c in fg.fft_list_configs(N):
            if c["path"] != fg.FFT_PATH_SINGLE_CTA or c["cluster_split"]:
                continue
            key = (N, c["points_per_thread"], tuple(c["radix"]))
            if key not in seen:
                seen.add(key)
                out.append(key)
    return out


@pytest.mark.parametrize("N,P,radices", schedules())
def test_schedule_index_algebra(N, P, radices):
    assert int(np.prod(radices)) == N and all(P % r == 0 for r in radices)
    rng = np.random.default_rng(N + P)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = np.fft.fft(x)
    pairable = len(radices) >= 3 and P // radices[-1] == 2
    for paired in ((False, True) if pairable else (False,)):
        for direction in (-1, 1):
            ways = []
            y = stockham_model(x, P, list(radices), direction, paired, ways)
            want = X if direction < 0 else np.fft.ifft(x) * N
            assert np.abs(y - want).max() <= 1e-12 * np.abs(X).max()
            assert max(ways) == 1, f"{max(ways)}-way bank conflict"
