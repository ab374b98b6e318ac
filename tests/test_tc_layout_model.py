"""A model of the tensor-core kernel's exchange stores (tc.cu, tc_exchange),
with the per-size constants read from the TcCfg definitions in tc.cu, no GPU.

After tensor-core stage s (stride p = 16^s) the thread owning TMEM row m
holds butterfly v = unrow_s(m) (b = its transform in the CTA, i = its index,
k = i mod p, u = i div p); its output j lands at position base + j p with
base = 16 p u + k, i.e. in operand row row_{s+1}(b, base mod NB) at K point
j2 = base div NB, and the row of j p is added as a compile-time constant.
Each output is one 4-byte store (16-bit real and imaginary parts) into the
hi and into the lo plane of the K-major operand layout: rows in core matrices
of 8 rows x 16 bytes, K-adjacent core matrices LBO bytes apart, 8-row groups
SBO bytes apart.

Checked: every row code is a permutation; the stores of one stage hit every
position of the plane exactly once and stay inside it; and the bank ways of a
warp's store (32 consecutive TMEM rows, one j) are 1 (conflict-free) except
at N = 4096's second exchange, whose unpadded layout (LBO 128 / SBO 512, for a
sixth resident CTA per SM) makes it 2-way.
"""
import os
import re

import numpy as np
import pytest

TC_CU = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_2603_27569_gb300", "csrc", "tc.cu")
EXPECTED_WAYS = {(4096, 1): 2}


def tc_configs():
    text = open(TC_CU).read()
    out = {}
    for N, body in re.findall(r"struct TcCfg<(\d+)>\s*\{(.*?)\};", text, flags=re.S):
        ints = dict((k, int(v)) for k, v in re.findall(r"\b([A-Z][A-Z0-9]*) = (\d+)\b", body))
        codes = dict((k, int(v, 16)) for k, v in re.findall(r"\b(R[0-2]) = (0x[0-9a-fA-F]+)ull", body))
        codes.update((k, 0) for k in re.findall(r"\b(R[0-2]) = 0\b", body))
        out[int(N)] = dict(ints, R=[codes["R0"], codes["R1"], codes["R2"]])
    return out


def ilog2(v):
    return int(v).bit_length() - 1


def tc_row(R, nbits, v):
    return sum((((v >> ((R >> (4 * b)) & 15)) & 1) << b) for b in range(nbits))


def tc_unrow(R, nbits, m):
    return sum((((m >> b) & 1) << ((R >> (4 * b)) & 15)) for b in range(nbits))


def rowoff(SBO, m):
    return (m >> 3) * SBO + (m & 7) * 16


CFG = tc_configs()


def test_every_size_is_described():
    assert sorted(CFG) == [256, 4096, 16384]
    for c in CFG.values():
        assert {"S", "TB", "NW", "LBO", "SBO"} <= set(c)


@pytest.mark.parametrize("N", sorted(CFG))
def test_exchange_stores(N):
    c = CFG[N]
    NB = N // 16
    IB = ilog2(NB)
    nbits = ilog2(c["TB"] * NB)
    rows = c["TB"] * NB
    plane = (rows // 8) * c["SBO"]
    for s in range(c["S"]):
        if c["R"][s] or s == 0:
            assert sorted(tc_row(c["R"][s], nbits, v) for v in range(rows)) == list(range(rows))
    for s in range(c["S"] - 1):
        p, LP = 16 ** s, 4 * s
        RS, RN = c["R"][s], c["R"][s + 1]
        addrs = np.empty((rows, 16), np.int64)
        for m in range(rows):
            v = tc_unrow(RS, nbits, m)
            b, i = v >> IB, v & (NB - 1)
            k, u = i & (p - 1), i >> LP
            base = (u << (LP + 4)) | k
            j2 = base >> IB
            m2 = tc_row(RN, nbits, (b << IB) | (base & (NB - 1)))
            off = rowoff(c["SBO"], m2) + (j2 >> 2) * c["LBO"] + (j2 & 3) * 4
            for j in range(16):
                addrs[m, j] = off + rowoff(c["SBO"], tc_row(RN, nbits, j * p))
        assert addrs.min() >= 0 and addrs.max() + 4 <= plane
        assert np.unique(addrs).size == rows * 16, "two outputs share a store address"
        worst = 1
        for g in range(rows // 32):
            for j in range(16):
                worst = max(worst, int(np.bincount((addrs[32 * g:32 * g + 32, j] // 4) % 32).max()))
        assert worst == EXPECTED_WAYS.get((N, s), 1), f"stage {s}: {worst}-way"
