"""Pins against numbers the paper prints (tests/golden/paper_numbers.json,
each entry with its citation): the DFT definition and the DFT_8 matrix, the
GFLOPS convention with its worked value, the stage counts of the radix table
and the single-buffer size rule applied to GB300."""
import json
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))


@pytest.fixture(scope="module", autouse=True)
def _oracle_built():
    oracle.build()


def test_dft8_matrix_entries_are_w8_powers():
    # F_8[j, k] = W_8^{jk}: the oracle applied to the unit vector e_k is column
    # k; W_8 is the printed (cos, -sin)(pi/4), powers formed exactly by octant.
    g = G["dft_definition"]
    w8 = complex(*g["W8_real_imag"])
    s = math.sqrt(0.5)
    exact = [1, complex(s, -s), -1j, complex(-s, -s), -1, complex(-s, s), 1j, complex(s, s)]
    assert abs(exact[1] - w8) < 1e-16
    F = np.array([[exact[(j * k) % 8] for k in range(8)] for j in range(8)])
    for k in range(8):
        e = np.zeros(8, np.complex128)
        e[k] = 1
        col = oracle.dft(e)
        assert np.max(np.abs(col - F[:, k])) < 1e-15
        assert np.max(np.abs(oracle.fft(e) - F[:, k])) < 1e-15


def test_gflops_convention_reproduces_the_printed_value():
    import bench

    g = G["gflops_convention"]
    half_ulp = 0.5 * 10 ** (-g["us_per_fft_digits"])
    lo = bench.flops(g["N"], 1) / ((g["us_per_fft"] + half_ulp) * 1e-6) / 1e9
    hi = bench.flops(g["N"], 1) / ((g["us_per_fft"] - half_ulp) * 1e-6) / 1e9
    assert bench.flops(g["N"], 1) == 5 * 4096 * 12
    assert lo <= g["gflops"] <= hi
    assert bench.flops(g["N"], g["batch"]) == g["batch"] * bench.flops(g["N"], 1)


def test_stage_counts_of_the_radix_table():
    import paper_2603_27569_gb300 as fg

    g = G["stages_n4096"]
    N = g["N"]
    for r, stages in g["stages_by_radix"].items():
        assert math.ceil(math.log(N, int(r)) - 1e-12) == stages
    cfgs = [c for c in fg.fft_list_configs(N) if c["path"] == fg.FFT_PATH_SINGLE_CTA]
    for r in (8, 16):
        pure = [c for c in cfgs if set(c["radix"]) == {r}]
        assert pure, f"no pure radix-{r} schedule for N = {N}"
        assert all(c["num_passes"] == g["stages_by_radix"][str(r)] for c in pure)


def test_single_buffer_rule_on_gb300():
    import paper_2603_27569_gb300 as fg

    g = G["bmax"]
    assert g["buffer_bytes"] // g["element_bytes"] == g["B_max"]
    gb300_cta_bytes = 227 * 1024            # opt-in shared memory per CTA
    b = gb300_cta_bytes // g["element_bytes"]
    b_pow2 = 1 << (b.bit_length() - 1)
    assert b_pow2 == 16384
    # one CTA holding the whole row (cluster configurations spread it over K CTAs)
    single = lambda N: any(c["path"] == fg.FFT_PATH_SINGLE_CTA and not c["cluster_split"]
                           for c in fg.fft_list_configs(N))
    assert single(b_pow2) and not single(2 * b_pow2)


def test_sar_estimate_fixture_is_consistent():
    g = G["sar_batch_estimate"]
    assert round(g["lines"] * g["us_per_fft"]) == g["total_us"]
