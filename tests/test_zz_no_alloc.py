"""The allocation-free four-step entry point (fft_fourstep_noalloc).

Some users of this library cannot allocate device memory while they run
(memory fixed at start-up, or the device heap owned by their own allocator),
so they cannot make a plan.  fft_fourstep_noalloc serves them from a fixed
device scratch array.  This file checks, through the C ABI, that two calls
in a row give the same results as the regular four-step plan (within the FP32
tolerance of the other tests), and that sizes beyond the fixed scratch are
refused.  It is named to be collected last and passes both alone in a fresh
process (where its first call performs the per-device set-up) and after the
other tests.
"""
import ctypes

import numpy as np
import pytest

import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INVALID_SIZE = 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


def regular_fourstep(x, direction):
    N = x.shape[-1]
    plan = fg.Plan(N, x.shape[0], direction, flags=fg.FFT_FLAG_FORCE_FOURSTEP)
    y = to_host(plan(to_dev(x)))
    plan.close()
    return y


def noalloc(x, direction):
    N = x.shape[-1]
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    rc = fg.lib().fft_fourstep_noalloc(xd.data_ptr(), yd.data_ptr(), N, x.shape[0], direction,
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == 0, fg.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return to_host(yd)


def test_two_calls_in_a_row_match_the_regular_entry_point():
    cases = [(16384, 96, fg.FFT_FORWARD, 1), (4096, 300, fg.FFT_INVERSE, 2)]
    for N, batch, direction, seed in cases:
        x = synth.gaussian((batch, N), seed=seed)
        got = noalloc(x, direction)
        want = regular_fourstep(x, direction)
        assert rel_l2_rows(got, want).max() <= TOL_FP32


def test_maximum_size_and_refusal_beyond_it():
    N = 8192
    batch = fg.FFT_NOALLOC_MAX_POINTS // N
    x = synth.gaussian((batch, N), seed=3)
    got = noalloc(x, fg.FFT_FORWARD)
    want = regular_fourstep(x, fg.FFT_FORWARD)
    assert rel_l2_rows(got, want).max() <= TOL_FP32
    buf = torch.empty(N * (batch + 1), dtype=torch.complex64, device="cuda")
    rc = fg.lib().fft_fourstep_noalloc(buf.data_ptr(), buf.data_ptr(), N, batch + 1,
                                       fg.FFT_FORWARD, None)
    assert rc == INVALID_SIZE
