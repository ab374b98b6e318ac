"""The allocation-free four-step entry point (fft_fourstep_noalloc).

Some users of this library cannot allocate device memory while they run
(memory fixed at start-up, or the device heap owned by their own allocator),
so they cannot make a plan.  fft_fourstep_noalloc serves them from a fixed
device scratch array.  This file checks, through the C ABI:
  - two calls in a row against the FP64 oracle (per-row relative L2 within
    the FP32 tolerance) and bit for bit against the regular four-step plan,
    which runs the same kernels on the same twiddle tables;
  - an in-place call and a call on a non-default stream;
  - the largest batch the scratch holds, and the refusal of a larger one;
  - the first call of a fresh process (which performs the per-device set-up)
    in a child process, whatever order the tests run in.
It is named to be collected last and passes both alone in a fresh process
and after the other tests.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INVALID_SIZE = 1
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def noalloc_dev(xd, yd, N, batch, direction, stream):
    rc = fg.lib().fft_fourstep_noalloc(xd.data_ptr(), yd.data_ptr(), N, batch, direction,
                                       stream.cuda_stream)
    assert rc == 0, fg.STATUS.get(rc, rc)


def noalloc(x, direction):
    N = x.shape[-1]
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    noalloc_dev(xd, yd, N, x.shape[0], direction, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return to_host(yd)


def test_two_calls_in_a_row_match_the_oracle_and_the_regular_entry_point():
    cases = [(16384, 96, fg.FFT_FORWARD, 1), (4096, 300, fg.FFT_INVERSE, 2)]
    for N, batch, direction, seed in cases:
        x = synth.gaussian((batch, N), seed=seed)
        got = noalloc(x, direction)
        want = oracle.fft(x, inverse=direction == fg.FFT_INVERSE, nthreads=NTHREADS)
        assert rel_l2_rows(got, want).max() <= TOL_FP32
        assert np.array_equal(got, regular_fourstep(x, direction))


def test_in_place_and_on_a_non_default_stream():
    N, batch = 2048, 200
    x = synth.gaussian((batch, N), seed=4)
    want = oracle.fft(x, nthreads=NTHREADS)
    side = torch.cuda.Stream()
    xd = to_dev(x)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        noalloc_dev(xd, xd, N, batch, fg.FFT_FORWARD, side)  # in == out
    side.synchronize()
    got = to_host(xd)
    assert rel_l2_rows(got, want).max() <= TOL_FP32
    assert np.array_equal(got, regular_fourstep(x, fg.FFT_FORWARD))


def test_maximum_size_and_refusal_beyond_it():
    N = 8192
    batch = fg.FFT_NOALLOC_MAX_POINTS // N
    x = synth.gaussian((batch, N), seed=3)
    got = noalloc(x, fg.FFT_FORWARD)
    rows = np.random.default_rng(5).choice(batch, 16, replace=False)
    want = oracle.fft(x[rows], nthreads=NTHREADS)
    assert rel_l2_rows(got[rows], want).max() <= TOL_FP32
    assert np.array_equal(got, regular_fourstep(x, fg.FFT_FORWARD))
    buf = torch.empty(N * (batch + 1), dtype=torch.complex64, device="cuda")
    rc = fg.lib().fft_fourstep_noalloc(buf.data_ptr(), buf.data_ptr(), N, batch + 1,
                                       fg.FFT_FORWARD, None)
    assert rc == INVALID_SIZE


CHILD = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np, torch
import oracle, paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import rel_l2_rows, to_dev, to_host
x = synth.gaussian((40, 1024), seed=6)
xd = to_dev(x); yd = torch.empty_like(xd)
for _ in range(2):   # the first call sets the device up
    rc = fg.lib().fft_fourstep_noalloc(xd.data_ptr(), yd.data_ptr(), 1024, 40, fg.FFT_INVERSE, None)
    assert rc == 0, rc
    torch.cuda.synchronize()
    err = rel_l2_rows(to_host(yd), oracle.fft(x, inverse=True)).max()
    assert err <= {tol}, err
print("child ok", err)
"""


def test_first_call_in_a_fresh_process():
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), tol=TOL_FP32)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "child ok" in r.stdout
