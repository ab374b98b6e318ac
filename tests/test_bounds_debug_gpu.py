"""The bounds-checking debug build (FFTGB_BOUNDS_CHECK), the library's
stand-in for a memory checker: every single-CTA Stockham configuration runs
under it in a child process (one CTA per tile with a ragged last tile, and
persistent grids over more than one round of tiles, both directions), and so
do the column kernels behind column plans (one and two launches, strided,
several scratch passes), the two-phase four-step and the allocation-free
entry point; the results must match the FP64 oracle and no check may fail.  A deliberate
failed check (the self-test, which accesses nothing) must be reported, so
the checks are known to be live.  No check traps: a failed one is recorded
and its access skipped."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np
import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import TOL_FP32, rel_l2_rows, to_dev, to_host
assert fg.library_path() == {lib!r}
assert fg.fft_debug_bounds_status() == 0
assert fg.fft_debug_bounds_selftest() == 0
assert fg.fft_debug_bounds_status() == 99, "the self-test's failed check was not reported"
assert fg.fft_debug_bounds_status() == 0, "reading clears the record"
runs = 0
for e in range(1, 15):
    N = 1 << e
    for c in fg.fft_list_configs(N):
        if c["path"] != fg.FFT_PATH_SINGLE_CTA or c["cluster_split"] or c["tma_slabs"]:
            continue
        tb = c["transforms_per_cta"]
        if c["ctas_per_sm"] == 0:
            batch = 3 * tb + 1                      # a ragged last tile
        else:
            probe = fg.Plan(N, 1, fg.FFT_FORWARD, config=c)
            grid = probe.info()["grid_ctas"]
            probe.close()
            batch = (grid + 2) * tb + 1             # more tiles than CTAs, ragged tail
        x = synth.gaussian((batch, N), seed=N + tb)
        rows = np.unique(np.r_[0, 1, batch // 2, batch - 2, batch - 1]) if batch > 5 \
            else np.arange(batch)
        for direction in (fg.FFT_FORWARD, fg.FFT_INVERSE):
            p = fg.Plan(N, batch, direction, config=c)
            y = to_host(p(to_dev(x))).reshape(batch, N)
            p.close()
            want = oracle.fft(x[rows], inverse=direction > 0)
            err = rel_l2_rows(y[rows], want).max()
            assert err <= TOL_FP32, (N, c, direction, err)
            runs += 1
st = fg.fft_debug_bounds_status()
assert st == 0, f"bounds check failed at site {{st}}"
print("bounds ok", runs)
"""


def test_every_stockham_configuration_under_bounds_checks():
    from paper_2603_27569_gb300 import build

    lib = build.build(debug=True)
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
    env = dict(os.environ, FFTGB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=1500, env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds ok" in r.stdout


COLUMN_CHILD = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np, torch
import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import TOL_FP32, rel_l2_rows, to_dev, to_host
assert fg.library_path() == {lib!r}
assert fg.fft_debug_bounds_status() == 0
runs = 0
# column plans: padded rows, gaps between matrices, both routes where there are two
cases = [(256, 0), (1024, 0), (2048, fg.FFT_FLAG_FORCE_SINGLE_CTA),
         (2048, fg.FFT_FLAG_FORCE_FOURSTEP), (4096, fg.FFT_FLAG_FORCE_SINGLE_CTA), (4096, 0),
         (8192, 0), (65536, 0)]
for L, flags in cases:
    nmat, ncols, pad, gap = 2, 32, 16, 24
    rs, ms = ncols + pad, L * (ncols + pad) + gap
    buf = synth.gaussian(nmat * ms, seed=L)
    e = buf.itemsize
    x = np.array(np.lib.stride_tricks.as_strided(buf, (nmat, L, ncols), (ms * e, rs * e, e)))
    for direction in (fg.FFT_FORWARD, fg.FFT_INVERSE):
        plan = fg.ColumnPlan(L, ncols, nmat, rs, ms, direction, flags=flags)
        out = to_host(plan(to_dev(buf)))
        plan.close()
        got = np.lib.stride_tricks.as_strided(out, (nmat, L, ncols), (ms * e, rs * e, e))
        cols = lambda a: np.transpose(a, (0, 2, 1)).reshape(-1, L)
        want = oracle.fft(cols(x), inverse=direction > 0)
        assert rel_l2_rows(cols(got), want).max() <= TOL_FP32, (L, flags, direction)
        runs += 1
# long columns in several scratch passes (3 matrices of 512 MiB, passes of 2 and 1)
L, ncols, nmat = 16384, 4096, 3
xd = torch.randn((nmat, L, ncols), dtype=torch.complex64, device="cuda",
                 generator=torch.Generator(device="cuda").manual_seed(1))
plan = fg.ColumnPlan(L, ncols, nmat)
yd = plan(xd)
torch.cuda.synchronize()
plan.close()
for m in range(nmat):
    c = [0, 17, ncols - 1]
    x1 = xd[m][:, c].cpu().numpy().T
    y1 = yd[m][:, c].cpu().numpy().T
    assert rel_l2_rows(y1, oracle.fft(x1)).max() <= TOL_FP32, m
runs += 1
del xd, yd
# the two-phase four-step (rows) and the allocation-free entry point
for N, batch in ((1 << 15, 5), (1 << 16, 3), (1 << 18, 2)):
    x = synth.gaussian((batch, N), seed=N)
    p = fg.Plan(N, batch, fg.FFT_FORWARD, flags=fg.FFT_FLAG_FORCE_FOURSTEP)
    y = to_host(p(to_dev(x))).reshape(batch, N)
    p.close()
    assert rel_l2_rows(y, oracle.fft(x)).max() <= TOL_FP32, N
    runs += 1
x = synth.gaussian((37, 4096), seed=3)
xd = to_dev(x); yd = torch.empty_like(xd)
assert fg.lib().fft_fourstep_noalloc(xd.data_ptr(), yd.data_ptr(), 4096, 37, fg.FFT_FORWARD, None) == 0
torch.cuda.synchronize()
assert rel_l2_rows(to_host(yd), oracle.fft(x)).max() <= TOL_FP32
runs += 1
st = fg.fft_debug_bounds_status()
assert st == 0, f"bounds check failed at site {{st}}"
print("bounds ok", runs)
"""


def test_column_kernels_under_bounds_checks():
    from paper_2603_27569_gb300 import build

    lib = build.build(debug=True)
    code = COLUMN_CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
    env = dict(os.environ, FFTGB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=1500, env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds ok" in r.stdout
