"""The bounds-checking debug build (FFTGB_BOUNDS_CHECK), the library's
stand-in for a memory checker: every single-CTA Stockham configuration runs
under it in a child process (one CTA per tile with a ragged last tile, and
persistent grids over more than one round of tiles, both directions); the
results must match the FP64 oracle and no check may fail.  A deliberate
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
