"""Split-precision tensor-core FFT against the FP64 oracle.

Target: relative L2 error <= 1e-5 per transform for FP16 hi+lo and for BF16
hi+lo alike (BF16 hi+lo keeps ~16 significant bits of each operand, enough
for the measured <= 6e-6 at these sizes).  The per-size error table is
printed (pytest -s)."""
import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_SPLIT, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"fp16x2": fg.FFT_PREC_FP16X2, "bf16x2": fg.FFT_PREC_BF16X2}
BOUND = {"fp16x2": TOL_SPLIT, "bf16x2": TOL_SPLIT}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


def run_tc(x, direction, prec):
    N = x.shape[-1]
    plan = fg.Plan(N, x.shape[0], direction, precision=PREC[prec])
    assert plan.info()["path"] == fg.FFT_PATH_TENSORCORE
    y = to_host(plan(to_dev(x)))
    plan.close()
    return y


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
@pytest.mark.parametrize("N", [256, 4096, 16384])
@pytest.mark.parametrize("dist", ["gaussian", "uniform"])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_split_precision_error_vs_oracle(prec, N, dist, direction):
    batch = 37
    x = synth.gaussian((batch, N), seed=0) if dist == "gaussian" else \
        synth.uniform((batch, N), seed=3)
    y = run_tc(x, direction, prec)
    want = oracle.fft(x, inverse=direction > 0, nthreads=NTHREADS)
    err = rel_l2_rows(y, want)
    print(f"\nTC {prec} N={N} {dist} {'inv' if direction > 0 else 'fwd'}: "
          f"max rel L2 {err.max():.3e} median {np.median(err):.3e}")
    assert err.max() <= BOUND[prec]


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
@pytest.mark.parametrize("N", [4096, 16384])
def test_config5_batch_sampled_rows(N, prec):
    # the config's batch (16384 rows), N(0,1); a seeded sample of 512 rows
    # (first and last included) checked against the oracle
    batch = 16384
    x = synth.gaussian((batch, N), seed=0)
    y = run_tc(x, fg.FFT_FORWARD, prec)
    rng = np.random.Generator(np.random.PCG64(11))
    rows = np.unique(np.concatenate([[0, batch - 1], rng.choice(batch, 510, replace=False)]))
    err = rel_l2_rows(y[rows], oracle.fft(x[rows], nthreads=NTHREADS))
    print(f"\nTC {prec} N={N} batch {batch}: {len(rows)} sampled rows, max rel L2 "
          f"{err.max():.3e} median {np.median(err):.3e}")
    assert err.max() <= BOUND[prec]
    assert np.isfinite(y).all()


def test_unsupported_sizes_are_refused():
    with pytest.raises(fg.FFTError) as e:
        fg.Plan(1024, 4, fg.FFT_FORWARD, precision=fg.FFT_PREC_FP16X2)
    assert e.value.status == 7


@pytest.mark.parametrize("N", [256, 4096, 16384])
@pytest.mark.parametrize("batch", [1, 17])
def test_small_and_ragged_batches(N, batch):
    # one row; and (N = 256, 16 rows per CTA) a partly filled last row group
    x = synth.gaussian((batch, N), seed=batch)
    y = run_tc(x, fg.FFT_FORWARD, "fp16x2")
    err = rel_l2_rows(y, oracle.fft(x, nthreads=NTHREADS))
    assert err.max() <= TOL_SPLIT


@pytest.mark.parametrize("N", [256, 4096, 16384])
def test_in_place_round_trip_and_determinism(N):
    x = synth.gaussian((9, N), seed=11)
    fwd = fg.Plan(N, 9, fg.FFT_FORWARD, precision=fg.FFT_PREC_FP16X2)
    inv = fg.Plan(N, 9, fg.FFT_INVERSE, precision=fg.FFT_PREC_FP16X2)
    xd = to_dev(x)
    a = to_host(fwd(xd))
    b = to_host(fwd(xd))
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))   # run-to-run bitwise
    fwd(xd, out=xd)                                                 # in place
    assert np.array_equal(to_host(xd).view(np.uint32), a.view(np.uint32))
    back = to_host(inv(xd))
    fwd.close()
    inv.close()
    assert rel_l2_rows(back, x).max() <= 2 * TOL_SPLIT
    assert np.isfinite(back).all()
