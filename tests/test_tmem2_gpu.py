"""Rows of 32768 points in one HBM pass on one SM (tmem2.cuh), through the C
ABI: a radix-2 decimation-in-frequency split into two 16384-point halves,
one held in tensor memory while the other transforms.  Checked against the
FP64 oracle per row: both directions, both twiddle modes, batches below,
at and beyond one row per SM with a ragged last round, in place, an output
that is 16- but not 32-byte aligned (the epilogue's narrower stores), and
the device status word after the runs."""
import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1 << 15


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


def configs():
    return [c for c in fg.fft_list_configs(N) if c["path"] == fg.FFT_PATH_TMEM_HALVES]


def want(x, direction):
    return oracle.fft(x, inverse=direction == fg.FFT_INVERSE, nthreads=NTHREADS)


def test_listed_and_default():
    cfgs = configs()
    assert sorted(c["twiddle_mode"] for c in cfgs) == [0, 1]
    for c in cfgs:
        assert c["threads_per_cta"] == 512 and c["points_per_thread"] == 32
        assert int(np.prod(c["radix"][:c["num_passes"]])) == N // 2
    plan = fg.Plan(N, 2, fg.FFT_FORWARD)
    info = plan.info()
    plan.close()
    assert info["path"] == fg.FFT_PATH_TMEM_HALVES and info["twiddle_mode"] == 1
    assert 0 < info["grid_ctas"] <= torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("twm", [0, 1])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
@pytest.mark.parametrize("batch", [1, 5, 152, 311])
def test_matches_oracle(batch, direction, twm):
    cfg = next(c for c in configs() if c["twiddle_mode"] == twm)
    x = synth.gaussian((batch, N), seed=batch * 7 + twm + (direction > 0))
    plan = fg.Plan(N, batch, direction, config=cfg)
    y = to_host(plan(to_dev(x))).reshape(batch, N)
    plan.close()
    # every row of the small batches; for the large ones the first rows, the
    # rows of the second round and the ragged last round (the persistent
    # grid has one CTA per SM)
    rows = np.arange(batch) if batch <= 5 else np.unique(
        np.r_[0:3, 150:156, batch - 4:batch])
    rows = rows[rows < batch]
    err = rel_l2_rows(y[rows], want(x[rows], direction))
    assert err.max() <= TOL_FP32, err.max()
    assert np.isfinite(y).all()


def test_in_place_and_unaligned_output():
    batch = 160
    x = synth.gaussian((batch, N), seed=11)
    rows = np.r_[0:2, 151:155, batch - 2:batch]
    ref = want(x[rows], fg.FFT_FORWARD)
    plan = fg.Plan(N, batch, fg.FFT_FORWARD)
    xd = to_dev(x).reshape(-1)
    plan(xd, out=xd)  # in place
    torch.cuda.synchronize()
    assert rel_l2_rows(to_host(xd).reshape(batch, N)[rows], ref).max() <= TOL_FP32
    # an output 16 bytes past a 32-byte boundary takes the 16-byte stores
    buf = torch.empty(batch * N + 2, dtype=torch.complex64, device="cuda")
    out = buf[2:]
    assert out.data_ptr() % 32 == 16
    plan(to_dev(x).reshape(-1), out=out)
    torch.cuda.synchronize()
    assert rel_l2_rows(to_host(out).reshape(batch, N)[rows], ref).max() <= TOL_FP32
    assert fg.fft_last_device_status(plan.handle) == 0
    plan.close()


def test_host_buffers():
    # fft_exec_host: pinned host input and output, the rows streamed through
    # the device in chunks (each chunk one launch of the one-pass kernel)
    batch = 40
    x = synth.gaussian((batch, N), seed=12)
    plan = fg.Plan(N, batch, fg.FFT_INVERSE)
    y = plan.exec_host(torch.from_numpy(x).pin_memory()).numpy().reshape(batch, N)
    plan.close()
    assert rel_l2_rows(y, want(x, fg.FFT_INVERSE)).max() <= TOL_FP32
