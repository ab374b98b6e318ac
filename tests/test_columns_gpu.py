"""Column transforms without a transpose (fft_plan_columns): the azimuth pass
over a strided [azimuth, range] matrix.  Every column of every matrix must
equal the FP64 oracle's transform of that column (5e-6 relative L2)."""
import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = {16: 16, 64: 16, 256: 16, 512: 16, 1024: 8, 2048: 8, 4096: 4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


def column_oracle(x: np.ndarray, inverse: bool) -> np.ndarray:
    """x [nmat, L, ncols]: transform every column (axis 1) with the oracle."""
    nmat, L, ncols = x.shape
    cols = np.ascontiguousarray(np.transpose(x, (0, 2, 1))).reshape(-1, L)
    y = oracle.fft(cols, inverse=inverse, nthreads=NTHREADS).reshape(nmat, ncols, L)
    return np.transpose(y, (0, 2, 1))


@pytest.mark.parametrize("L", [16, 256, 1024, 2048, 4096])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_strided_columns_match_oracle(L, direction):
    C = TILE[L]
    for nmat, ncols, pad, gap in ((1, C, 0, 0), (2, 3 * C, 16, 40), (3, 2 * C, 5, 0)):
        rs = ncols + pad                       # padded rows
        ms = L * rs + gap                      # gap between matrices
        buf = synth.gaussian(nmat * ms, seed=L + ncols + pad)
        e = buf.itemsize
        view = np.lib.stride_tricks.as_strided(
            buf, shape=(nmat, L, ncols), strides=(ms * e, rs * e, e))
        x = np.array(view)
        plan = fg.ColumnPlan(L, ncols, nmat, rs, ms, direction)
        assert plan.info()["path"] == fg.FFT_PATH_COLUMNS
        dev_in = to_dev(buf)
        dev_out = torch.full_like(dev_in, complex(7.0, -7.0))   # canary outside the extent
        plan(dev_in, dev_out)
        torch.cuda.synchronize()
        out = to_host(dev_out)
        plan.close()
        got = np.lib.stride_tricks.as_strided(out, shape=(nmat, L, ncols),
                                              strides=(ms * e, rs * e, e))
        want = column_oracle(x, direction > 0)
        err = rel_l2_rows(np.transpose(got, (0, 2, 1)).reshape(-1, L),
                          np.transpose(want, (0, 2, 1)).reshape(-1, L))
        assert err.max() <= TOL_FP32, (nmat, ncols, pad, gap, err.max())
        # elements outside the strided extent are untouched
        mask = np.ones(out.shape, bool)
        for m in range(nmat):
            for r in range(L):
                mask[m * ms + r * rs: m * ms + r * rs + ncols] = False
        assert np.all(out[mask] == complex(7.0, -7.0))


def test_in_place_and_torch_wrapper():
    L, ncols = 1024, 48
    x = synth.gaussian((2, L, ncols), seed=3)
    t = to_dev(x)
    y = fg.fft_columns(t)                          # [nmat, L, ncols]
    want = column_oracle(x, False)
    assert rel_l2_rows(np.transpose(to_host(y), (0, 2, 1)).reshape(-1, L),
                       np.transpose(want, (0, 2, 1)).reshape(-1, L)).max() <= TOL_FP32
    plan = fg.ColumnPlan(L, ncols, 2)
    plan(t, t)                                     # in place
    assert np.array_equal(to_host(t).view(np.uint32), to_host(y).view(np.uint32))
    plan.close()
    back = fg.fft_columns(y, inverse=True)
    assert rel_l2_rows(to_host(back).reshape(-1, ncols), x.reshape(-1, ncols)).max() <= 2e-6


def test_column_plan_rejects_bad_geometry():
    with pytest.raises(fg.FFTError) as e:      # ncols not a multiple of the tile
        fg.ColumnPlan(4096, 6, 1)
    assert e.value.status == 1
    with pytest.raises(fg.FFTError) as e:      # L beyond the column kernels
        fg.ColumnPlan(8192, 16, 1)
    assert e.value.status == 1
    with pytest.raises(fg.FFTError) as e:      # overlapping rows
        fg.ColumnPlan(256, 32, 1, row_stride=16)
    assert e.value.status == 2
    with pytest.raises(fg.FFTError) as e:      # overlapping matrices
        fg.ColumnPlan(256, 32, 2, row_stride=32, mat_stride=100)
    assert e.value.status == 2
