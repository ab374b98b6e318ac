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
    # at 4096: 4, 12 and 8 columns take the one-launch 4-column tile (the
    # two-launch default needs multiples of 16)
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
        assert plan.info()["path"] == fg.FFT_PATH_COLUMNS and plan.info()["n2"] == 0
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
    with pytest.raises(fg.FFTError) as e:      # L beyond the longest column
        fg.ColumnPlan(1 << 22, 16, 1)
    assert e.value.status == 1
    with pytest.raises(fg.FFTError) as e:      # long columns take 16-column tiles
        fg.ColumnPlan(16384, 8, 1)
    assert e.value.status == 1
    with pytest.raises(fg.FFTError) as e:      # overlapping rows
        fg.ColumnPlan(256, 32, 1, row_stride=16)
    assert e.value.status == 2
    with pytest.raises(fg.FFTError) as e:      # overlapping matrices
        fg.ColumnPlan(256, 32, 2, row_stride=32, mat_stride=100)
    assert e.value.status == 2


# ---------------------------------------------------------------------------
# Columns longer than 4096: two launches through the plan's scratch (the
# four-step factorisation down the column, L = n1 n2).
# ---------------------------------------------------------------------------
def strided_case(L, nmat, ncols, pad, gap, seed):
    rs = ncols + pad
    ms = L * rs + gap
    buf = synth.gaussian(nmat * ms, seed=seed)
    e = buf.itemsize
    x = np.array(np.lib.stride_tricks.as_strided(buf, shape=(nmat, L, ncols),
                                                 strides=(ms * e, rs * e, e)))
    return buf, x, rs, ms


def run_strided(plan, buf, nmat, L, ncols, rs, ms, canary=complex(7.0, -7.0)):
    dev_in = to_dev(buf)
    dev_out = torch.full_like(dev_in, canary)
    plan(dev_in, dev_out)
    torch.cuda.synchronize()
    out = to_host(dev_out)
    e = out.itemsize
    got = np.array(np.lib.stride_tricks.as_strided(out, shape=(nmat, L, ncols),
                                                   strides=(ms * e, rs * e, e)))
    return out, got


def col_err(got, want):
    L = got.shape[1]
    return rel_l2_rows(np.transpose(got, (0, 2, 1)).reshape(-1, L),
                       np.transpose(want, (0, 2, 1)).reshape(-1, L))


@pytest.mark.parametrize("L", [8192, 16384, 32768, 65536])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_long_strided_columns_match_oracle(L, direction):
    for nmat, ncols, pad, gap in ((1, 16, 0, 0), (2, 48, 16, 40), (3, 32, 5, 0)):
        buf, x, rs, ms = strided_case(L, nmat, ncols, pad, gap, seed=L + ncols + pad)
        plan = fg.ColumnPlan(L, ncols, nmat, rs, ms, direction)
        info = plan.info()
        assert info["path"] == fg.FFT_PATH_COLUMNS
        assert info["n1"] * info["n2"] == L and info["n2"] == min(512, 1 << ((L.bit_length()) // 2))
        assert info["scratch_bytes"] == 8 * L * ncols * nmat
        out, got = run_strided(plan, buf, nmat, L, ncols, rs, ms)
        plan.close()
        err = col_err(got, column_oracle(x, direction > 0))
        assert err.max() <= TOL_FP32, (L, nmat, ncols, pad, gap, err.max())
        mask = np.ones(out.shape, bool)
        for m in range(nmat):
            for r in range(L):
                mask[m * ms + r * rs: m * ms + r * rs + ncols] = False
        assert np.all(out[mask] == complex(7.0, -7.0))


def test_long_column_plan_without_matrices():
    plan = fg.ColumnPlan(16384, 64, 0)
    assert plan.info()["scratch_bytes"] == 0
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    fg.fft_exec(plan.handle, x, x, None)     # nothing to do
    plan.close()


def test_longest_column():
    L, ncols = 1 << 21, 16
    x = synth.gaussian((1, L, ncols), seed=21)
    plan = fg.ColumnPlan(L, ncols, 1)
    assert (plan.info()["n1"], plan.info()["n2"]) == (4096, 512)
    y = to_host(plan(to_dev(x)))
    plan.close()
    assert col_err(y, column_oracle(x, False)).max() <= TOL_FP32


def test_long_columns_in_place_round_trip_and_wrapper():
    L, ncols, nmat = 16384, 64, 2
    x = synth.gaussian((nmat, L, ncols), seed=5)
    t = to_dev(x)
    y = fg.fft_columns(t)
    assert col_err(to_host(y), column_oracle(x, False)).max() <= TOL_FP32
    plan = fg.ColumnPlan(L, ncols, nmat)
    plan(t, t)                                     # in place
    assert np.array_equal(to_host(t).view(np.uint32), to_host(y).view(np.uint32))
    plan.close()
    back = to_host(fg.fft_columns(y, inverse=True))
    assert rel_l2_rows(back.reshape(-1, ncols), x.reshape(-1, ncols)).max() <= 2e-6


def test_long_column_twiddle_grid_is_exact():
    """The phase-1 table holds W_L^{j k} (j < n1, k < n2) at j * n2 + k, each
    entry the FP64 value rounded once to FP32."""
    L = 8192
    plan = fg.ColumnPlan(L, 16, 1)
    n1, n2 = plan.info()["n1"], plan.info()["n2"]
    tab = fg.fft_twiddle_table(plan.handle)[-L:]
    plan.close()
    j, k = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    e = (j * k) % L
    want = np.exp(-2j * np.pi * e.reshape(-1) / L)
    assert np.abs(tab.astype(np.complex128) - want).max() <= 6e-8


def test_long_columns_over_several_scratch_passes():
    """A batch larger than the 1 GiB scratch runs as several pairs of
    launches: 3 matrices of 16384 x 4096 (512 MiB each) in passes of 2 and 1.
    Sampled columns of every matrix against the oracle; the in-place run is
    bit-identical to the out-of-place one."""
    L, ncols, nmat = 16384, 4096, 3
    g = torch.Generator(device="cuda").manual_seed(9)
    xd = torch.randn((nmat, L, ncols), dtype=torch.complex64, device="cuda", generator=g)
    plan = fg.ColumnPlan(L, ncols, nmat)
    assert plan.info()["scratch_bytes"] == 2 * 8 * L * ncols
    yd = plan(xd)
    torch.cuda.synchronize()
    cols = np.random.default_rng(2).choice(ncols, 8, replace=False)
    for m in range(nmat):
        x = xd[m][:, cols].cpu().numpy()[None]
        y = yd[m][:, cols].cpu().numpy()[None]
        assert col_err(y, column_oracle(x, False)).max() <= TOL_FP32, m
    plan(xd, xd)
    torch.cuda.synchronize()
    assert torch.equal(xd.view(torch.float32), yd.view(torch.float32))
    plan.close()


@pytest.mark.parametrize("L", [2048, 4096])
def test_forced_routes_at_2048_and_4096(L):
    """Both routes of a 2048- or 4096-point column (one CTA per column tile,
    or the two launches of the long path) match the oracle."""
    nmat, ncols, pad, gap = 2, 48, 16, 40
    buf, x, rs, ms = strided_case(L, nmat, ncols, pad, gap, seed=L + 1)
    for flags, two in ((fg.FFT_FLAG_FORCE_SINGLE_CTA, False), (fg.FFT_FLAG_FORCE_FOURSTEP, True),
                       (0, L == 4096)):
        for direction in (fg.FFT_FORWARD, fg.FFT_INVERSE):
            plan = fg.ColumnPlan(L, ncols, nmat, rs, ms, direction, flags=flags)
            assert (plan.info()["n2"] > 0) == two
            _, got = run_strided(plan, buf, nmat, L, ncols, rs, ms)
            plan.close()
            err = col_err(got, column_oracle(x, direction > 0))
            assert err.max() <= TOL_FP32, (flags, direction, err.max())


@pytest.mark.parametrize("L,flags", [(1024, 0), (2048, 0), (4096, 0), (4096, fg.FFT_FLAG_FORCE_SINGLE_CTA),
                                     (16384, 0), (65536, 0)])
def test_bench_column_workload_sampled(L, flags):
    """The bench's azimuth workload: one contiguous [L, 2^25 / L] matrix (256
    MiB), in the launch the bench times; sampled columns against the oracle."""
    ncols = (1 << 25) // L
    g = torch.Generator(device="cuda").manual_seed(L)
    xd = torch.randn((L, ncols), dtype=torch.complex64, device="cuda", generator=g)
    plan = fg.ColumnPlan(L, ncols, 1, flags=flags)
    yd = plan(xd)
    torch.cuda.synchronize()
    plan.close()
    cols = np.unique(np.r_[0, 1, ncols - 1, np.random.default_rng(L).choice(ncols, 13)])
    x = xd[:, cols].cpu().numpy().T
    y = yd[:, cols].cpu().numpy().T
    assert rel_l2_rows(y, oracle.fft(x, nthreads=NTHREADS)).max() <= TOL_FP32
