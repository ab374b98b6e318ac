"""Ragged (mixed-length, mixed-direction) batches in one persistent launch,
against the FP64 oracle per transform and against plain per-size plans."""
import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


def packed_case(count, seed, lo=4, hi=14):
    d = synth.ragged_draw(count, seed=seed, log2_lo=lo, log2_hi=hi)
    x = synth.gaussian(d["total"], seed=seed + 100)
    return d, x


def run_ragged(d, x, flags=0, out_offset=None):
    out_offset = d["offset"] if out_offset is None else out_offset
    plan = fg.fft_ragged_plan(d["N"], d["direction"], d["offset"], out_offset, flags)
    xd = to_dev(x)
    yd = torch.full((int(out_offset.max() + d["N"].max()) if len(d["N"]) else 1,),
                    float("nan"), dtype=torch.complex64, device="cuda")
    fg.fft_exec(plan, xd, yd, torch.cuda.current_stream())
    torch.cuda.synchronize()
    info = fg.fft_plan_info(plan)
    assert fg.fft_last_device_status(plan) == 0
    fg.fft_destroy(plan)
    return to_host(yd), info


def check_rows(d, x, y, rows, tol=TOL_FP32, unnormalized=False):
    for i in rows:
        N = int(d["N"][i])
        o = int(d["offset"][i])
        inv = d["direction"][i] > 0
        want = oracle.fft(x[o:o + N], inverse=inv)
        if inv and unnormalized:
            want = want * N
        err = rel_l2_rows(y[o:o + N][None], want[None])[0]
        assert err <= tol, f"row {i} N={N} inv={inv}: rel L2 {err:.2e}"


def test_small_ragged_batch_every_row_matches_oracle():
    d, x = packed_case(400, seed=0)
    y, info = run_ragged(d, x)
    assert info["path"] == fg.FFT_PATH_RAGGED and info["batch"] == 400
    check_rows(d, x, y, range(400))
    assert np.isfinite(y[: d["total"]]).all()


def test_unnormalized_inverse_flag():
    d, x = packed_case(60, seed=1)
    y, _ = run_ragged(d, x, flags=fg.FFT_FLAG_UNNORMALIZED_INVERSE)
    check_rows(d, x, y, range(60), unnormalized=True)


def test_separate_output_offsets_and_graph_replay():
    d, x = packed_case(120, seed=2)
    rng = np.random.Generator(np.random.PCG64(5))
    # scatter the outputs into a larger buffer in a permuted order
    perm = rng.permutation(len(d["N"]))
    out_off = np.zeros_like(d["offset"])
    pos = 0
    for i in perm:
        out_off[i] = pos
        pos += int(d["N"][i]) + 16
    plan = fg.fft_ragged_plan(d["N"], d["direction"], d["offset"], out_off)
    xd = to_dev(x)
    y1 = torch.zeros(pos, dtype=torch.complex64, device="cuda")
    y2 = torch.zeros(pos, dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream()
    fg.fft_exec(plan, xd, y1, st)
    fg.fft_exec(plan, xd, y1, st)      # replay of the captured graph
    fg.fft_exec(plan, xd, y2, st)      # new output pointer: re-capture
    torch.cuda.synchronize()
    fg.fft_destroy(plan)
    a, b = to_host(y1), to_host(y2)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    for i in range(len(d["N"])):
        N, o, oo = int(d["N"][i]), int(d["offset"][i]), int(out_off[i])
        want = oracle.fft(x[o:o + N], inverse=d["direction"][i] > 0)
        assert rel_l2_rows(a[oo:oo + N][None], want[None])[0] <= TOL_FP32


def test_config3_size_20000_transforms():
    # 20000 transforms, log2 N ~ U{8..14}, mixed directions (seed 0)
    d, x = packed_case(20000, seed=0, lo=8, hi=14)
    y, _ = run_ragged(d, x)
    assert np.isfinite(y[: d["total"]]).all()
    rng = np.random.Generator(np.random.PCG64(7))
    rows = rng.choice(20000, size=60, replace=False)
    check_rows(d, x, y, rows)
    # identical math to per-(N, direction) plain plans, to the FP32 tolerance
    xd = to_dev(x)
    worst = 0.0
    for N in np.unique(d["N"]):
        for dirn in (-1, 1):
            sel = np.nonzero((d["N"] == N) & (d["direction"] == dirn))[0]
            if len(sel) == 0:
                continue
            idx = (d["offset"][sel][:, None] + np.arange(N)[None, :]).reshape(-1)
            it = torch.from_numpy(idx).cuda()
            grp = xd[it].contiguous()
            plan = fg.Plan(int(N), len(sel), dirn)
            ref = plan(grp).reshape(len(sel), int(N))
            plan.close()
            got = torch.from_numpy(y[idx]).cuda().reshape(len(sel), int(N))
            err = (torch.linalg.vector_norm(got - ref, dim=1) /
                   torch.linalg.vector_norm(ref, dim=1)).max().item()
            worst = max(worst, err)
    assert worst <= 2 * TOL_FP32


def test_ragged_argument_errors():
    L = fg.lib()
    import ctypes
    h = ctypes.c_void_p()
    N = np.array([256, 8], np.int32)
    dr = np.array([-1, -1], np.int32)
    off = np.array([0, 256], np.int64)
    assert L.fft_ragged_plan(ctypes.byref(h), 2, N.ctypes.data, dr.ctypes.data, off.ctypes.data,
                             off.ctypes.data, 0) == 7           # N = 8: not supported
    N = np.array([256, 12], np.int32)
    assert L.fft_ragged_plan(ctypes.byref(h), 2, N.ctypes.data, dr.ctypes.data, off.ctypes.data,
                             off.ctypes.data, 0) == 1           # not a power of two
    N = np.array([256, 256], np.int32)
    bad = np.array([0, 257], np.int64)
    assert L.fft_ragged_plan(ctypes.byref(h), 2, N.ctypes.data, dr.ctypes.data, bad.ctypes.data,
                             off.ctypes.data, 0) == 3           # odd offset
    dz = np.array([-1, 0], np.int32)
    assert L.fft_ragged_plan(ctypes.byref(h), 2, N.ctypes.data, dz.ctypes.data, off.ctypes.data,
                             off.ctypes.data, 0) == 2           # bad direction
    plan = fg.fft_ragged_plan(np.zeros(0, np.int32), np.zeros(0, np.int32),
                              np.zeros(0, np.int64), np.zeros(0, np.int64))
    fg.fft_exec(plan, 16, 16)                                     # empty: nothing to do
    fg.fft_destroy(plan)


def _explicit_case(sizes_dirs_counts, seed):
    """Rows of given (N, direction, count), packed in an interleaved order."""
    N, D = [], []
    for n, dirn, cnt in sizes_dirs_counts:
        N += [n] * cnt
        D += [dirn] * cnt
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(len(N))
    N = np.array(N, np.int32)[perm]
    D = np.array(D, np.int32)[perm]
    off = np.concatenate([[0], np.cumsum(N.astype(np.int64))[:-1]]).astype(np.int64)
    d = {"N": N, "direction": D, "offset": off, "total": int(N.sum())}
    return d, synth.gaussian(d["total"], seed=seed + 100)


@pytest.mark.parametrize("N", [16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384])
def test_every_compiled_routine_matches_oracle(N):
    """Each compiled routine of class N, forced through fft_ragged_choose, on
    one and a half units of rows per direction (a partial last unit), mixed
    with rows of another class."""
    other = 1024 if N != 1024 else 256
    try:
        for cfg in fg.fft_ragged_list_configs(N):
            fg.fft_ragged_choose(N, fg.FFT_FORWARD, cfg)
            fg.fft_ragged_choose(N, fg.FFT_INVERSE, cfg)
            per = cfg["transforms_per_cta"]
            cnt = per + max(1, per // 2)
            d, x = _explicit_case([(N, -1, cnt), (N, 1, cnt), (other, 1, 3)], seed=N)
            plan = fg.fft_ragged_plan(d["N"], d["direction"], d["offset"], d["offset"])
            assert fg.fft_ragged_class_config(plan, N, fg.FFT_FORWARD) == cfg
            assert fg.fft_ragged_class_config(plan, N, fg.FFT_INVERSE) == cfg
            fg.fft_destroy(plan)
            y, _ = run_ragged(d, x)
            check_rows(d, x, y, range(len(d["N"])))
    finally:
        fg.fft_autotune_clear()


def test_one_launch_plan_info_and_class_configs():
    d, x = packed_case(300, seed=9, lo=8, hi=14)
    plan = fg.fft_ragged_plan(d["N"], d["direction"], d["offset"], d["offset"],
                              fg.FFT_FLAG_NO_AUTOTUNE_CACHE)
    info = fg.fft_plan_info(plan)
    assert info["path"] == fg.FFT_PATH_RAGGED and info["threads_per_cta"] == 512
    for N in np.unique(d["N"]):
        for dirn in (-1, 1):
            present = np.any((d["N"] == N) & (d["direction"] == dirn))
            if present:
                c = fg.fft_ragged_class_config(plan, int(N), dirn)
                assert c == fg.fft_ragged_list_configs(int(N))[0]      # the built-in routine
                # a unit fills its worker: the whole CTA for 16384, a 256-thread half otherwise
                assert c["threads_per_cta"] == (512 if N == 16384 else 256)
                assert c["transforms_per_cta"] * int(N) == c["threads_per_cta"] * c["points_per_thread"]
            else:
                with pytest.raises(fg.FFTError):
                    fg.fft_ragged_class_config(plan, int(N), dirn)
    fg.fft_destroy(plan)


def test_autotune_flag_chooses_and_remembers_per_class():
    d, x = packed_case(600, seed=11, lo=8, hi=14)
    try:
        y, _ = run_ragged(d, x, flags=fg.FFT_FLAG_RAGGED_AUTOTUNE)
        check_rows(d, x, y, range(0, 600, 7))
        tuned = fg.fft_ragged_plan(d["N"], d["direction"], d["offset"], d["offset"],
                                   fg.FFT_FLAG_RAGGED_AUTOTUNE)
        later = fg.fft_ragged_plan(d["N"], d["direction"], d["offset"], d["offset"])
        for N in np.unique(d["N"]):
            for dirn in (-1, 1):
                if np.any((d["N"] == N) & (d["direction"] == dirn)):
                    c = fg.fft_ragged_class_config(tuned, int(N), dirn)
                    assert c in fg.fft_ragged_list_configs(int(N))
                    assert fg.fft_ragged_class_config(later, int(N), dirn) == c
        fg.fft_destroy(tuned)
        fg.fft_destroy(later)
    finally:
        fg.fft_autotune_clear()
