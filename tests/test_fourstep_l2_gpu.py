"""Single-launch four-step with the intermediate in an L2 ring (N = L * L).

Both phases of the two-phase four-step (Sec. IV-B, Eq. 3) run in one
persistent launch whose work items are ordered by a device counter; a chunk's
intermediate lives in a ring slot that is reused once its phase 2 is done.
Batches here span many chunks, so every slot is reused several times and the
last chunk is ragged.  Parity is against the FP64 oracle (5e-6 relative L2
per transform) and against the two-launch four-step with the same split,
which runs the same arithmetic.
"""
import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C = 16  # columns per CTA


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def l2_configs(N):
    return [c for c in fg.fft_list_configs(N) if c["l2_chunk_rows"] > 0]


def ring_batch(N, rows, grid):
    """A batch that reuses every ring slot at least three times, ragged tail."""
    L = int(round(N ** 0.5))
    rnd = 2 * rows * (L // C)
    lag = (2 * grid + rnd - 1) // rnd + 1
    slots = 2 * lag
    return (slots + 3) * rows + rows // 2 + 1


def check_rows(x, y, direction, rows):
    want = oracle.fft(x[rows], inverse=(direction == fg.FFT_INVERSE), nthreads=NTHREADS)
    err = rel_l2_rows(y[rows], want)
    assert err.max() <= TOL_FP32, f"max rel L2 {err.max():.3e}"


def test_configs_are_listed():
    for N in (4096, 16384, 65536):
        cfgs = l2_configs(N)
        assert cfgs, N
        for c in cfgs:
            assert c["path"] == fg.FFT_PATH_FOURSTEP and c["n1"] ** 2 == N
    assert not l2_configs(8192) and not l2_configs(32768)   # n1 != n2


@pytest.mark.parametrize("N", [4096, 16384, 65536])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_ring_reuse_matches_oracle_and_two_launch_fourstep(N, direction):
    for cfg in l2_configs(N):
        R = cfg["l2_chunk_rows"]
        probe = fg.Plan(N, 1, direction, config=cfg)
        grid = probe.info()["grid_ctas"]
        probe.close()
        batch = ring_batch(N, R, grid)
        x = synth.gaussian((batch, N), seed=N + R + direction)
        plan = fg.Plan(N, batch, direction, config=cfg)
        info = plan.info()
        assert info["l2_chunk_rows"] == R and info["n1"] * info["n2"] == N
        xd = to_dev(x)
        y = to_host(plan(xd))
        # rows at chunk edges, the ragged tail and a random sample
        rng = np.random.Generator(np.random.PCG64(R))
        edges = [r for c in range(0, batch, R) for r in (c, c + R - 1) if r < batch]
        rows = np.unique(np.concatenate([edges, [batch - 1], rng.integers(0, batch, 24)]))
        if N <= 16384:
            rows = np.arange(batch)
        check_rows(x, y, direction, rows)
        # the two-launch four-step with the same split computes the same values
        two = dict(cfg, l2_chunk_rows=0, ctas_per_sm=0)
        ref_plan = fg.Plan(N, batch, direction, config=two)
        ref = to_host(ref_plan(xd))
        ref_plan.close()
        assert rel_l2_rows(y, ref).max() <= 1e-6
        # repeated launches: the counters clear themselves, results are bitwise equal
        for _ in range(2):
            again = to_host(plan(xd))
            assert np.array_equal(again.view(np.uint32), y.view(np.uint32))
        assert plan.device_status() == 0
        plan.close()


@pytest.mark.parametrize("batch", [1, 3, 8, 9, 33])
def test_small_batches(batch):
    # fewer chunks than ring slots, single partial chunk, exact multiples
    N = 16384
    for cfg in l2_configs(N):
        x = synth.gaussian((batch, N), seed=batch)
        plan = fg.Plan(N, batch, fg.FFT_FORWARD, config=cfg)
        y = to_host(plan(to_dev(x)))
        plan.close()
        check_rows(x, y, fg.FFT_FORWARD, np.arange(batch))


def test_in_place_and_host_buffers():
    N = 16384
    cfg = l2_configs(N)[0]
    batch = 700     # several 32 MiB staging chunks through the host path
    x = synth.gaussian((batch, N), seed=5)
    plan = fg.Plan(N, batch, fg.FFT_FORWARD, config=cfg)
    dev = to_host(plan(to_dev(x)))
    xd = to_dev(x)
    plan(xd, out=xd)    # in place: phase 2 of a chunk starts after its phase 1 read it
    assert np.array_equal(to_host(xd).view(np.uint32), dev.view(np.uint32))
    host = plan.exec_host(torch.from_numpy(x).pin_memory()).numpy()
    plan.close()
    assert np.array_equal(host.view(np.uint32), dev.view(np.uint32))
    check_rows(x, dev, fg.FFT_FORWARD, np.array([0, 1, 350, 699]))


def test_plan_rejects_bad_chunk_rows():
    N = 16384
    cfg = l2_configs(N)[0]
    for bad in (-1, 4097):
        with pytest.raises(fg.FFTError):
            fg.Plan(N, 4, fg.FFT_FORWARD, config=dict(cfg, l2_chunk_rows=bad))
    with pytest.raises(fg.FFTError):   # n1 != n2 has no single-launch kernel
        c8 = [c for c in fg.fft_list_configs(8192) if c["path"] == fg.FFT_PATH_FOURSTEP][0]
        fg.Plan(8192, 4, fg.FFT_FORWARD, config=dict(c8, l2_chunk_rows=16))
