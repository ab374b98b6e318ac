"""Cluster-split kernel (a row on a cluster of K CTAs) against the FP64 oracle.

The kernel computes the four-step with N1 = K (paper Sec. IV-B, Eq. 3): each
CTA transforms the stride-K subsequence of a row, multiplies by W_N^{r k2},
and the cluster combines with K-point DFTs through distributed shared memory.
Clusters are persistent over rows, so batches larger than the resident
clusters run the row loop several times with a ragged last round.
"""
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


def cluster_configs():
    out = []
    for N in (8192, 16384, 32768, 65536):
        for cfg in fg.fft_list_configs(N):
            if cfg["cluster_split"]:
                out.append((N, cfg))
    return out


CFGS = cluster_configs()
IDS = [f"N{N}-K{c['cluster_split']}-twm{c['twiddle_mode']}" for N, c in CFGS]


def check(x, y, direction):
    want = oracle.fft(x, inverse=direction > 0, nthreads=NTHREADS)
    err = rel_l2_rows(y, want)
    assert err.max() <= TOL_FP32, f"max rel L2 {err.max():.3e}"


def test_cluster_configs_are_listed():
    ks = {(N, c["cluster_split"]) for N, c in CFGS}
    assert (32768, 2) in ks and (65536, 4) in ks and (16384, 2) in ks


@pytest.mark.parametrize("N,cfg", CFGS, ids=IDS)
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_several_rounds_ragged_last(N, cfg, direction):
    K = cfg["cluster_split"]
    probe = fg.Plan(N, 1, direction, config=cfg)
    info = probe.info()
    probe.close()
    assert info["cluster_split"] == K and info["grid_ctas"] % K == 0
    clusters = info["grid_ctas"] // K
    assert clusters > 0
    batch = 2 * clusters + 5          # two full rounds and a ragged third
    x = synth.gaussian((batch, N), seed=N + K + direction)
    plan = fg.Plan(N, batch, direction, config=cfg)
    y = to_host(plan(to_dev(x)))
    plan.close()
    check(x, y, direction)


@pytest.mark.parametrize("N,cfg", CFGS, ids=IDS)
def test_single_row_in_place_and_determinism(N, cfg):
    x = synth.gaussian((1, N), seed=5)
    plan = fg.Plan(N, 1, fg.FFT_FORWARD, config=cfg)
    xd = to_dev(x)
    a = to_host(plan(xd))
    b = to_host(plan(xd))
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    plan(xd, out=xd)                  # in place: every load of a row precedes its stores
    assert np.array_equal(to_host(xd).view(np.uint32), a.view(np.uint32))
    plan.close()
    check(x, a, fg.FFT_FORWARD)


def test_empty_batch_and_closed_forms():
    N = 32768
    cfg = next(c for c in fg.fft_list_configs(N) if c["cluster_split"] == 2)
    plan = fg.Plan(N, 0, fg.FFT_FORWARD, config=cfg)
    assert plan.info()["cluster_split"] == 2
    assert fg.lib().fft_exec(plan.handle, None, None, None) == 0   # nothing to do
    plan.close()
    # impulse -> all ones; constant -> N at bin 0 (exact in FP32)
    x = np.zeros((2, N), np.complex64)
    x[0, 0] = 1
    x[1, :] = 1
    plan = fg.Plan(N, 2, fg.FFT_FORWARD, config=cfg)
    y = to_host(plan(to_dev(x)))
    plan.close()
    assert np.array_equal(y[0], np.ones(N, np.complex64))
    want = np.zeros(N, np.complex64)
    want[0] = N
    assert np.abs(y[1] - want).max() <= 1e-3
