"""16-bit-storage FFT (4 bytes per point in HBM, FP32 arithmetic) against the
FP64 oracle applied to the same 16-bit inputs widened exactly.

The error is set by the final rounding to the storage type: about
2^-11 / sqrt(3) ~ 3e-4 relative RMS per element for FP16 (bound 1e-3 per
transform) and 2^-8 / sqrt(3) ~ 2.3e-3 for BF16 (bound 5e-3)."""
import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, rel_l2_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL_FP16_STORAGE = 1e-3
TOL_BF16_STORAGE = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


def to_half_pairs(x: np.ndarray) -> np.ndarray:
    h = np.empty(x.shape + (2,), np.float16)
    h[..., 0] = x.real
    h[..., 1] = x.imag
    return h


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192, 16384])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_fp16_storage_matches_oracle(N, direction):
    batch = 33
    x = synth.gaussian((batch, N), seed=N + 3)
    xh = to_half_pairs(x)
    xin = xh[..., 0].astype(np.float64) + 1j * xh[..., 1].astype(np.float64)
    dev = torch.from_numpy(xh).cuda().view(torch.complex32).reshape(batch, N)
    plan = fg.Plan(N, batch, direction, precision=fg.FFT_PREC_FP16_STORAGE)
    y = plan(dev)
    torch.cuda.synchronize()
    plan.close()
    yh = y.view(torch.float16).reshape(batch, N, 2).cpu().numpy().astype(np.float64)
    got = yh[..., 0] + 1j * yh[..., 1]
    want = oracle.fft(xin, inverse=direction > 0, nthreads=NTHREADS)
    err = rel_l2_rows(got, want)
    print(f"\nFP16 storage N={N} {'inv' if direction > 0 else 'fwd'}: max rel L2 {err.max():.3e}")
    assert np.isfinite(got).all()
    assert err.max() <= TOL_FP16_STORAGE


def test_fp16_storage_rejects_small_n():
    with pytest.raises(fg.FFTError):
        fg.Plan(64, 4, fg.FFT_FORWARD, precision=fg.FFT_PREC_FP16_STORAGE)


def to_bf16_pairs(x: np.ndarray):
    """Interleaved (re, im) as a torch.bfloat16 tensor, and the exact values."""
    t = torch.from_numpy(np.stack([x.real, x.imag], -1).astype(np.float32)).to(torch.bfloat16)
    back = t.to(torch.float64).numpy()
    return t, back[..., 0] + 1j * back[..., 1]


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192, 16384])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_bf16_storage_matches_oracle(N, direction):
    batch = 33
    x = synth.gaussian((batch, N), seed=N + 5)
    t, xin = to_bf16_pairs(x)
    plan = fg.Plan(N, batch, direction, precision=fg.FFT_PREC_BF16_STORAGE)
    assert plan.dtype == torch.bfloat16
    y = plan(t.cuda().reshape(-1))
    torch.cuda.synchronize()
    plan.close()
    yb = y.to(torch.float64).cpu().numpy().reshape(batch, N, 2)
    got = yb[..., 0] + 1j * yb[..., 1]
    want = oracle.fft(xin, inverse=direction > 0, nthreads=NTHREADS)
    err = rel_l2_rows(got, want)
    print(f"\nBF16 storage N={N} {'inv' if direction > 0 else 'fwd'}: max rel L2 {err.max():.3e}")
    assert np.isfinite(got).all()
    assert err.max() <= TOL_BF16_STORAGE


def test_bf16_storage_wrong_dtype_and_size():
    plan = fg.Plan(256, 4, fg.FFT_FORWARD, precision=fg.FFT_PREC_BF16_STORAGE)
    with pytest.raises(TypeError):
        plan(torch.zeros(4 * 256, dtype=torch.complex32, device="cuda"))
    with pytest.raises(ValueError):   # two elements per point
        plan(torch.zeros(4 * 256, dtype=torch.bfloat16, device="cuda"))
    plan.close()
