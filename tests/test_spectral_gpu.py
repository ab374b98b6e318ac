"""Differentiable spectral filter (SAR range compression) and FFT autograd on
the GPU path, against the oracle's analytic gradient (itself pinned to FP64
central differences in test_oracle.py)."""
import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, TOL_GRAD, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


def rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def sar_case(rows, N, Np, seed=0):
    x, pulse = synth.sar_echoes(rows, N, Np=Np, seed=seed)
    H = np.conj(oracle.fft(pulse)).astype(np.complex64)
    m = synth.real_mask((rows, N), seed=2)
    return x, H, m


def gpu_filter_grads(x, H, m, fused=True):
    xd = to_dev(x).requires_grad_(True)
    layer = fg.SpectralFilter(to_dev(H), fused=fused)
    y = layer(xd)
    md = to_dev(m)
    loss = (md * (y.real ** 2 + y.imag ** 2)).sum()
    loss.backward()
    torch.cuda.synchronize()
    return to_host(y), to_host(xd.grad), to_host(layer.H.grad), float(loss.detach())


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("rows,N,Np", [(4, 256, 64), (37, 1024, 256), (64, 8192, 2048),
                                       (3, 16384, 4096)])
def test_spectral_filter_forward_and_grads_match_oracle(rows, N, Np, fused):
    x, H, m = sar_case(rows, N, Np)
    y, gx, gH, loss = gpu_filter_grads(x, H, m, fused=fused)
    want_y = oracle.spectral_filter_forward(x, H)
    assert rel_l2_rows(y, want_y).max() <= 2 * TOL_FP32
    ogx, ogH = oracle.spectral_filter_grads(x, H, m)
    assert rel(gx, ogx) <= TOL_GRAD
    assert rel(gH, ogH) <= TOL_GRAD
    assert abs(loss - oracle.spectral_filter_loss(x, H, m)) <= 1e-5 * abs(loss)


@pytest.mark.parametrize("fused", [True, False])
def test_spectral_filter_grad_h_is_bitwise_reproducible(fused):
    x, H, m = sar_case(100, 1024, 256, seed=4)
    _, _, g1, _ = gpu_filter_grads(x, H, m, fused)
    _, _, g2, _ = gpu_filter_grads(x, H, m, fused)
    assert np.array_equal(g1.view(np.uint32), g2.view(np.uint32))


@pytest.mark.parametrize("N", [256, 512, 2048, 4096, 8192, 16384])
def test_fused_filter_abi_conj_and_saved_spectrum(N):
    # through the C ABI: conj_h, the saved spectrum, and an odd row count
    rows = 7
    x = synth.gaussian((rows, N), seed=N)
    H = synth.gaussian(N, seed=N + 1)
    plan = fg.fft_filter_plan(N, rows)
    xd, Hd = to_dev(x), to_dev(H)
    y = torch.empty_like(xd)
    X = torch.empty_like(xd)
    st = torch.cuda.current_stream()
    fg.fft_filter_forward(plan, xd, Hd, y, X, True, st)
    torch.cuda.synchronize()
    fg.fft_destroy(plan)
    want_X = oracle.fft(x)
    want_y = oracle.ifft(want_X * np.conj(H.astype(np.complex128)))
    assert rel_l2_rows(to_host(X), want_X).max() <= TOL_FP32
    assert rel_l2_rows(to_host(y), want_y).max() <= 2 * TOL_FP32


@pytest.mark.parametrize("N", [256, 16384])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft_autograd_uses_the_adjoint(N, inverse):
    # L = sum m |T x|^2  ->  grad_x = T^H (2 m T x), T = F or G
    x = synth.gaussian((3, N), seed=5)
    m = synth.real_mask((3, N), seed=6)
    xd = to_dev(x).requires_grad_(True)
    y = fg.fft(xd, inverse=inverse)
    loss = (to_dev(m) * (y.real ** 2 + y.imag ** 2)).sum()
    loss.backward()
    g = to_host(xd.grad)
    Tx = oracle.fft(x, inverse=inverse)
    gy = 2.0 * m * Tx
    want = N * oracle.ifft(gy) if not inverse else oracle.fft(gy) / N
    assert rel(g, want) <= TOL_GRAD


@pytest.mark.parametrize("batch", [1, 33, 32 * 700 + 17, 32 * 4096 + 5])
def test_grad_h_reduction_both_tree_forms(batch):
    # grad_H = sum_rows conj(X) * G: 32-row chunk sums, then a pairwise tree
    # over the chunks (one launch, 8-chunk blocks in registers and the rest in
    # shared memory, up to 4096 chunks; level by level above); checked against
    # the FP64 sum and bitwise run to run
    N = 64
    X = synth.gaussian((batch, N), seed=batch)
    G = synth.gaussian((batch, N), seed=batch + 1)
    Xd, Gd = to_dev(X), to_dev(G)
    work = torch.empty(fg.fft_filter_grad_h_workspace(N, batch) // 8, dtype=torch.complex64,
                       device="cuda")
    st = torch.cuda.current_stream()
    out = []
    for _ in range(2):
        gH = torch.empty(N, dtype=torch.complex64, device="cuda")
        fg.fft_filter_grad_h(Xd, Gd, gH, N, batch, work, st)
        out.append(to_host(gH))
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))
    terms = np.conj(X.astype(np.complex128)) * G.astype(np.complex128)
    want = terms.sum(0)
    scale = np.abs(terms).sum(0)
    assert (np.abs(out[0] - want) / scale).max() <= 1e-6


@pytest.mark.parametrize("N", [4096, 8192])
def test_filter_plan_rejects_aliased_buffers(N):
    # host-side checks before any launch: grad_x holds g_z between the
    # backward's kernels, and from 8192 on X_save holds the forward's spectrum
    rows = 3
    plan = fg.fft_filter_plan(N, rows)
    L = fg.lib()
    a = torch.zeros(rows * N, dtype=torch.complex64, device="cuda")
    b = torch.zeros_like(a)
    c = torch.zeros_like(a)
    H = torch.ones(N, dtype=torch.complex64, device="cuda")
    gH = torch.empty_like(H)
    pa, pb, pc, ph, pg = a.data_ptr(), b.data_ptr(), c.data_ptr(), H.data_ptr(), gH.data_ptr()
    assert L.fft_filter_backward(plan, pa, ph, pb, pa, pg, None) == 2   # grad_x is g_y
    assert L.fft_filter_backward(plan, pa, ph, pb, pb, pg, None) == 2   # grad_x is X_saved
    assert L.fft_filter_backward(plan, pa, ph, pb, pc, pg, None) == 0
    if N >= 8192:
        assert L.fft_filter_forward(plan, pa, ph, pb, pa, 0, None) == 2  # X_save is x
        assert L.fft_filter_forward(plan, pa, ph, pb, pb, 0, None) == 2  # X_save is y
    assert L.fft_filter_forward(plan, pa, ph, pa, pc, 0, None) == 0      # y may be x
    torch.cuda.synchronize()
    fg.fft_destroy(plan)
