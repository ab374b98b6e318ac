"""Parity of the CUDA FFT path (through the C ABI) with the FP64 oracle.

The bar (paper Sec. II-A definition; tolerance from the target): every
transform's relative L2 error against the oracle is at most 5e-6.  Inputs are
the seeded generators; the oracle runs on the same float32 values widened
exactly to float64.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL_N = [1 << e for e in range(1, 15)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def run(x: np.ndarray, direction: int, config=None, flags=0, out=None):
    N = x.shape[-1]
    batch = x.size // N
    plan = fg.Plan(N, batch, direction, flags=flags, config=config)
    xd = to_dev(x)
    y = plan(xd, out=out)
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    return to_host(y).reshape(x.shape), info


def check(x, y, direction, tol=TOL_FP32):
    want = oracle.fft(x, inverse=(direction == fg.FFT_INVERSE), nthreads=NTHREADS)
    err = rel_l2_rows(y, want)
    assert err.max() <= tol, f"max rel L2 {err.max():.3e} (median {np.median(err):.3e})"
    return err


@pytest.mark.parametrize("N", ALL_N)
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_default_plan_matches_oracle(N, direction):
    batch = max(3, min(257, (1 << 16) // N))  # spans several CTAs and a ragged tail
    x = synth.gaussian((batch, N), seed=N + direction)
    y, info = run(x, direction)
    check(x, y, direction)


@pytest.mark.parametrize("N", [64, 256, 512, 1024, 2048, 4096, 8192, 16384])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_every_compiled_config_matches_oracle(N, direction):
    cfgs = fg.fft_list_configs(N)
    assert cfgs
    for cfg in cfgs:
        tb = max(cfg["transforms_per_cta"], 1)
        batch = 2 * tb + 1 if cfg["path"] == fg.FFT_PATH_SINGLE_CTA else 5
        x = synth.gaussian((batch, N), seed=7 * N + cfg["points_per_thread"] + cfg["n1"])
        y, info = run(x, direction, config=cfg)
        assert info["path"] == cfg["path"]
        check(x, y, direction)


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192, 16384])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_persistent_configs_over_several_rounds_of_tiles(N, direction):
    """Every persistent single-CTA configuration with each CTA taking at least
    two tiles and a partial last tile: the epilogue that loads a CTA's next
    tile while it stores the current one runs on every round but the last.
    Rows of the second round and of the tail are checked against the oracle,
    every row for being finite."""
    cfgs = [c for c in fg.fft_list_configs(N)
            if c["path"] == fg.FFT_PATH_SINGLE_CTA and c["ctas_per_sm"] == -1
            and not c["tma_slabs"] and not c["cluster_split"]]
    assert cfgs
    for cfg in cfgs:
        tb = cfg["transforms_per_cta"]
        probe = fg.Plan(N, 1, direction, config=cfg)
        G = probe.info()["grid_ctas"]
        probe.close()
        assert G > 0
        batch = 2 * G * tb + tb + max(1, tb // 2)   # two full rounds, a third partial round
        x = synth.gaussian((batch, N), seed=11 * N + cfg["points_per_thread"] + tb)
        y, info = run(x, direction, config=cfg)
        assert info["grid_ctas"] == G and np.isfinite(y).all()
        rng = np.random.Generator(np.random.PCG64(N + tb))
        second = np.arange(G * tb, G * tb + min(4 * tb, 64))        # round two, first CTAs
        tail = np.arange(max(0, batch - 2 * tb - 3), batch)        # last tiles, partial tile
        rows = np.unique(np.concatenate([second, tail, rng.integers(G * tb, batch, 24)]))
        check(x[rows], y[rows], direction)


@pytest.mark.parametrize("N", [512, 1024, 2048, 4096, 8192, 16384, 32768])
def test_full_size_sampled_rows(N):
    # the benchmark's size: 2^25 points (256 MiB) per call, batch = 2^25 / N
    batch = (1 << 25) // N
    x = synth.gaussian((batch, N), seed=0)
    plan = fg.Plan(N, batch, fg.FFT_FORWARD)
    y = to_host(plan(to_dev(x)))
    plan.close()
    rng = np.random.Generator(np.random.PCG64(N))
    rows = np.unique(np.concatenate([[0, 1, batch - 1], rng.integers(0, batch, 13)]))
    check(x[rows], y[rows], fg.FFT_FORWARD)
    assert np.isfinite(y).all()


@pytest.mark.parametrize("N", [1024, 8192, 16384])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_chirp_input(N, direction):
    x = synth.lfm_chirp(33, N, seed=1)
    y, _ = run(x, direction)
    check(x, y, direction)


@pytest.mark.parametrize("N", [8192, 16384])
def test_fourstep_and_single_cta_agree(N):
    x = synth.gaussian((9, N), seed=3)
    a, ia = run(x, fg.FFT_FORWARD, flags=fg.FFT_FLAG_FORCE_SINGLE_CTA)
    b, ib = run(x, fg.FFT_FORWARD, flags=fg.FFT_FLAG_FORCE_FOURSTEP)
    assert ia["path"] == fg.FFT_PATH_SINGLE_CTA and ib["path"] == fg.FFT_PATH_FOURSTEP
    assert ib["n1"] * ib["n2"] == N
    check(x, a, fg.FFT_FORWARD)
    check(x, b, fg.FFT_FORWARD)
    assert rel_l2_rows(a, b).max() <= 2 * TOL_FP32


@pytest.mark.parametrize("N", [16, 256, 4096, 16384])
def test_impulse_and_constant(N):
    d = np.zeros((2, N), np.complex64)
    d[:, 0] = 1
    y, _ = run(d, fg.FFT_FORWARD)
    assert np.max(np.abs(y - 1)) <= 1e-6
    c = np.ones((2, N), np.complex64)
    y, _ = run(c, fg.FFT_FORWARD)
    want = np.zeros((2, N))
    want[:, 0] = N
    assert np.max(np.abs(y - want)) <= 1e-6 * N


@pytest.mark.parametrize("N", [256, 4096, 16384])
def test_round_trip(N):
    x = synth.gaussian((5, N), seed=11)
    X, _ = run(x, fg.FFT_FORWARD)
    xr, _ = run(X, fg.FFT_INVERSE)
    assert rel_l2_rows(xr, x).max() <= 2 * TOL_FP32


@pytest.mark.parametrize("N", [256, 8192])
def test_unnormalized_inverse_and_adjoint_flags(N):
    x = synth.gaussian((3, N), seed=12)
    y, _ = run(x, fg.FFT_INVERSE, flags=fg.FFT_FLAG_UNNORMALIZED_INVERSE)
    check(x, y / N, fg.FFT_INVERSE)
    # adjoint of forward = unnormalised inverse; adjoint of inverse = forward / N
    a, _ = run(x, fg.FFT_FORWARD, flags=fg.FFT_FLAG_ADJOINT)
    check(x, a / N, fg.FFT_INVERSE)
    b, _ = run(x, fg.FFT_INVERSE, flags=fg.FFT_FLAG_ADJOINT)
    check(x, b * N, fg.FFT_FORWARD)
    # dot-product test <F x, v> = <x, F^H v> entirely on the GPU path
    v = synth.gaussian((3, N), seed=13)
    Fx, _ = run(x, fg.FFT_FORWARD)
    FHv, _ = run(v, fg.FFT_FORWARD, flags=fg.FFT_FLAG_ADJOINT)
    lhs = np.vdot(v.astype(np.complex128), Fx.astype(np.complex128))
    rhs = np.vdot(FHv.astype(np.complex128), x.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("N", [256, 16384])
def test_in_place(N):
    x = synth.gaussian((7, N), seed=14)
    xd = to_dev(x)
    plan = fg.Plan(N, 7, fg.FFT_FORWARD)
    plan(xd, out=xd)
    torch.cuda.synchronize()
    plan.close()
    check(x, to_host(xd), fg.FFT_FORWARD)


@pytest.mark.parametrize("flags", [0, fg.FFT_FLAG_FORCE_FOURSTEP])
def test_nan_poison_and_guard_canaries(flags):
    # every output element written, nothing written outside the output
    N, batch, G = 8192, 5, 4096
    x = synth.gaussian((batch, N), seed=15)
    buf = torch.full((batch * N + 2 * G,), float("nan"), dtype=torch.complex64, device="cuda")
    canary = torch.full((G,), complex(123.25, -7.5), dtype=torch.complex64, device="cuda")
    buf[:G] = canary
    buf[-G:] = canary
    out = buf[G:G + batch * N]
    plan = fg.Plan(N, batch, fg.FFT_FORWARD, flags=flags)
    plan(to_dev(x).reshape(-1), out=out)
    torch.cuda.synchronize()
    plan.close()
    assert torch.equal(buf[:G], canary) and torch.equal(buf[-G:], canary)
    y = to_host(out).reshape(batch, N)
    assert np.isfinite(y).all()
    check(x, y, fg.FFT_FORWARD)


def test_batch_zero_and_argument_errors():
    plan = fg.Plan(256, 0, fg.FFT_FORWARD)
    L = fg.lib()
    assert L.fft_exec(plan.handle, None, None, None) == 0     # nothing to do
    plan.close()
    plan = fg.Plan(256, 4, fg.FFT_FORWARD)
    buf = torch.zeros(4 * 256 + 8, dtype=torch.complex64, device="cuda")
    p = buf.data_ptr()
    assert L.fft_exec(plan.handle, p + 8, p + 8, None) == 3       # misaligned
    assert L.fft_exec(plan.handle, p, p + 16, None) == 2          # partial overlap
    assert L.fft_exec(plan.handle, p, None, None) == 2
    assert L.fft_exec(plan.handle, p, p, None) == 0               # in place is fine
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    plan.close()


@pytest.mark.parametrize("N", [64, 1024, 16384])
def test_twiddle_tables_round_fp64_angles(N):
    for flags in (0, fg.FFT_FLAG_FORCE_FOURSTEP):
        if flags and N < 256:
            continue
        plan = fg.Plan(N, 1, fg.FFT_FORWARD, flags=flags)
        tab = fg.fft_twiddle_table(plan.handle)
        M = np.empty(tab.size, np.int64)
        e = np.empty(tab.size, np.int64)
        for i in range(tab.size):
            M[i], e[i] = fg.fft_twiddle_index(plan.handle, i)
        plan.close()
        want = exact_root(M, e).astype(np.complex64)  # FP64, rounded to FP32
        ulp_re = np.abs(tab.real.view(np.int32).astype(np.int64) - want.real.view(np.int32))
        ulp_im = np.abs(tab.imag.view(np.int32).astype(np.int64) - want.imag.view(np.int32))
        # +-0 differ in bits but not in value
        ulp_re[(tab.real == 0) & (want.real == 0)] = 0
        ulp_im[(tab.imag == 0) & (want.imag == 0)] = 0
        assert max(ulp_re.max(), ulp_im.max()) <= 1
        assert np.mean((ulp_re == 0) & (ulp_im == 0)) >= 0.999


def exact_root(M, e):
    """exp(-2 pi i e / M) in FP64 with the angle reduced to the first octant by
    exact symmetries, so quarter and half turns give exact 0 and +-1."""
    e = np.asarray(e, np.int64) % M
    M = np.asarray(M, np.int64)
    # angle fraction f = e / M in [0, 1); work with 8 e = octant * M + rem
    e8 = 8 * e
    octant = e8 // M
    rem = (e8 - octant * M).astype(np.float64) / M.astype(np.float64)  # in [0, 1)
    th = rem * (np.pi / 4)                                           # in [0, pi/4)
    c0, s0 = np.cos(th), np.sin(th)
    cp, sp = np.cos(np.pi / 4 - th), np.sin(np.pi / 4 - th)
    # cos/sin of (octant * pi/4 + th) via the octant symmetries
    tbl = {0: (c0, s0), 1: (sp, cp), 2: (-s0, c0), 3: (-cp, sp),
           4: (-c0, -s0), 5: (-sp, -cp), 6: (s0, -c0), 7: (cp, -sp)}
    c = np.empty(e.shape)
    s = np.empty(e.shape)
    for o, (co, so) in tbl.items():
        mask = octant == o
        c[mask] = co[mask]
        s[mask] = so[mask]
    return c - 1j * s


@pytest.mark.gpu
def test_exact_root_reference_is_the_root():
    M = np.array([8, 16, 1024, 16384, 96])
    for m in M:
        e = np.arange(m)
        np.testing.assert_allclose(exact_root(np.full(m, m), e), np.exp(-2j * np.pi * e / m),
                                   atol=1e-15)
    assert exact_root(np.array([4]), np.array([1]))[0] == -1j
    assert exact_root(np.array([8]), np.array([4]))[0] == -1


def test_bitwise_determinism():
    x = synth.gaussian((64, 4096), seed=16)
    a, _ = run(x, fg.FFT_FORWARD)
    b, _ = run(x, fg.FFT_FORWARD)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("N,flags", [(4096, 0), (16384, 0), (16384, fg.FFT_FLAG_FORCE_FOURSTEP)])
def test_host_buffer_exec_matches_device_exec(N, flags):
    batch = 3000 if N == 4096 else 700   # several 32 MiB staging chunks
    x = synth.gaussian((batch, N), seed=17)
    plan = fg.Plan(N, batch, fg.FFT_FORWARD, flags=flags)
    dev = to_host(plan(to_dev(x)))
    xh = torch.from_numpy(x).pin_memory()
    host = plan.exec_host(xh).numpy()
    plan.close()
    assert np.array_equal(dev.view(np.uint32), host.view(np.uint32))
    check(x[:4], host[:4], fg.FFT_FORWARD)


@pytest.mark.parametrize("N", [1 << e for e in range(15, 21)])
@pytest.mark.parametrize("direction", [fg.FFT_FORWARD, fg.FFT_INVERSE])
def test_beyond_one_cta(N, direction):
    # N > 16384: the two-phase four-step (phase 1 <= 512 points, phase 2 <=
    # 4096), also forced; every listed configuration (four-step splits,
    # cluster rows, halves in tensor memory), ragged CTA tail included.  The
    # default is the one-pass kernel with half of each row in tensor memory
    # at 32768, the four-step above (phase 1 of 256 points up to 2^17, of 512
    # beyond).
    cfgs = fg.fft_list_configs(N)
    assert cfgs
    x = synth.gaussian((3, N), seed=N)
    y, info = run(x, direction)
    if N == 1 << 15:
        assert info["path"] == fg.FFT_PATH_TMEM_HALVES and info["n1"] == 0
    else:
        assert info["path"] == fg.FFT_PATH_FOURSTEP and info["n1"] * info["n2"] == N
        assert info["n2"] == (256 if N <= 1 << 17 else 512)
    check(x, y, direction)
    y, info = run(x, direction, flags=fg.FFT_FLAG_FORCE_FOURSTEP)
    assert info["path"] == fg.FFT_PATH_FOURSTEP and info["n1"] * info["n2"] == N
    check(x, y, direction)
    for cfg in cfgs:
        y, info = run(x[:2], direction, config=cfg)
        assert info["n1"] == cfg["n1"] and info["cluster_split"] == cfg["cluster_split"]
        check(x[:2], y, direction)


@pytest.mark.parametrize("N,batch", [(4096, 3000), (16384, 1000), (32768, 400)])
def test_dependent_calls_back_to_back(N, batch):
    # Kernels launched with programmatic dependent launch may become resident
    # while the previous kernel of the stream runs; each call here reads the
    # previous call's output with no host synchronisation in between (forward,
    # inverse, forward, inverse, in place on the second buffer), so a kernel
    # that touched memory before the previous one completed would be caught.
    x = synth.gaussian((batch, N), seed=21)
    a = to_dev(x)
    b = torch.empty_like(a)
    fwd, inv = fg.Plan(N, batch, fg.FFT_FORWARD), fg.Plan(N, batch, fg.FFT_INVERSE)
    fwd(a, out=b)
    inv(b, out=b)
    fwd(b, out=a)
    inv(a, out=b)
    X = to_host(a)
    y = to_host(b)
    torch.cuda.synchronize()
    fwd.close()
    inv.close()
    rows = np.array([0, 1, batch // 2, batch - 1])
    check(x[rows], X[rows], fg.FFT_FORWARD, tol=4 * TOL_FP32)
    assert rel_l2_rows(y, x).max() <= 4 * TOL_FP32
