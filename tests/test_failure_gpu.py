"""Error paths through the C ABI, reached without any GPU fault, trap or hang.

- A bounded device wait on something that never arrives (the mbarrier wait of
  the bulk-copy kernels, the counter wait of the single-launch four-step)
  gives up after its limit and reports FFT_ERR_TIMEOUT; the context stays
  usable and the next transform is correct.
- An allocation failure injected at every allocation of every kind of plan
  creation (and of the host-buffer staging) comes back as FFT_ERR_ALLOC with
  a NULL plan and nothing leaked; the next real creation succeeds.
"""
import ctypes
import time

import numpy as np
import pytest

import oracle
import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import synth
from gpu_util import NTHREADS, TOL_FP32, rel_l2_rows, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OK, INVALID_VALUE, ALLOC, TIMEOUT = 0, 2, 4, 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_27569_gb300 import build

    build.build()


@pytest.fixture(autouse=True)
def _disarm():
    fg.fft_debug_fail_alloc(-1)
    yield
    fg.fft_debug_fail_alloc(-1)


def transform_ok(seed):
    x = synth.gaussian((4, 1024), seed=seed)
    plan = fg.Plan(1024, 4, fg.FFT_FORWARD)
    y = to_host(plan(to_dev(x)))
    plan.close()
    return rel_l2_rows(y, oracle.fft(x, nthreads=NTHREADS)).max() <= TOL_FP32


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_times_out_and_the_context_stays_usable(kind):
    t0 = time.perf_counter()
    assert fg.fft_debug_bounded_wait(kind, 20000) == TIMEOUT  # 20 ms limit
    assert 0.019 <= time.perf_counter() - t0 < 10.0
    assert transform_ok(kind)
    assert fg.fft_debug_bounded_wait(2, 1000) == INVALID_VALUE
    assert fg.fft_debug_bounded_wait(kind, 0) == INVALID_VALUE


def ragged_args(count=300):
    d = synth.ragged_draw(count, seed=5)
    N = np.ascontiguousarray(d["N"], np.int32)
    dr = np.ascontiguousarray(d["direction"], np.int32)
    off = np.ascontiguousarray(d["offset"], np.int64)
    return N, dr, off


def creators():
    L = fg.lib()
    N, dr, off = ragged_args()
    return {
        "plain 4096": lambda h: L.fft_plan_ex(ctypes.byref(h), 4096, 64, -1, 0, 0),
        "four-step 65536 (scratch)": lambda h: L.fft_plan_ex(ctypes.byref(h), 65536, 512, -1, 0,
                                                             fg.FFT_FLAG_FORCE_FOURSTEP),
        "tmem halves 32768": lambda h: L.fft_plan_ex(ctypes.byref(h), 32768, 8, 1, 0, 0),
        "tensor core 4096": lambda h: L.fft_plan_ex(ctypes.byref(h), 4096, 64, -1,
                                                    fg.FFT_PREC_FP16X2, 0),
        "filter 8192": lambda h: L.fft_filter_plan(ctypes.byref(h), 8192, 64),
        "columns 1024": lambda h: L.fft_plan_columns(ctypes.byref(h), 1024, 256, 2, 256,
                                                     1024 * 256, -1, 0),
        "ragged": lambda h: L.fft_ragged_plan(
            ctypes.byref(h), len(N), N.ctypes.data, dr.ctypes.data, off.ctypes.data,
            off.ctypes.data, fg.FFT_FLAG_NO_AUTOTUNE_CACHE),
        # a failure inside the tuning runs is not an error: the class keeps
        # its built-in routine and the creation goes on
        "ragged (autotuned)": lambda h: L.fft_ragged_plan(
            ctypes.byref(h), len(N), N.ctypes.data, dr.ctypes.data, off.ctypes.data,
            off.ctypes.data, fg.FFT_FLAG_RAGGED_AUTOTUNE | fg.FFT_FLAG_NO_AUTOTUNE_CACHE),
    }


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("name", sorted(creators()))
def test_injected_allocation_failures(name):
    make = creators()[name]
    before = free_bytes()
    for _ in range(2):
        failures = 0
        for k in range(64):
            fg.fft_debug_fail_alloc(k)
            h = ctypes.c_void_p(1234)
            rc = make(h)
            fg.fft_debug_fail_alloc(-1)
            if rc == ALLOC:
                assert not h.value, "a failed creation returns no plan"
                failures += 1
                continue
            assert rc == OK, fg.STATUS.get(rc, rc)
            assert h.value
            assert fg.lib().fft_destroy(h) == OK
            break
        else:
            pytest.fail("creation never succeeded")
        assert failures >= 1  # every creation allocates
    # nothing leaked: a leaked twiddle table, scratch or workspace (up to
    # hundreds of MiB here) would show; allocator granularity is ~2 MiB
    assert before - free_bytes() < 8 << 20
    assert transform_ok(7)


def test_host_buffer_staging_failure():
    N, batch = 4096, 64
    x = synth.gaussian((batch, N), seed=8)
    plan = fg.Plan(N, batch, fg.FFT_FORWARD)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    fg.fft_debug_fail_alloc(0)  # the staging buffers of the first host exec
    rc = fg.lib().fft_exec_host(plan.handle, xh.data_ptr(), yh.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    fg.fft_debug_fail_alloc(-1)
    assert rc == ALLOC
    rc = fg.lib().fft_exec_host(plan.handle, xh.data_ptr(), yh.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == OK
    torch.cuda.synchronize()
    assert rel_l2_rows(yh.numpy(), oracle.fft(x, nthreads=NTHREADS)).max() <= TOL_FP32
    plan.close()
