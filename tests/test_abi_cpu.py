"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/fftgb.h declares, and rejects bad arguments on the host
before any CUDA call is made."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2603_27569_gb300 as fg
from paper_2603_27569_gb300 import build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fftgb.h")

OK, INVALID_SIZE, INVALID_VALUE, MISALIGNED = 0, 1, 2, 3
NOT_SUPPORTED = 7


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fft_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    fbuild.build()
    return fg.lib()


def test_header_declares_the_plan_exec_interface():
    names = declared_functions()
    for required in ("fft_plan", "fft_exec", "fft_destroy", "fft_plan_ex", "fft_ragged_plan",
                     "fft_autotune", "fft_status_string", "fft_last_device_status"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", fg.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fft_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        assert hasattr(L, n)


def test_binding_covers_the_header_exactly():
    assert sorted(fg.EXPORTED_SYMBOLS) == declared_functions()


def test_library_has_no_torch_dependency():
    out = subprocess.run(["ldd", fg.library_path()], capture_output=True, text=True).stdout
    assert "torch" not in out and "c10" not in out


def test_status_strings(L):
    for code, name in fg.STATUS.items():
        assert fg.fft_status_string(code) == name
    assert fg.fft_status_string(99) == "FFT_ERR_UNKNOWN"


def _plan_ex(L, N, batch, direction, prec=0, flags=0):
    h = ctypes.c_void_p(1234)
    rc = L.fft_plan_ex(ctypes.byref(h), N, batch, direction, prec, flags)
    return rc, h.value


@pytest.mark.parametrize("N", [0, 1, 3, 12, 100, 3 << 16, 1 << 21, 1 << 24])
def test_plan_rejects_bad_sizes(L, N):
    rc, h = _plan_ex(L, N, 4, -1)
    assert rc == INVALID_SIZE and h is None


def test_plan_rejects_bad_arguments(L):
    assert _plan_ex(L, 256, -1, -1)[0] == INVALID_SIZE
    assert _plan_ex(L, 256, 4, 0)[0] == INVALID_VALUE
    assert _plan_ex(L, 256, 4, 2)[0] == INVALID_VALUE
    assert _plan_ex(L, 256, 4, -1, prec=7)[0] == INVALID_VALUE
    assert _plan_ex(L, 256, 4, -1, flags=0x100)[0] == INVALID_VALUE
    assert _plan_ex(L, 256, 4, -1, flags=fg.FFT_FLAG_FORCE_FOURSTEP | fg.FFT_FLAG_FORCE_SINGLE_CTA)[0] \
        == INVALID_VALUE
    assert _plan_ex(L, 32768, 4, -1, flags=fg.FFT_FLAG_FORCE_SINGLE_CTA)[0] == 7
    assert _plan_ex(L, 32768, 4, -1, prec=fg.FFT_PREC_FP16X2)[0] == 7
    assert L.fft_plan_ex(None, 256, 4, -1, 0, 0) == INVALID_VALUE


def test_null_handles(L):
    assert L.fft_exec(None, None, None, None) == INVALID_VALUE
    assert L.fft_exec_host(None, None, None, None) == INVALID_VALUE
    assert L.fft_destroy(None) == OK
    assert L.fft_plan_info(None, None) == INVALID_VALUE
    assert L.fft_last_device_status(None) == INVALID_VALUE
    assert L.fft_plan_config(None, 256, 1, -1, 0, None) == INVALID_VALUE


def test_configs_listed_for_every_supported_size(L):
    for e in range(1, 15):
        N = 1 << e
        cfgs = fg.fft_list_configs(N)
        assert any(c["path"] == fg.FFT_PATH_SINGLE_CTA for c in cfgs), N
        for c in cfgs:
            prod = 1
            for r in c["radix"]:
                prod *= r
            if c["path"] == fg.FFT_PATH_SINGLE_CTA and c["cluster_split"]:
                # each CTA of the cluster transforms N/K points
                K = c["cluster_split"]
                assert K in (2, 4, 8) and prod == N // K
                assert c["threads_per_cta"] == (N // K) // c["points_per_thread"]
            elif c["path"] == fg.FFT_PATH_SINGLE_CTA:
                assert prod == N
                assert all(c["points_per_thread"] % r == 0 for r in c["radix"])
                assert c["threads_per_cta"] == c["transforms_per_cta"] * N // c["points_per_thread"]
                assert c["threads_per_cta"] <= 1024
            else:
                assert prod == N // c["n1"] and N % c["n1"] == 0
    assert fg.fft_list_configs(12) == []
    assert fg.fft_list_configs(1 << 21) == []
    for e in range(15, 21):   # beyond one CTA: four-step, clusters up to 2^16, halves at 2^15
        N = 1 << e
        cfgs = fg.fft_list_configs(N)
        four = [c for c in cfgs if c["path"] == fg.FFT_PATH_FOURSTEP]
        split = [c for c in cfgs if c["path"] == fg.FFT_PATH_SINGLE_CTA]
        halves = [c for c in cfgs if c["path"] == fg.FFT_PATH_TMEM_HALVES]
        assert four and len(four) + len(split) + len(halves) == len(cfgs)
        # one SM per row, half of it in tensor memory: each half is one
        # 16384-point Stockham schedule of 512 threads x 32 points
        assert bool(halves) == (N == 1 << 15)
        for c in halves:
            assert int(np.prod(c["radix"][:c["num_passes"]])) * 2 == N
            assert c["threads_per_cta"] * c["points_per_thread"] * 2 == N
            assert c["points_per_thread"] == 32 and not c["cluster_split"]
        assert all(c["cluster_split"] in (2, 4, 8) for c in split)
        assert bool(split) == (N <= 1 << 16)
        for c in split:
            prod = 1
            for r in c["radix"]:
                prod *= r
            assert prod * c["cluster_split"] == N and prod <= 16384
        for c in four:
            n2 = N // c["n1"]
            assert c["n1"] * n2 == N and 16 <= n2 <= 512 and c["n1"] <= 4096
    for N in (8192, 16384):
        assert any(c["path"] == fg.FFT_PATH_FOURSTEP for c in fg.fft_list_configs(N))


def test_filter_entry_points_validate_on_host(L):
    assert L.fft_filter_apply(16, 16, 16, 12, 1, 0, ctypes.c_float(1.0), None) == INVALID_SIZE
    assert L.fft_filter_apply(None, 16, 16, 256, 1, 0, ctypes.c_float(1.0), None) == INVALID_VALUE
    assert L.fft_filter_apply(24, 16, 16, 256, 1, 0, ctypes.c_float(1.0), None) == MISALIGNED
    assert L.fft_filter_apply(16, 16, 16, 256, 0, 0, ctypes.c_float(1.0), None) == OK
    assert L.fft_filter_grad_h_workspace(8192, 4096) == (4096 // 32) * 8192 * 8
    assert L.fft_filter_grad_h_workspace(8192, 33) == 2 * 8192 * 8
    assert L.fft_filter_grad_h(16, 16, 16, 12, 1, 16, None) == INVALID_SIZE
    assert L.fft_filter_grad_h(16, 16, 16, 256, 1, None, None) == INVALID_VALUE


def test_column_plan_validates_on_host(L):
    h = ctypes.c_void_p(1234)
    assert L.fft_plan_columns(None, 256, 16, 1, 16, 4096, -1, 0) == INVALID_VALUE
    assert L.fft_plan_columns(ctypes.byref(h), 8, 16, 1, 16, 128, -1, 0) == INVALID_SIZE
    assert h.value is None
    assert L.fft_plan_columns(ctypes.byref(h), 1 << 22, 16, 1, 16, 1 << 26, -1, 0) == INVALID_SIZE
    assert L.fft_plan_columns(ctypes.byref(h), 3 << 12, 16, 1, 16, 3 << 16, -1, 0) == INVALID_SIZE
    # L > 4096: 16-column tile, and n1 * row_stride (n1 = 64 at L = 8192) below 2^31
    assert L.fft_plan_columns(ctypes.byref(h), 8192, 8, 1, 8, 8192 * 8, -1, 0) == INVALID_SIZE
    assert L.fft_plan_columns(ctypes.byref(h), 8192, 16, 1, 1 << 25, 1 << 38, -1, 0) == INVALID_SIZE
    assert L.fft_plan_columns(ctypes.byref(h), 256, 17, 1, 17, 256 * 17, -1, 0) == INVALID_SIZE
    assert L.fft_plan_columns(ctypes.byref(h), 4096, 6, 1, 6, 4096 * 6, -1, 0) == INVALID_SIZE
    assert L.fft_plan_columns(ctypes.byref(h), 256, 16, 1, 8, 4096, -1, 0) == INVALID_VALUE
    assert L.fft_plan_columns(ctypes.byref(h), 256, 16, 2, 16, 1000, -1, 0) == INVALID_VALUE
    assert L.fft_plan_columns(ctypes.byref(h), 256, 16, 1, 16, 4096, 0, 0) == INVALID_VALUE
    assert L.fft_plan_columns(ctypes.byref(h), 256, 16, 1, 16, 4096, -1, 0x8) == INVALID_VALUE
    assert L.fft_plan_columns(ctypes.byref(h), 2048, 16, 1, 16, 2048 * 16, -1, 0x6) == INVALID_VALUE
    assert L.fft_plan_columns(ctypes.byref(h), 1024, 16, 1, 16, 1024 * 16, -1, 0x4) == NOT_SUPPORTED
    assert L.fft_plan_columns(ctypes.byref(h), 8192, 16, 1, 16, 8192 * 16, -1, 0x2) == NOT_SUPPORTED


def test_every_declaration_cites_its_passage():
    """Each exported function's comment (the nearest comment block before its
    declaration) names the paper passage it implements, or says the paper has
    no counterpart."""
    text = open(HEADER).read()
    body = text[text.index("#ifdef __cplusplus"):]
    missing = []
    for m in re.finditer(r"\b(fft_[a-z0-9_]+)\s*\(", body):
        before = body[:m.start()]
        if before.rstrip().endswith("*/") is False and "/*" not in before:
            missing.append(m.group(1))
            continue
        comment = before[before.rindex("/*"):]
        if "*/" not in comment:        # the name appears inside a comment
            continue
        comment = comment[:comment.index("*/")]
        if not re.search(r"Paper: (Sec\.|Eq\.|Table)", comment) and \
                "paper has no counterpart" not in comment.lower():
            missing.append(m.group(1))
    assert not missing, f"declarations without a cited passage: {sorted(set(missing))}"
