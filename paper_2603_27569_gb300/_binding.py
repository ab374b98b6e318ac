"""ctypes binding of libfftgb.so: the C-ABI names, argument marshalling only.

Every transform runs in the library's CUDA kernels.  There is no fallback:
if ``_build/libfftgb.so`` is missing, the first call raises ``FFTError``
(run ``paper_2603_27569_gb300.build.build()`` or ``__graft_entry__.build()``).
PyTorch supplies device memory (``data_ptr``) and streams
(``torch.cuda.current_stream().cuda_stream``) only.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "FFTError", "FFT_FORWARD", "FFT_INVERSE", "FFT_PREC_FP32", "FFT_PREC_FP16X2",
    "FFT_PREC_BF16X2", "FFT_PREC_FP16_STORAGE", "FFT_PREC_BF16_STORAGE", "FFT_FLAG_UNNORMALIZED_INVERSE", "FFT_FLAG_FORCE_SINGLE_CTA",
    "FFT_FLAG_FORCE_FOURSTEP", "FFT_FLAG_NO_AUTOTUNE_CACHE", "FFT_FLAG_ADJOINT",
    "FFT_PATH_SINGLE_CTA", "FFT_PATH_FOURSTEP", "FFT_PATH_RAGGED", "FFT_PATH_TENSORCORE",
    "STATUS", "lib", "library_path", "fft_status_string", "fft_plan", "fft_plan_ex", "fft_exec",
    "fft_exec_host", "fft_destroy", "fft_plan_info", "fft_last_device_status",
    "fft_twiddle_table", "fft_twiddle_index", "fft_ragged_plan", "fft_autotune",
    "fft_autotune_load", "fft_autotune_clear", "fft_filter_apply",
    "fft_filter_grad_h_workspace", "fft_filter_grad_h", "fft_filter_plan",
    "fft_filter_forward", "fft_filter_backward", "fft_filter_step", "FFT_PATH_FILTER",
    "PlanInfo", "Config", "EXPORTED_SYMBOLS", "fft_list_configs", "fft_plan_config",
    "fft_fourstep_noalloc", "FFT_NOALLOC_MAX_POINTS", "fft_plan_columns", "FFT_PATH_COLUMNS",
    "FFT_PATH_TMEM_HALVES",
    "fft_ragged_class_config", "FFT_FLAG_RAGGED_AUTOTUNE", "fft_ragged_list_configs",
    "fft_ragged_choose", "fft_debug_fail_alloc", "fft_debug_bounded_wait",
    "fft_debug_bounds_status", "fft_debug_bounds_selftest",
]

FFT_FORWARD = -1
FFT_INVERSE = 1
FFT_PREC_FP32, FFT_PREC_FP16X2, FFT_PREC_BF16X2, FFT_PREC_FP16_STORAGE = 0, 1, 2, 3
FFT_PREC_BF16_STORAGE = 4
FFT_FLAG_UNNORMALIZED_INVERSE = 0x1
FFT_FLAG_FORCE_SINGLE_CTA = 0x2
FFT_FLAG_FORCE_FOURSTEP = 0x4
FFT_FLAG_NO_AUTOTUNE_CACHE = 0x8
FFT_FLAG_ADJOINT = 0x10
FFT_FLAG_RAGGED_AUTOTUNE = 0x20
FFT_PATH_SINGLE_CTA, FFT_PATH_FOURSTEP, FFT_PATH_RAGGED, FFT_PATH_TENSORCORE = 1, 2, 3, 4
FFT_PATH_FILTER = 5
FFT_PATH_COLUMNS = 6
FFT_PATH_TMEM_HALVES = 7
FFT_NOALLOC_MAX_POINTS = 2097152

STATUS = {
    0: "FFT_OK", 1: "FFT_ERR_INVALID_SIZE", 2: "FFT_ERR_INVALID_VALUE", 3: "FFT_ERR_MISALIGNED",
    4: "FFT_ERR_ALLOC", 5: "FFT_ERR_CUDA", 6: "FFT_ERR_TIMEOUT", 7: "FFT_ERR_NOT_SUPPORTED",
}

_HERE = os.path.dirname(os.path.abspath(__file__))
# The product library, or the bounds-checking debug build when FFTGB_LIBRARY
# names it (build.build(debug=True) returns its path).
_LIB_PATH = os.environ.get("FFTGB_LIBRARY") or os.path.join(_HERE, "_build", "libfftgb.so")
_lock = threading.Lock()
_lib = None


class FFTError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS.get(self.status, self.status)}")


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("batch", ctypes.c_int64), ("direction", ctypes.c_int),
        ("precision", ctypes.c_int), ("path", ctypes.c_int),
        ("points_per_thread", ctypes.c_int), ("transforms_per_cta", ctypes.c_int),
        ("threads_per_cta", ctypes.c_int), ("num_passes", ctypes.c_int),
        ("radix", ctypes.c_int * 8), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
        ("scratch_bytes", ctypes.c_int64), ("twiddle_mode", ctypes.c_int),
        ("grid_ctas", ctypes.c_int), ("tma_slabs", ctypes.c_int),
        ("cluster_split", ctypes.c_int), ("l2_chunk_rows", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "radix"}
        d["radix"] = [r for r in self.radix[: self.num_passes]]
        return d


class Config(ctypes.Structure):
    _fields_ = [
        ("path", ctypes.c_int), ("points_per_thread", ctypes.c_int),
        ("transforms_per_cta", ctypes.c_int), ("threads_per_cta", ctypes.c_int),
        ("num_passes", ctypes.c_int), ("radix", ctypes.c_int * 8), ("n1", ctypes.c_int),
        ("twiddle_mode", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
        ("tma_slabs", ctypes.c_int), ("cluster_split", ctypes.c_int),
        ("l2_chunk_rows", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "radix"}
        d["radix"] = [r for r in self.radix[: self.num_passes]]
        return d

    @classmethod
    def from_dict(cls, d: dict) -> "Config":
        c = cls()
        for f, _ in cls._fields_:
            if f == "radix":
                for i, r in enumerate(d["radix"]):
                    c.radix[i] = r
            elif f in d:
                setattr(c, f, d[f])
        c.num_passes = len(d["radix"])
        return c


_vp, _i32, _i64, _f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
_SIGS = {
    "fft_status_string": ([_i32], ctypes.c_char_p),
    "fft_plan": ([ctypes.POINTER(_vp), _i32, _i64, _i32], _i32),
    "fft_plan_ex": ([ctypes.POINTER(_vp), _i32, _i64, _i32, _i32, _i32], _i32),
    "fft_exec": ([_vp, _vp, _vp, _vp], _i32),
    "fft_exec_host": ([_vp, _vp, _vp, _vp], _i32),
    "fft_destroy": ([_vp], _i32),
    "fft_plan_info": ([_vp, ctypes.POINTER(PlanInfo)], _i32),
    "fft_last_device_status": ([_vp], _i32),
    "fft_twiddle_table": ([_vp, _vp, _i64, ctypes.POINTER(_i64)], _i32),
    "fft_twiddle_index": ([_vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _i32),
    "fft_ragged_plan": ([ctypes.POINTER(_vp), _i32, _vp, _vp, _vp, _vp, _i32], _i32),
    "fft_ragged_class_config": ([_vp, _i32, _i32, ctypes.POINTER(Config)], _i32),
    "fft_ragged_list_configs": ([_i32, _vp, _i32], _i32),
    "fft_ragged_choose": ([_i32, _i32, ctypes.POINTER(Config)], _i32),
    "fft_autotune": ([_i32, _i32, _i32, _i64, ctypes.c_char_p], _i32),
    "fft_autotune_load": ([ctypes.c_char_p], _i32),
    "fft_autotune_clear": ([], _i32),
    "fft_filter_apply": ([_vp, _vp, _vp, _i32, _i64, _i32, _f32, _vp], _i32),
    "fft_filter_grad_h_workspace": ([_i32, _i64], _i64),
    "fft_filter_grad_h": ([_vp, _vp, _vp, _i32, _i64, _vp, _vp], _i32),
    "fft_filter_plan": ([ctypes.POINTER(_vp), _i32, _i64], _i32),
    "fft_filter_forward": ([_vp, _vp, _vp, _vp, _vp, _i32, _vp], _i32),
    "fft_filter_backward": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "fft_filter_step": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "fft_list_configs": ([_i32, _vp, _i32], _i32),
    "fft_plan_config": ([ctypes.POINTER(_vp), _i32, _i64, _i32, _i32, ctypes.POINTER(Config)], _i32),
    "fft_fourstep_noalloc": ([_vp, _vp, _i32, _i64, _i32, _vp], _i32),
    "fft_plan_columns": ([ctypes.POINTER(_vp), _i32, _i64, _i64, _i64, _i64, _i32, _i32], _i32),
    "fft_debug_fail_alloc": ([_i32], None),
    "fft_debug_bounded_wait": ([_i32, _i32, _vp], _i32),
    "fft_debug_bounds_status": ([], _i32),
    "fft_debug_bounds_selftest": ([_vp], _i32),
}
EXPORTED_SYMBOLS = tuple(_SIGS)


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libfftgb.so (once).  Raises FFTError-free RuntimeError if absent."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(_LIB_PATH):
                    raise RuntimeError(
                        f"libfftgb.so is not built ({_LIB_PATH}); run "
                        "paper_2603_27569_gb300.build.build() first")
                L = ctypes.CDLL(_LIB_PATH)
                for name, (args, res) in _SIGS.items():
                    f = getattr(L, name)
                    f.argtypes = args
                    f.restype = res
                _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != 0:
        raise FFTError(status, where)


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def fft_status_string(status: int) -> str:
    return lib().fft_status_string(status).decode()


def fft_plan(N: int, batch: int, direction: int) -> int:
    h = _vp()
    _check(lib().fft_plan(ctypes.byref(h), N, batch, direction), "fft_plan")
    return h.value


def fft_plan_ex(N: int, batch: int, direction: int, precision: int = 0, flags: int = 0) -> int:
    h = _vp()
    _check(lib().fft_plan_ex(ctypes.byref(h), N, batch, direction, precision, flags),
           "fft_plan_ex")
    return h.value


def fft_exec(plan: int, inp, out, stream=None) -> None:
    _check(lib().fft_exec(plan, _ptr(inp), _ptr(out), _stream(stream)), "fft_exec")


def fft_exec_host(plan: int, host_in, host_out, stream=None) -> None:
    _check(lib().fft_exec_host(plan, _ptr(host_in), _ptr(host_out), _stream(stream)),
           "fft_exec_host")


def fft_destroy(plan: int) -> None:
    _check(lib().fft_destroy(plan), "fft_destroy")


def fft_plan_info(plan: int) -> dict:
    info = PlanInfo()
    _check(lib().fft_plan_info(plan, ctypes.byref(info)), "fft_plan_info")
    return info.as_dict()


def fft_last_device_status(plan: int) -> int:
    return int(lib().fft_last_device_status(plan))


def fft_twiddle_table(plan: int):
    """Return the plan's twiddle table as a complex64 NumPy array."""
    import numpy as np

    n = _i64()
    _check(lib().fft_twiddle_table(plan, None, 0, ctypes.byref(n)), "fft_twiddle_table")
    out = np.empty(n.value, dtype=np.complex64)
    if n.value:
        _check(lib().fft_twiddle_table(plan, out.ctypes.data, n.value, ctypes.byref(n)),
               "fft_twiddle_table")
    return out


def fft_twiddle_index(plan: int, pos: int):
    M, e = _i64(), _i64()
    _check(lib().fft_twiddle_index(plan, pos, ctypes.byref(M), ctypes.byref(e)),
           "fft_twiddle_index")
    return M.value, e.value


def fft_ragged_plan(N, direction, in_offset, out_offset, flags: int = 0) -> int:
    import numpy as np

    N = np.ascontiguousarray(N, dtype=np.int32)
    d = np.ascontiguousarray(direction, dtype=np.int32)
    oi = np.ascontiguousarray(in_offset, dtype=np.int64)
    oo = np.ascontiguousarray(out_offset, dtype=np.int64)
    h = _vp()
    _check(lib().fft_ragged_plan(ctypes.byref(h), len(N), N.ctypes.data, d.ctypes.data,
                                 oi.ctypes.data, oo.ctypes.data, flags), "fft_ragged_plan")
    return h.value


def fft_ragged_class_config(plan: int, N: int, direction: int) -> dict:
    """The routine a ragged plan runs for its class (N, direction)."""
    c = Config()
    _check(lib().fft_ragged_class_config(plan, N, direction, ctypes.byref(c)),
           "fft_ragged_class_config")
    return c.as_dict()


def fft_ragged_list_configs(N: int) -> list:
    n = lib().fft_ragged_list_configs(N, None, 0)
    arr = (Config * max(n, 1))()
    lib().fft_ragged_list_configs(N, ctypes.cast(arr, _vp), n)
    return [arr[i].as_dict() for i in range(n)]


def fft_ragged_choose(N: int, direction: int, config: dict) -> None:
    c = Config.from_dict(config)
    _check(lib().fft_ragged_choose(N, direction, ctypes.byref(c)), "fft_ragged_choose")


def fft_autotune(N: int, direction: int, precision: int = 0, batch: int = 0,
                 cache_path: str | None = None) -> None:
    _check(lib().fft_autotune(N, direction, precision, batch,
                              cache_path.encode() if cache_path else None), "fft_autotune")


def fft_autotune_load(cache_path: str) -> None:
    _check(lib().fft_autotune_load(cache_path.encode()), "fft_autotune_load")


def fft_autotune_clear() -> None:
    _check(lib().fft_autotune_clear(), "fft_autotune_clear")


def fft_filter_apply(X, H, Z, N: int, batch: int, conj_h: bool = False, scale: float = 1.0,
                     stream=None) -> None:
    _check(lib().fft_filter_apply(_ptr(X), _ptr(H), _ptr(Z), N, batch, int(bool(conj_h)),
                                  float(scale), _stream(stream)), "fft_filter_apply")


def fft_filter_grad_h_workspace(N: int, batch: int) -> int:
    return int(lib().fft_filter_grad_h_workspace(N, batch))


def fft_filter_grad_h(X, G, grad_H, N: int, batch: int, work, stream=None) -> None:
    _check(lib().fft_filter_grad_h(_ptr(X), _ptr(G), _ptr(grad_H), N, batch, _ptr(work),
                                   _stream(stream)), "fft_filter_grad_h")


def fft_filter_plan(N: int, batch: int) -> int:
    h = _vp()
    _check(lib().fft_filter_plan(ctypes.byref(h), N, batch), "fft_filter_plan")
    return h.value


def fft_filter_forward(plan: int, x, H, y, X_save=None, conj_h: bool = False,
                       stream=None) -> None:
    _check(lib().fft_filter_forward(plan, _ptr(x), _ptr(H), _ptr(y), _ptr(X_save),
                                    int(bool(conj_h)), _stream(stream)), "fft_filter_forward")


def fft_filter_backward(plan: int, g_y, H, X_saved, grad_x, grad_H, stream=None) -> None:
    _check(lib().fft_filter_backward(plan, _ptr(g_y), _ptr(H), _ptr(X_saved), _ptr(grad_x),
                                     _ptr(grad_H), _stream(stream)), "fft_filter_backward")


def fft_filter_step(plan: int, x, H, mask, y, grad_x, grad_H, loss, stream=None) -> None:
    """Fused forward + masked-energy loss + backward (y may be None)."""
    _check(lib().fft_filter_step(plan, _ptr(x), _ptr(H), _ptr(mask), _ptr(y), _ptr(grad_x),
                                 _ptr(grad_H), _ptr(loss), _stream(stream)), "fft_filter_step")


def fft_list_configs(N: int) -> list:
    n = lib().fft_list_configs(N, None, 0)
    arr = (Config * max(n, 1))()
    lib().fft_list_configs(N, ctypes.cast(arr, _vp), n)
    return [arr[i].as_dict() for i in range(n)]


def fft_plan_config(N: int, batch: int, direction: int, config: dict, flags: int = 0) -> int:
    c = Config.from_dict(config)
    h = _vp()
    _check(lib().fft_plan_config(ctypes.byref(h), N, batch, direction, flags, ctypes.byref(c)),
           "fft_plan_config")
    return h.value


def fft_plan_columns(L: int, ncols: int, nmat: int, row_stride: int, mat_stride: int,
                     direction: int, flags: int = 0) -> int:
    """Plan L-point transforms down the columns of nmat strided matrices."""
    h = _vp()
    _check(lib().fft_plan_columns(ctypes.byref(h), L, ncols, nmat, row_stride, mat_stride,
                                  direction, flags), "fft_plan_columns")
    return h.value


def fft_debug_fail_alloc(after: int) -> None:
    """Failure injection: the allocation after the next `after` fails (-1 disarms)."""
    lib().fft_debug_fail_alloc(int(after))


def fft_debug_bounded_wait(kind: int, limit_us: int, stream=None) -> int:
    """Runs a bounded device wait that nothing satisfies; returns the status code."""
    return int(lib().fft_debug_bounded_wait(int(kind), int(limit_us), _stream(stream)))


def fft_debug_bounds_status() -> int:
    """Debug build: first failed bounds-check site since the last call (0: none,
    cleared on read); -1 in the product build (no checks compiled)."""
    return int(lib().fft_debug_bounds_status())


def fft_debug_bounds_selftest(stream=None) -> int:
    """Debug build: fails one bounds check on purpose (nothing is accessed)."""
    return int(lib().fft_debug_bounds_selftest(_stream(stream)))


def fft_fourstep_noalloc(inp, out, N: int, batch: int, direction: int, stream=None) -> None:
    """Four-step transform that allocates nothing (fixed device scratch)."""
    _check(lib().fft_fourstep_noalloc(_ptr(inp), _ptr(out), N, batch, direction,
                                      _stream(stream)), "fft_fourstep_noalloc")
