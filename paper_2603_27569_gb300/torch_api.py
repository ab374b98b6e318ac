"""PyTorch-facing wrappers over the C ABI: plans, ``fft``/``ifft`` and autograd.

PyTorch provides device memory and the current stream; every transform,
pointwise multiply and reduction runs in libfftgb's kernels.

Differentiation (the adjoint of a linear map is its conjugate transpose):
  y = F x     (unnormalised forward)   ->  grad_x = F^H grad_y
  y = G x     (inverse, G = F^H / N)   ->  grad_x = G^H grad_y = (1/N) F grad_y
Both adjoints are library plans built with FFT_FLAG_ADJOINT.  Complex
gradients follow PyTorch's convention grad = dL/dRe + i dL/dIm.

SpectralFilter implements SAR range compression (paper Sec. II-D):
  y = IFFT(FFT(x) * H), with H learnable.
  backward: g_z = G^H g_y;  grad_H = sum_rows conj(FFT(x)) * g_z;
            grad_x = F^H (conj(H) * g_z).
"""
from __future__ import annotations

import collections
import threading

import torch

from . import _binding as B

__all__ = ["Plan", "get_plan", "fft", "ifft", "fft_host", "SpectralFilter",
           "spectral_filter", "clear_plan_cache", "ColumnPlan", "fft_columns"]

_PREC = {"fp32": B.FFT_PREC_FP32, "fp16x2": B.FFT_PREC_FP16X2, "bf16x2": B.FFT_PREC_BF16X2,
         "fp16_storage": B.FFT_PREC_FP16_STORAGE, "bf16_storage": B.FFT_PREC_BF16_STORAGE}


def _check_tensor(x: torch.Tensor, N: int, batch: int, what: str,
                  dtype=torch.complex64) -> None:
    """Complex dtypes hold one point per element; torch.bfloat16 (BF16 pairs,
    torch has no complex BF16 type) holds interleaved (re, im), two per point."""
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{what} must be a torch.Tensor")
    if x.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    per_point = 2 if dtype == torch.bfloat16 else 1
    if x.numel() != per_point * N * batch:
        raise ValueError(f"{what} has {x.numel()} elements, plan needs {per_point * N * batch}")


class Plan:
    """Owns one fft_plan_t on one CUDA device."""

    def __init__(self, N: int, batch: int, direction: int = B.FFT_FORWARD, precision: int = 0,
                 flags: int = 0, config: dict | None = None, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        with torch.cuda.device(self.device):
            if config is not None:
                self.handle = B.fft_plan_config(N, batch, direction, config, flags)
            else:
                self.handle = B.fft_plan_ex(N, batch, direction, precision, flags)
        self.N, self.batch, self.direction = N, batch, direction
        self.precision, self.flags = precision, flags

    def __call__(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        return self.exec(x, out, stream)

    @property
    def dtype(self):
        """complex64; torch.complex32 (FP16 pairs) for FP16 storage; torch.bfloat16
        with interleaved (re, im), 2 elements per point, for BF16 storage."""
        if self.precision == B.FFT_PREC_FP16_STORAGE:
            return torch.complex32
        if self.precision == B.FFT_PREC_BF16_STORAGE:
            return torch.bfloat16
        return torch.complex64

    def exec(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        if not x.is_cuda or x.device != self.device:
            raise ValueError(f"input must live on {self.device}")
        _check_tensor(x, self.N, self.batch, "input", self.dtype)
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_tensor(out, self.N, self.batch, "output", self.dtype)
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        B.fft_exec(self.handle, x, out, st)
        return out

    def exec_host(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """Transform a host (ideally pinned) complex64 tensor; returns a host tensor."""
        if x.is_cuda:
            raise ValueError("exec_host takes a host tensor")
        _check_tensor(x, self.N, self.batch, "input", self.dtype)
        if out is None:
            out = torch.empty_like(x, pin_memory=x.is_pinned())
        else:
            _check_tensor(out, self.N, self.batch, "output", self.dtype)
        with torch.cuda.device(self.device):
            st = torch.cuda.current_stream(self.device) if stream is None else stream
            B.fft_exec_host(self.handle, x, out, st)
        return out

    def info(self) -> dict:
        return B.fft_plan_info(self.handle)

    def device_status(self) -> int:
        return B.fft_last_device_status(self.handle)

    def close(self) -> None:
        h, self.handle = getattr(self, "handle", None), None
        if h:
            try:
                with torch.cuda.device(self.device):
                    B.fft_destroy(h)
            except Exception:
                pass

    def __del__(self):
        self.close()


_cache: "collections.OrderedDict[tuple, Plan]" = collections.OrderedDict()
_cache_lock = threading.Lock()
_CACHE_MAX = 64


def get_plan(N: int, batch: int, direction: int, precision: int = 0, flags: int = 0,
             device=None) -> Plan:
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    key = (dev.index, N, batch, direction, precision, flags)
    with _cache_lock:
        p = _cache.get(key)
        if p is not None:
            _cache.move_to_end(key)
            return p
    p = Plan(N, batch, direction, precision, flags, device=dev)
    with _cache_lock:
        _cache[key] = p
        while len(_cache) > _CACHE_MAX:
            _cache.popitem(last=False)
    return p


def clear_plan_cache() -> None:
    with _cache_lock:
        _cache.clear()
        _col_cache.clear()


def _raw(x: torch.Tensor, direction: int, precision: int, flags: int, out=None) -> torch.Tensor:
    N = x.shape[-1]
    batch = x.numel() // N if N else 0
    plan = get_plan(N, batch, direction, precision, flags, x.device)
    return plan.exec(x.contiguous(), out).view(x.shape)


class _FFTFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, direction, precision, flags):
        ctx.direction, ctx.precision, ctx.flags = direction, precision, flags
        return _raw(x, direction, precision, flags)

    @staticmethod
    def backward(ctx, g):
        gx = _raw(g.contiguous(), ctx.direction, ctx.precision, ctx.flags | B.FFT_FLAG_ADJOINT)
        return gx, None, None, None


def fft(x: torch.Tensor, inverse: bool = False, precision: str = "fp32",
        unnormalized_inverse: bool = False) -> torch.Tensor:
    """Batched C2C FFT along the last dimension of a CUDA complex64 tensor.

    forward: unnormalised, W_N = exp(-2 pi i / N); inverse: scaled by 1/N
    unless ``unnormalized_inverse``.  Differentiable (adjoint plans).
    """
    direction = B.FFT_INVERSE if inverse else B.FFT_FORWARD
    flags = B.FFT_FLAG_UNNORMALIZED_INVERSE if unnormalized_inverse else 0
    prec = _PREC[precision]
    if torch.is_grad_enabled() and x.requires_grad:
        return _FFTFn.apply(x, direction, prec, flags)
    return _raw(x, direction, prec, flags)


def ifft(x: torch.Tensor, precision: str = "fp32") -> torch.Tensor:
    return fft(x, inverse=True, precision=precision)


def fft_host(x: torch.Tensor, inverse: bool = False, device=None) -> torch.Tensor:
    """Host tensor in, host tensor out; copies pipelined with the transforms."""
    N = x.shape[-1]
    batch = x.numel() // N
    plan = get_plan(N, batch, B.FFT_INVERSE if inverse else B.FFT_FORWARD, 0, 0, device)
    return plan.exec_host(x.contiguous()).view(x.shape)


class ColumnPlan:
    """L-point transforms down the columns of [nmat, L, ncols] complex64 views
    (row and matrix strides in elements): the azimuth pass of SAR processing
    without a transpose (C ABI: fft_plan_columns)."""

    def __init__(self, L: int, ncols: int, nmat: int = 1, row_stride: int | None = None,
                 mat_stride: int | None = None, direction: int = B.FFT_FORWARD, flags: int = 0,
                 device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.L, self.ncols, self.nmat = L, ncols, nmat
        self.row_stride = ncols if row_stride is None else row_stride
        self.mat_stride = L * self.row_stride if mat_stride is None else mat_stride
        with torch.cuda.device(self.device):
            self.handle = B.fft_plan_columns(L, ncols, nmat, self.row_stride, self.mat_stride,
                                             direction, flags)

    def _check(self, x: torch.Tensor, what: str) -> None:
        if not isinstance(x, torch.Tensor) or x.dtype != torch.complex64:
            raise TypeError(f"{what} must be a complex64 torch.Tensor")
        if not x.is_cuda or x.device != self.device:
            raise ValueError(f"{what} must live on {self.device}")
        need = (self.nmat - 1) * self.mat_stride + (self.L - 1) * self.row_stride + self.ncols
        if self.nmat and x.storage_offset() + need > x.untyped_storage().nbytes() // 8:
            raise ValueError(f"{what} does not hold the planned strided extent")

    def __call__(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """x (and out): tensors whose data pointer is the first matrix's (0, 0)."""
        self._check(x, "input")
        if out is None:
            out = torch.empty_like(x)
        self._check(out, "output")
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        B.fft_exec(self.handle, x, out, st)
        return out

    def info(self) -> dict:
        return B.fft_plan_info(self.handle)

    def close(self) -> None:
        h, self.handle = getattr(self, "handle", None), None
        if h:
            try:
                with torch.cuda.device(self.device):
                    B.fft_destroy(h)
            except Exception:
                pass

    def __del__(self):
        self.close()


def fft_columns(x: torch.Tensor, inverse: bool = False) -> torch.Tensor:
    """Transform along dim -2 of a complex64 CUDA tensor [..., L, ncols] whose
    last dim is contiguous (other strides are passed to the kernel as they
    are); returns a tensor of the same shape and strides."""
    if x.dim() < 2 or x.stride(-1) != 1:
        raise ValueError("need [..., L, ncols] with a contiguous last dimension")
    lead = x.shape[:-2]
    if len(lead) > 1:
        x = x.reshape((-1,) + tuple(x.shape[-2:]))
    L, ncols = x.shape[-2], x.shape[-1]
    nmat = x.shape[0] if x.dim() == 3 else 1
    mat_stride = x.stride(0) if x.dim() == 3 else L * x.stride(-2)
    key = (L, ncols, nmat, x.stride(-2), mat_stride, bool(inverse), x.device)
    with _cache_lock:
        plan = _col_cache.get(key)
        if plan is None:
            plan = ColumnPlan(L, ncols, nmat, x.stride(-2), mat_stride,
                              B.FFT_INVERSE if inverse else B.FFT_FORWARD, device=x.device)
            _col_cache[key] = plan
            while len(_col_cache) > _CACHE_MAX:
                _col_cache.popitem(last=False)[1].close()
        else:
            _col_cache.move_to_end(key)
    out = torch.empty_strided(x.shape, x.stride(), dtype=x.dtype, device=x.device)
    plan(x, out)
    return out.reshape(lead + (L, ncols)) if len(lead) > 1 else out


_col_cache: "collections.OrderedDict[tuple, ColumnPlan]" = collections.OrderedDict()


class _SpectralFilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, H):
        N = x.shape[-1]
        batch = x.numel() // N
        xc = x.contiguous()
        Hc = H.contiguous()
        X = _raw(xc, B.FFT_FORWARD, 0, 0)                       # F x
        Z = torch.empty_like(X)
        st = torch.cuda.current_stream(x.device)
        B.fft_filter_apply(X, Hc, Z, N, batch, False, 1.0, st)   # F x * H
        y = _raw(Z, B.FFT_INVERSE, 0, 0, out=Z)                   # G (F x * H), in place
        ctx.save_for_backward(X, Hc)
        ctx.shape = x.shape
        return y.view(x.shape)

    @staticmethod
    def backward(ctx, gy):
        X, H = ctx.saved_tensors
        N = X.shape[-1]
        batch = X.numel() // N
        st = torch.cuda.current_stream(X.device)
        gz = _raw(gy.contiguous(), B.FFT_INVERSE, 0, B.FFT_FLAG_ADJOINT)  # G^H g_y = F g_y / N
        grad_x = grad_H = None
        if ctx.needs_input_grad[1]:
            grad_H = torch.empty(N, dtype=torch.complex64, device=X.device)
            ws = B.fft_filter_grad_h_workspace(N, batch)
            work = torch.empty(max(ws, 8), dtype=torch.uint8, device=X.device)
            B.fft_filter_grad_h(X, gz, grad_H, N, batch, work, st)
        if ctx.needs_input_grad[0]:
            B.fft_filter_apply(gz, H, gz, N, batch, True, 1.0, st)           # conj(H) g_z
            grad_x = _raw(gz, B.FFT_FORWARD, 0, B.FFT_FLAG_ADJOINT, out=gz)  # F^H (.)
            grad_x = grad_x.view(ctx.shape)
        return grad_x, grad_H


class _FilterPlan:
    """Owns one fused spectral-filter plan (fft_filter_plan)."""

    def __init__(self, N: int, batch: int, device):
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.handle = B.fft_filter_plan(N, batch)

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            try:
                with torch.cuda.device(self.device):
                    B.fft_destroy(h)
            except Exception:
                pass

    def __del__(self):
        self.close()


_fcache: "collections.OrderedDict[tuple, _FilterPlan]" = collections.OrderedDict()


def _filter_plan(N: int, batch: int, device) -> _FilterPlan:
    key = (torch.device(device).index, N, batch)
    with _cache_lock:
        p = _fcache.get(key)
        if p is not None:
            _fcache.move_to_end(key)
            return p
    p = _FilterPlan(N, batch, device)
    with _cache_lock:
        _fcache[key] = p
        while len(_fcache) > _CACHE_MAX:
            _fcache.popitem(last=False)
    return p


class _FusedSpectralFilterFn(torch.autograd.Function):
    """Forward FFT, * H and inverse FFT in one kernel per row (and the backward
    likewise): each row crosses HBM once each way."""

    @staticmethod
    def forward(ctx, x, H):
        N = x.shape[-1]
        batch = x.numel() // N
        xc = x.contiguous()
        Hc = H.contiguous()
        plan = _filter_plan(N, batch, x.device)
        y = torch.empty_like(xc)
        need_grad = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        X = torch.empty_like(xc) if need_grad else None
        B.fft_filter_forward(plan.handle, xc, Hc, y, X, False,
                             torch.cuda.current_stream(x.device))
        ctx.save_for_backward(X if X is not None else xc, Hc)
        ctx.shape = x.shape
        return y.view(x.shape)

    @staticmethod
    def backward(ctx, gy):
        X, H = ctx.saved_tensors
        N = X.shape[-1]
        batch = X.numel() // N
        plan = _filter_plan(N, batch, X.device)
        gx = torch.empty_like(X)
        gH = torch.empty(N, dtype=torch.complex64, device=X.device)
        B.fft_filter_backward(plan.handle, gy.contiguous(), H, X, gx, gH,
                              torch.cuda.current_stream(X.device))
        return (gx.view(ctx.shape) if ctx.needs_input_grad[0] else None,
                gH if ctx.needs_input_grad[1] else None)


# Largest N at which the filter plan's kernels measured faster than separate
# transforms and multiplies on GB300 (forward with the saved spectrum plus
# backward): every supported N.
FUSED_MAX_N = 16384


def spectral_filter(x: torch.Tensor, H: torch.Tensor, fused: bool | None = None) -> torch.Tensor:
    """y = IFFT(FFT(x) * H) along the last dimension; differentiable in x and H.

    fused=True runs forward FFT, multiply and inverse FFT in one kernel per row
    (N = 256..16384); fused=False runs them as separate library kernels;
    None picks the faster for N (fused up to FUSED_MAX_N)."""
    N = x.shape[-1]
    if fused is None:
        fused = N <= FUSED_MAX_N
    if fused and 256 <= N <= 16384:
        return _FusedSpectralFilterFn.apply(x, H)
    return _SpectralFilterFn.apply(x, H)


def spectral_filter_step(x: torch.Tensor, H: torch.Tensor, mask: torch.Tensor,
                         keep_y: bool = True):
    """One fused training step of the filter under L = sum(mask * |y|^2):
    returns (y or None, L, grad_x, grad_H) from one persistent kernel per call
    (C ABI: fft_filter_step; N = 8192 or 16384, x [..., N] complex64, mask the
    same shape as float32)."""
    N = x.shape[-1]
    batch = x.numel() // N
    xc = x.contiguous()
    Hc = H.detach().contiguous()
    m = mask.to(torch.float32).contiguous()
    if m.shape != x.shape:
        raise ValueError("mask must have x's shape")
    plan = _filter_plan(N, batch, x.device)
    y = torch.empty_like(xc) if keep_y else None
    gx = torch.empty_like(xc)
    gH = torch.empty(N, dtype=torch.complex64, device=x.device)
    loss = torch.empty((), dtype=torch.float32, device=x.device)
    B.fft_filter_step(plan.handle, xc, Hc, m, y, gx, gH, loss,
                      torch.cuda.current_stream(x.device))
    return (y.view(x.shape) if keep_y else None), loss, gx.view(x.shape), gH


class SpectralFilter(torch.nn.Module):
    """Learnable matched filter H (complex64 [N]) applied in the frequency domain."""

    def __init__(self, H: torch.Tensor, fused: bool | None = None):
        super().__init__()
        self.H = torch.nn.Parameter(H.detach().clone().to(torch.complex64))
        self.fused = fused

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return spectral_filter(x, self.H, self.fused)
