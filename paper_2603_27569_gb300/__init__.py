"""GB300-native batched complex-to-complex FFT (Stockham, radix-8/16 with
radix-4/2 tails, four-step), after arxiv 2603.27569.

The compute path is the C-ABI library ``libfftgb.so`` built from ``csrc/``;
``_binding`` is its ctypes binding with the C names, ``torch_api`` the
PyTorch-facing wrappers (plans, fft/ifft, autograd, spectral filter).
Importing the package does not load the library; the first call that needs
it does, and raises if it is missing.
"""
import importlib as _importlib

from ._binding import *  # noqa: F401,F403

_TORCH_NAMES = ("Plan", "get_plan", "fft", "ifft", "fft_host", "SpectralFilter",
                "spectral_filter", "spectral_filter_step", "clear_plan_cache", "ColumnPlan",
                "fft_columns")


def __getattr__(name):
    # torch-level API, imported on first use so that ``synth`` and the
    # C-ABI names stay importable without paying for ``import torch``.
    if name in _TORCH_NAMES:
        return getattr(_importlib.import_module(__name__ + ".torch_api"), name)
    raise AttributeError(name)
