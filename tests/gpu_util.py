"""Shared helpers for the GPU tests (CUDA path vs the FP64 oracle)."""
import os

import numpy as np

TOL_FP32 = 5e-6      # max per-transform relative L2 error, FP32 path
TOL_SPLIT = 1e-5     # tensor-core split-precision path
TOL_GRAD = 1e-5      # gradients vs the oracle's analytic gradient

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def rel_l2_rows(got, want) -> np.ndarray:
    """Relative L2 error of each transform (row); absolute if the row is zero."""
    got = np.asarray(got, np.complex128).reshape(-1, np.shape(want)[-1])
    want = np.asarray(want, np.complex128).reshape(got.shape)
    num = np.linalg.norm(got - want, axis=1)
    den = np.linalg.norm(want, axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1), num)


def to_dev(x: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t) -> np.ndarray:
    return t.detach().cpu().numpy()
