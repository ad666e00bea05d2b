"""Helpers for the GPU parity tests: device selection and the error metrics."""
import numpy as np


def cuda_device():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is visible")
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(cuda_device()).contiguous()


def rel_max_force(F, F0):
    """max_i |F_i - F0_i| / RMS(F0) (FP64 path metric)."""
    rms = np.sqrt(np.mean(np.sum(F0 * F0, axis=1)))
    return np.max(np.linalg.norm(F - F0, axis=1)) / rms


def rel_rms_force(F, F0):
    """RMS(F - F0) / RMS(F0) (FP32-phase path metric)."""
    return np.sqrt(np.mean(np.sum((F - F0) ** 2, axis=1)) / np.mean(np.sum(F0 * F0, axis=1)))


def rel_frob(W, W0):
    return np.linalg.norm(W - W0) / np.linalg.norm(W0)
