"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np


def rel_max(a, b):
    """max |a - b| / max |b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def f32(a):
    """Round to FP32 and return (fp32 array for the GPU, the same values in FP64 for the oracle)."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return x, x.astype(np.float64)
