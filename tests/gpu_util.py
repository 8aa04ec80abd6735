"""Shared fixtures/helpers for the GPU parity tests."""
import numpy as np


def rel_l2(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
