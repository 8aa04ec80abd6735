"""Shared fixtures/helpers for the GPU parity tests."""
import numpy as np


def rel_l2(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def elementwise_ratio(x, ref, abs_rel, rel):
    """max over elements of |x - ref| / (abs_rel max|ref| + rel |ref|): the
    per-element error against a bound of that form (<= 1 passes)."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = abs_rel * np.abs(ref).max() + rel * np.abs(ref)
    return float(np.max(np.abs(x - ref) / tol))
