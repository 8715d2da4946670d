"""Shared helpers of the GPU parity tests (seeded inputs to device tensors, error metrics)."""
import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def to_dev_points(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev())


def to_dev_mu(m):
    import torch
    return torch.from_numpy(np.ascontiguousarray(m, dtype=np.float64)).to(dev())


def inf_rel_err(approx, ref):
    """max_i |approx_i - ref_i| / max_i |ref_i| (the matvec error measure, infinity norm)."""
    approx = np.asarray(approx, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(approx - ref)) / np.max(np.abs(ref)))


def problem_tensors(prob):
    return [to_dev_points(a) for a in prob.x], [to_dev_mu(m) for m in prob.mu]
