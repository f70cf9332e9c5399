"""Shared helpers of the GPU tests (device copies of seeded inputs)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev():
    return torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev())


def device_problem(P):
    import paper_1810_12437_gb300 as pb
    X = pb.DeviceDesign.from_host(P.X, dev())
    args = dict(omega=T(P.omega), z=T(P.z), lam=T(P.lam), eta=T(P.eta), delta=T(P.delta))
    return X, args


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
