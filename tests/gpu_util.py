"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev())


def zeros(n):
    return torch.zeros(int(n), dtype=torch.float64, device=dev())


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_max(a, b):
    """max |a - b| / max |b| (element-wise comparison scaled by the reference's size)."""
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d
