"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import pytest


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_np(t):
    return t.detach().double().cpu().numpy()


def periodic_box(a, center, radius):
    """Box of edge 2*radius+1 around center (z, y, x) of a periodic array."""
    idx = [np.arange(c - radius, c + radius + 1) % n for c, n in zip(center, a.shape)]
    return a[np.ix_(*idx)]
