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


# Element-wise bound beside every relative-L2 bound: for each compared array,
# max |gpu - ref| <= ELEMENTWISE_C * tol * max |ref|.  With C = 1 a single
# cell wrong by more than tol (relative to the field's scale) fails even
# where the pooled relative L2 would absorb it.
ELEMENTWISE_C = 1.0


def assert_parity(got, ref, tol, what=""):
    """Relative L2 over all components < tol, and the element-wise bound on
    every component.  got, ref: arrays or equal-length sequences of arrays."""
    if not isinstance(got, (list, tuple)):
        got, ref = [got], [ref]
    assert len(got) == len(ref)
    num = den = 0.0
    for k, (a, b) in enumerate(zip(got, ref)):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        assert a.shape == b.shape, (what, k, a.shape, b.shape)
        d = np.abs(a - b)
        num += float(np.sum(d * d))
        den += float(np.sum(b * b))
        scale = float(np.max(np.abs(b))) if b.size else 0.0
        worst = float(np.max(d)) if d.size else 0.0
        assert worst <= ELEMENTWISE_C * tol * scale, (
            f"{what} component {k}: max |diff| {worst:.3e} at {np.unravel_index(int(np.argmax(d)), d.shape)} "
            f"> {ELEMENTWISE_C} * {tol:g} * {scale:.3e}")
    rel = float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))
    assert rel < tol, f"{what} relative L2 {rel:.3e} >= {tol:g}"
    return rel
