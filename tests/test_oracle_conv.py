"""Pins for the oracle's 3D periodic convolution (learned surrogate).

* A kernel with only the centre tap is a per-cell matrix product x @ W + b
  (numpy matmul).
* A kernel with a single off-centre tap (dz,dy,dx) is the input rolled so that
  cell p reads p + offset (numpy roll), then x @ W.
* dgrad and wgrad are the exact gradients of the scalar loss
  L = sum(y * g): checked by FP64 central differences.
"""
import numpy as np
import pytest

import oracle


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_centre_tap_is_matmul():
    x = _rand((3, 4, 5, 2), 0)
    w = np.zeros((27, 2, 3))
    w[13] = _rand((2, 3), 1)
    b = _rand(3, 2)
    y = oracle.conv3d_fwd(x, w, b)
    assert np.allclose(y, x @ w[13] + b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("off", [(1, 0, 0), (0, -1, 0), (0, 0, 1), (-1, 1, -1)])
def test_single_tap_is_rolled_matmul(off):
    dz, dy, dx = off
    x = _rand((4, 3, 5, 2), 3)
    w = np.zeros((27, 2, 4))
    tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
    w[tap] = _rand((2, 4), 4)
    y = oracle.conv3d_fwd(x, w)
    shifted = np.roll(x, shift=(-dz, -dy, -dx), axis=(0, 1, 2))  # shifted[p] = x[p + off]
    assert np.allclose(y, shifted @ w[tap], rtol=0, atol=1e-14)


def test_gradients_by_central_differences():
    D, H, W, Ci, Co = 3, 4, 3, 2, 3
    x = _rand((D, H, W, Ci), 5)
    w = _rand((27, Ci, Co), 6)
    b = _rand(Co, 7)
    g = _rand((D, H, W, Co), 8)

    def loss(xx, ww, bb):
        return float(np.sum(oracle.conv3d_fwd(xx, ww, bb) * g))

    dx = oracle.conv3d_dgrad(g, w)
    dw, db = oracle.conv3d_wgrad(x, g)
    h = 1e-6
    rng = np.random.default_rng(9)
    for _ in range(12):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss(xp, w, b) - loss(xm, w, b)) / (2 * h)
        assert abs(fd - dx[idx]) < 1e-7 * max(1.0, abs(fd))
    for _ in range(12):
        idx = tuple(rng.integers(0, s) for s in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (loss(x, wp, b) - loss(x, wm, b)) / (2 * h)
        assert abs(fd - dw[idx]) < 1e-7 * max(1.0, abs(fd))
    for o in range(Co):
        bp, bm = b.copy(), b.copy()
        bp[o] += h
        bm[o] -= h
        fd = (loss(x, w, bp) - loss(x, w, bm)) / (2 * h)
        assert abs(fd - db[o]) < 1e-7 * max(1.0, abs(fd))
