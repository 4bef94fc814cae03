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


def test_bf16_round_known_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties go to the even mantissa
    assert oracle.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert oracle.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert oracle.bf16_round(np.array([-2.5]))[0] == -2.5
    x = np.random.default_rng(0).standard_normal(1000)
    y = oracle.bf16_round(x)
    assert np.all(np.abs(y - x) <= np.abs(x) * 2.0 ** -8)
    assert np.array_equal(oracle.bf16_round(y), y)


def test_surrogate_gradient_by_central_differences():
    import synthetic_inputs as si
    D, H, W = 3, 4, 3
    rng = np.random.default_rng(1)
    params = si.surrogate_init_params(seed=3, last_layer_scale=0.5).astype(np.float64)
    u = 1.0 + 0.1 * rng.standard_normal((D, H, W))
    v = 0.1 * rng.standard_normal((D, H, W))
    ut = u + 0.01 * rng.standard_normal((D, H, W))
    vt = v + 0.01 * rng.standard_normal((D, H, W))
    norm = ((1.0, 0.0), (0.1, 0.1), (0.01, 0.01))
    loss, g = oracle.surrogate_loss_grad(params, u, v, ut, vt, *norm, emulate_bf16=False)
    assert g.size == oracle.surrogate_param_count() == params.size
    h = 1e-6
    idx = rng.choice(params.size, 16, replace=False)
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        lp = oracle.surrogate_loss_grad(pp, u, v, ut, vt, *norm, emulate_bf16=False)[0]
        lm = oracle.surrogate_loss_grad(pm, u, v, ut, vt, *norm, emulate_bf16=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # the forward pass agrees with the loss definition
    pu, pv = oracle.surrogate_forward(params, u, v, *norm, emulate_bf16=False)
    ref = np.mean(np.concatenate([(((pu - u) - (ut - u)) / 0.01).ravel(), (((pv - v) - (vt - v)) / 0.01).ravel()]) ** 2)
    assert abs(ref - loss) < 1e-12 * max(1.0, loss)
