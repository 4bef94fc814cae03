"""Seeded synthetic inputs for the Gray-Scott and pointwise-ODE workloads.

This module is the only code shared between the CPU oracle's tests and the
CUDA path's tests and benchmark.  It holds no arithmetic of the time-stepping
method: it only draws random numbers and lays out initial conditions.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
draw of the stream keyed by (seed, stream) is the SplitMix64 output mix(key +
(i+1)*golden) where key = mix(seed*golden ^ mix(stream)).  The top 53 bits give
a double in [0, 1).

Workload recipes (the paper prints no data; every input is generated):

* Gray-Scott state (Eq. 2, periodic cube [0, 2.5]^3): u = 1, v = 0 except a
  centred cube, u = 0.5 and v = 0.25, covering indices [floor(3n/8),
  floor(5n/8)) on each axis (8 cells at n = 32, the same physical size at any
  n); then i.i.d. U[-0.01, 0.01] noise is added to u and to v at every cell.
* Pointwise ODE initial values: x0 ~ U(0, 1) (open interval).
* Batched ensembles: per instance, per-axis edges n_d ~ U{16..96}, feed rate
  F ~ U[0.02, 0.06], kill rate k ~ U[0.04, 0.07].
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (arbitrary distinct constants)
STREAM_NOISE_U = 1
STREAM_NOISE_V = 2
STREAM_X0 = 3
STREAM_BATCH = 4


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed], dtype=np.uint64) * _GOLDEN
        k = s ^ _mix(np.array([stream], dtype=np.uint64))
    return _mix(k)[0]


def uniform01(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start..start+count-1 of stream (seed, stream) as doubles in [0,1)."""
    key = stream_key(seed, stream)
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(key + idx * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def cube_bounds(n: int) -> tuple[int, int]:
    """Index range [lo, hi) of the centred cube along an axis of n cells."""
    return (3 * n) // 8, (5 * n) // 8


def gs_initial_state(nx: int, ny: int, nz: int, seed: int = 0,
                     noise: float = 0.01) -> tuple[np.ndarray, np.ndarray]:
    """FP64 Gray-Scott initial state (u, v), each shaped (nz, ny, nx), x fastest."""
    u = np.ones((nz, ny, nx), dtype=np.float64)
    v = np.zeros((nz, ny, nx), dtype=np.float64)
    (x0, x1), (y0, y1), (z0, z1) = cube_bounds(nx), cube_bounds(ny), cube_bounds(nz)
    u[z0:z1, y0:y1, x0:x1] = 0.5
    v[z0:z1, y0:y1, x0:x1] = 0.25
    if noise != 0.0:
        n = nx * ny * nz
        ru = uniform01(seed, STREAM_NOISE_U, n).reshape(nz, ny, nx)
        rv = uniform01(seed, STREAM_NOISE_V, n).reshape(nz, ny, nx)
        u += noise * (2.0 * ru - 1.0)
        v += noise * (2.0 * rv - 1.0)
    return u, v


def ode_initial_values(n: int, seed: int = 1) -> np.ndarray:
    """n values x0 ~ U(0,1), open interval (half-ulp offset keeps 0 out)."""
    r = uniform01(seed, STREAM_X0, n)
    return r + 0.5 / 9007199254740992.0


def batch_instances(count: int, seed: int = 3, edge_lo: int = 16, edge_hi: int = 96,
                    f_range=(0.02, 0.06), k_range=(0.04, 0.07)):
    """Per-instance grid edges and reaction parameters for a batched ensemble.

    Returns a list of dicts {nx, ny, nz, F, k}.  Edges are drawn per axis from
    the integers edge_lo..edge_hi inclusive.
    """
    r = uniform01(seed, STREAM_BATCH, 5 * count).reshape(count, 5)
    span = edge_hi - edge_lo + 1
    out = []
    for i in range(count):
        nx, ny, nz = (edge_lo + np.minimum((r[i, :3] * span).astype(np.int64), span - 1)).tolist()
        F = f_range[0] + (f_range[1] - f_range[0]) * r[i, 3]
        k = k_range[0] + (k_range[1] - k_range[0]) * r[i, 4]
        out.append({"nx": int(nx), "ny": int(ny), "nz": int(nz), "F": float(F), "k": float(k)})
    return out


# Physical constants of the Gray-Scott workloads (the paper's domain [0,2.5]^3
# with the diffusivities and rates fixed for this build; see the design notes).
GS_L = 2.5
GS_DU = 2e-5
GS_DV = 1e-5
GS_F = 0.053
GS_K = 0.014


def surrogate_init_params(seed: int = 7, last_layer_scale: float = 0.0) -> np.ndarray:
    """Initial parameters of the 4-layer conv surrogate (2-32-32-32-2, 3^3
    taps), flat FP32 vector laid out per layer as W[27][cin][cout], b[cout]:
    W ~ U(-sqrt(6/fan_in), sqrt(6/fan_in)), fan_in = 27 cin, biases 0; the
    last layer's weights are scaled by last_layer_scale (0: the initial
    network predicts no change)."""
    layers = [(2, 32), (32, 32), (32, 32), (32, 2)]
    total = sum(27 * a * b + b for a, b in layers)
    r = uniform01(seed, 5, total)
    out = np.zeros(total, dtype=np.float64)
    off = 0
    for l, (cin, cout) in enumerate(layers):
        nw = 27 * cin * cout
        bound = np.sqrt(6.0 / (27 * cin))
        w = bound * (2.0 * r[off:off + nw] - 1.0)
        if l == 3:
            w *= last_layer_scale
        out[off:off + nw] = w
        off += nw + cout
    return out.astype(np.float32)
