"""Brute-force pin of the oracle's Gray-Scott right-hand side (Eq. 2 with the
v-equation of Listing 2) and of one Runge-Kutta step on it, on 8^3 grids.

The periodic 7-point Laplacian is built here as a dense N x N matrix from its
definition -- for every cell i and axis d, weight 1/h_d^2 on the cell's two
periodic neighbours along d and -2/h_d^2 on itself, accumulated entry by
entry so that coinciding neighbours (n_d = 2) or the cell itself (n_d = 1)
add up -- and applied by a matrix-vector product.  The reaction terms are
evaluated on whole arrays, and the RK4 / Dormand-Prince steps are the
textbook stage formulas written out with the dense right-hand side.  Nothing
here calls the oracle's stencil loops or its generic tableau step; the two
must agree element by element (1e-14 of the terms' magnitude).
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

EPS = np.finfo(np.float64).eps


def _dense_laplacian(p):
    n = (p.nx, p.ny, p.nz)
    h = (p.Lx / p.nx, p.Ly / p.ny, p.Lz / p.nz)
    N = p.nx * p.ny * p.nz
    L = np.zeros((N, N))
    absL = np.zeros((N, N))
    for z in range(p.nz):
        for y in range(p.ny):
            for x in range(p.nx):
                i = x + p.nx * (y + p.ny * z)
                c = [x, y, z]
                for d in range(3):
                    w = 1.0 / (h[d] * h[d])
                    for s in (-1, 1):
                        q = list(c)
                        q[d] = (q[d] + s) % n[d]
                        j = q[0] + p.nx * (q[1] + p.ny * q[2])
                        L[i, j] += w
                        absL[i, j] += w
                    L[i, i] -= 2.0 * w
                    absL[i, i] += 2.0 * w
    return L, absL


def _rhs_dense(p, L, u, v):
    uvv = u * v * v
    fu = p.Du * (L @ u) - uvv + p.F * (1.0 - u)
    fv = p.Dv * (L @ v) + uvv - (p.F + p.k) * v
    return fu, fv


def _rhs_magnitude(p, absL, u, v):
    """Sum of the magnitudes of every term of F, per element (rounding scale)."""
    a = np.abs
    uvv = a(u * v * v)
    mu = p.Du * (absL @ a(u)) + uvv + a(p.F) * (1.0 + a(u))
    mv = p.Dv * (absL @ a(v)) + uvv + a(p.F + p.k) * a(v)
    return mu, mv


_GRIDS = [
    ((8, 8, 8), dict(L=2.5)),
    ((8, 8, 8), dict(L=2.5, Ly=1.3, Lz=3.7)),
    ((8, 4, 2), dict(L=2.5)),      # n_z = 2: both z-neighbours are the same cell
    ((8, 3, 1), dict(L=2.5)),      # n_z = 1: the z-term vanishes
]


def _state(dims, seed):
    u0, v0 = si.gs_initial_state(*dims, seed=seed)
    return u0.reshape(-1), v0.reshape(-1)


def test_dense_laplacian_definition_sanity():
    p = oracle.GSParams(8, 8, 8)
    L, _ = _dense_laplacian(p)
    # rows sum to zero (constants are annihilated); the matrix is symmetric
    assert np.max(np.abs(L.sum(axis=1))) < 1e-12 * np.max(np.abs(L))
    assert np.array_equal(L, L.T)
    # 7 nonzeros per row on an 8^3 grid
    assert np.all(np.count_nonzero(L, axis=1) == 7)


@pytest.mark.parametrize("dims,geo", _GRIDS)
@pytest.mark.parametrize("phys", [dict(Du=2e-5, Dv=1e-5, F=0.053, k=0.014),
                                  dict(Du=2e-2, Dv=1e-2, F=0.03, k=0.06)])
def test_rhs_matches_dense_brute_force(dims, geo, phys):
    p = oracle.GSParams(*dims, **geo, **phys)
    L, absL = _dense_laplacian(p)
    u, v = _state(dims, seed=11)
    fu, fv = oracle.gs_rhs(p, u.reshape(dims[::-1]), v.reshape(dims[::-1]))
    eu, ev = _rhs_dense(p, L, u, v)
    mu, mv = _rhs_magnitude(p, absL, u, v)
    assert np.all(np.abs(fu.reshape(-1) - eu) <= 1e-14 * mu + 1e-300)
    assert np.all(np.abs(fv.reshape(-1) - ev) <= 1e-14 * mv + 1e-300)
    # the comparison is not vacuous: diffusion and reaction both contribute
    assert np.max(np.abs(p.Du * (L @ u))) > 1e-7 and np.max(np.abs(eu)) > 1e-4


def _rk4_dense(p, L, u, v, dt):
    F = lambda a, b: _rhs_dense(p, L, a, b)
    k1 = F(u, v)
    k2 = F(u + dt / 2 * k1[0], v + dt / 2 * k1[1])
    k3 = F(u + dt / 2 * k2[0], v + dt / 2 * k2[1])
    k4 = F(u + dt * k3[0], v + dt * k3[1])
    return tuple(w + dt / 6 * (a + 2 * b + 2 * c + d) for w, a, b, c, d in zip((u, v), k1, k2, k3, k4))


def _dopri5_dense(p, L, u, v, dt):
    F = lambda a, b: _rhs_dense(p, L, a, b)
    k1 = F(u, v)
    Y = lambda *terms: tuple(w + dt * sum(c * k[i] for c, k in terms) for i, w in enumerate((u, v)))
    k2 = F(*Y((1 / 5, k1)))
    k3 = F(*Y((3 / 40, k1), (9 / 40, k2)))
    k4 = F(*Y((44 / 45, k1), (-56 / 15, k2), (32 / 9, k3)))
    k5 = F(*Y((19372 / 6561, k1), (-25360 / 2187, k2), (64448 / 6561, k3), (-212 / 729, k4)))
    k6 = F(*Y((9017 / 3168, k1), (-355 / 33, k2), (46732 / 5247, k3), (49 / 176, k4), (-5103 / 18656, k5)))
    return Y((35 / 384, k1), (500 / 1113, k3), (125 / 192, k4), (-2187 / 6784, k5), (11 / 84, k6))


@pytest.mark.parametrize("dims,geo", _GRIDS)
@pytest.mark.parametrize("method", ["rk4", "dopri5"])
def test_one_step_matches_dense_brute_force(dims, geo, method):
    p = oracle.GSParams(*dims, **geo, Du=2e-2, Dv=1e-2, F=0.053, k=0.014)
    L, _ = _dense_laplacian(p)
    u, v = _state(dims, seed=12)
    dt = 0.05
    shape = dims[::-1]
    if method == "rk4":
        ou, ov = oracle.gs_integrate_const(p, u.reshape(shape), v.reshape(shape), oracle.RK4, dt, 1)
        eu, ev = _rk4_dense(p, L, u, v, dt)
    else:
        ou, ov = oracle.gs_integrate_const(p, u.reshape(shape), v.reshape(shape), oracle.DOPRI5, dt, 1)
        eu, ev = _dopri5_dense(p, L, u, v, dt)
    # the step's increment dt * sum b_i k_i is bounded by dt * max|k| ~ 1e-2 here,
    # so 1e-14 absolute on values of order 1 is the rounding scale
    assert np.max(np.abs(ou.reshape(-1) - eu)) <= 1e-14
    assert np.max(np.abs(ov.reshape(-1) - ev)) <= 1e-14
    assert np.max(np.abs(eu - u)) > 1e-4  # the step moved the state


@pytest.mark.parametrize("dims,geo", _GRIDS[:3])
def test_error_estimate_matches_dense_brute_force(dims, geo):
    """One Dormand-Prince attempt: y5, err = dt sum_j (b_j - bhat_j) k_j with
    k7 = F(y5), and the scaled L-infinity norm, against the dense stages."""
    p = oracle.GSParams(*dims, **geo, Du=2e-2, Dv=1e-2, F=0.053, k=0.014)
    L, _ = _dense_laplacian(p)
    u, v = _state(dims, seed=13)
    dt, atol, rtol = 0.3, 1e-7, 1e-6
    F = lambda a, b: _rhs_dense(p, L, a, b)
    k = [F(u, v)]
    A = [[], [1 / 5], [3 / 40, 9 / 40], [44 / 45, -56 / 15, 32 / 9],
         [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
         [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
         [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84]]
    for i in range(1, 7):
        k.append(F(*(w + dt * sum(a * kj[c] for a, kj in zip(A[i], k)) for c, w in enumerate((u, v)))))
    y5 = [w + dt * sum(a * kj[c] for a, kj in zip(A[6], k)) for c, w in enumerate((u, v))]
    e = [71 / 57600, 0.0, -71 / 16695, 71 / 1920, -17253 / 339200, 22 / 525, -1 / 40]
    err = [dt * sum(ej * kj[c] for ej, kj in zip(e, k)) for c in range(2)]
    E = max(np.max(np.abs(err[c]) / (atol + rtol * (np.abs(w) + dt * np.abs(k[0][c]))))
            for c, w in enumerate((u, v)))
    shape = dims[::-1]
    ou, ov, eu, ev, Eo = oracle.gs_dopri5_attempt(p, u.reshape(shape), v.reshape(shape), dt, atol, rtol)
    assert np.max(np.abs(ou.reshape(-1) - y5[0])) <= 1e-14 and np.max(np.abs(ov.reshape(-1) - y5[1])) <= 1e-14
    # err is a difference of stage sums of size ~dt max|k|: 1e-15 absolute
    assert np.max(np.abs(eu.reshape(-1) - err[0])) <= 1e-15 and np.max(np.abs(ev.reshape(-1) - err[1])) <= 1e-15
    assert abs(Eo - E) <= 1e-15 / (atol + rtol * 0.5) and Eo > 1e-2
