"""Pins for the oracle's Gray-Scott system (Eq. 2, Listing 2) and its
integrators, against closed forms of the mathematics.

* 7-point periodic Laplacian: Fourier modes are eigenvectors with eigenvalue
  -sum_d (4/h_d^2) sin^2(pi m_d / n_d) (anisotropic grids, odd sizes), and
  the sum over the periodic grid of Lap(w) is zero.
* Reaction: u=1, v=0 and the two uniform nontrivial steady states
  v = (F +- sqrt(F^2 - 4F(F+k)^2)) / (2(F+k)), u = (F+k)/v are fixed points.
* Linear sub-case v = 0, u = 1 + eps*mode: u - 1 obeys w' = lambda w with
  lambda = -(Du mu + F), so n steps of a Runge-Kutta method give exactly
  R(lambda dt)^n (R the stability polynomial).
* Symmetry of the noiseless cube initial state under axis permutations and
  reflections.
* Self-convergence order of RK4 / Dopri5 on the full nonlinear problem.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as si


def _mode(p, m):
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    return np.cos(2 * np.pi * (m[0] * x / p.nx + m[1] * y / p.ny + m[2] * z / p.nz))


def _mu(p, m):
    h = (p.Lx / p.nx, p.Ly / p.ny, p.Lz / p.nz)
    n = (p.nx, p.ny, p.nz)
    return sum(4.0 / h[d] ** 2 * math.sin(math.pi * m[d] / n[d]) ** 2 for d in range(3))


@pytest.mark.parametrize("dims,m", [((8, 8, 8), (1, 2, 3)), ((9, 6, 5), (2, 1, 2)),
                                    ((16, 4, 7), (5, 0, 3)), ((3, 1, 2), (1, 0, 1))])
def test_laplacian_fourier_eigenvalues(dims, m):
    p = oracle.GSParams(*dims, L=2.5, Ly=1.7, Lz=3.1)
    w = _mode(p, m)
    lap = oracle.gs_laplacian(p, w)
    assert np.allclose(lap, -_mu(p, m) * w, atol=1e-9 * _mu(p, m), rtol=0)


def test_laplacian_sums_to_zero():
    p = oracle.GSParams(7, 5, 6)
    rng = np.random.default_rng(0)
    w = rng.standard_normal((6, 5, 7))
    lap = oracle.gs_laplacian(p, w)
    scale = np.max(np.abs(lap))
    assert abs(lap.sum()) < 1e-12 * scale * lap.size


def _steady_states(F, k):
    disc = F * F - 4 * F * (F + k) ** 2
    out = [(1.0, 0.0)]
    if disc > 0:
        for sgn in (+1, -1):
            v = (F + sgn * math.sqrt(disc)) / (2 * (F + k))
            out.append(((F + k) / v, v))
    return out


@pytest.mark.parametrize("F,k", [(0.053, 0.014), (0.03, 0.05), (0.05, 0.055)])
def test_uniform_steady_states_are_fixed_points(F, k):
    p = oracle.GSParams(4, 3, 5, F=F, k=k)
    sts = _steady_states(F, k)
    assert len(sts) == 3
    for (us, vs) in sts:
        u = np.full((5, 3, 4), us)
        v = np.full((5, 3, 4), vs)
        fu, fv = oracle.gs_rhs(p, u, v)
        assert np.max(np.abs(fu)) < 1e-15 and np.max(np.abs(fv)) < 1e-15
    # a perturbed uniform state is not a fixed point (the test can fail)
    fu, fv = oracle.gs_rhs(p, np.full((5, 3, 4), 0.9), np.full((5, 3, 4), 0.1))
    assert np.max(np.abs(fu)) > 1e-4


def _R(method, z):
    if method == oracle.RK4:
        return sum(z ** j / math.factorial(j) for j in range(5))
    return sum(z ** j / math.factorial(j) for j in range(6)) + z ** 6 / 600.0


@pytest.mark.parametrize("method", [oracle.RK4, oracle.DOPRI5])
def test_linear_subcase_exact_discrete_solution(method):
    # large diffusivity so the Laplacian term matters at this dt
    p = oracle.GSParams(8, 6, 10, L=2.5, Ly=2.0, Lz=3.0, Du=2e-2, Dv=1e-2, F=0.053, k=0.014)
    m = (1, 2, 3)
    eps = 1e-3
    mode = _mode(p, m)
    u0 = 1.0 + eps * mode
    v0 = np.zeros_like(u0)
    dt, n = 0.1, 25
    u, v = oracle.gs_integrate_const(p, u0, v0, method, dt, n)
    lam = -(p.Du * _mu(p, m) + p.F)
    expect = 1.0 + eps * _R(method, lam * dt) ** n * mode
    assert np.array_equal(v, np.zeros_like(v))
    assert np.max(np.abs(u - expect)) < 1e-14


def test_noiseless_cube_symmetries():
    n = 16
    p = oracle.GSParams(n, n, n, Du=2e-3, Dv=1e-3)
    u0, v0 = si.gs_initial_state(n, n, n, noise=0.0)
    u, v = oracle.gs_integrate_const(p, u0, v0, oracle.RK4, 0.5, 6)
    for w in (u, v):
        assert np.max(np.abs(w - np.transpose(w, (1, 0, 2)))) < 1e-14
        assert np.max(np.abs(w - np.transpose(w, (2, 1, 0)))) < 1e-14
        # cube [6,10) is symmetric under i -> n-1-i
        assert np.max(np.abs(w - w[::-1, :, :])) < 1e-14
        assert np.max(np.abs(w - w[:, :, ::-1])) < 1e-14
    # the dynamics moved the state (the symmetry test is not vacuous)
    assert np.max(np.abs(u - u0)) > 1e-3


@pytest.mark.parametrize("method,order", [(oracle.RK4, 4), (oracle.DOPRI5, 5)])
def test_gs_self_convergence(method, order):
    n = 8
    p = oracle.GSParams(n, n, n, Du=2e-3, Dv=1e-3)
    u0, v0 = si.gs_initial_state(n, n, n, seed=5)
    T = 4.0
    sols = [oracle.gs_integrate_const(p, u0, v0, method, T / m, m) for m in (4, 8, 16)]
    e1 = oracle.rel_l2(list(sols[0]), list(sols[1]))
    e2 = oracle.rel_l2(list(sols[1]), list(sols[2]))
    assert abs(math.log2(e1 / e2) - order) < 0.5, (e1, e2)


def test_gs_ab4_self_convergence():
    n = 8
    p = oracle.GSParams(n, n, n, Du=2e-3, Dv=1e-3)
    u0, v0 = si.gs_initial_state(n, n, n, seed=6)
    T = 4.0
    sols = [oracle.gs_integrate_ab4(p, u0, v0, T / m, m) for m in (16, 32, 64)]
    e1 = oracle.rel_l2(list(sols[0]), list(sols[1]))
    e2 = oracle.rel_l2(list(sols[1]), list(sols[2]))
    assert abs(math.log2(e1 / e2) - 4) < 0.5, (e1, e2)


def test_gs_uniform_state_reduces_to_reaction_ode():
    # with no spatial variation the Laplacian vanishes and every cell follows
    # the same reaction ODE; compare with scipy's DOP853 at tight tolerance on
    # the rates read off the oracle's own RHS at the current state
    from scipy.integrate import solve_ivp
    p = oracle.GSParams(3, 4, 2)

    def f(t, y):
        fu, fv = oracle.gs_rhs(p, np.full((2, 4, 3), y[0]), np.full((2, 4, 3), y[1]))
        return [fu[0, 0, 0], fv[0, 0, 0]]

    y0 = [0.6, 0.3]
    ref = solve_ivp(f, (0, 5), y0, method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    u, v = oracle.gs_integrate_const(p, np.full((2, 4, 3), y0[0]), np.full((2, 4, 3), y0[1]),
                                     oracle.RK4, 0.01, 500)
    assert abs(u[0, 0, 0] - ref[0]) < 1e-9 and abs(v[0, 0, 0] - ref[1]) < 1e-9
    assert np.ptp(u) == 0.0 and np.ptp(v) == 0.0


# ------------------------------------------- DC-PSE Laplacian (the paper's operator)
def _mono_lap_at_0(e):
    """Laplacian at the origin of x^a y^b z^c."""
    return 2.0 if (sum(e) == 2 and max(e) == 2) else 0.0


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.1, 0.2, 0.3), (2.5 / 64, 2.5 / 64, 2.5 / 64)])
def test_dcpse_exact_on_cubics_not_quartics(h):
    # the moment conditions make the stencil reproduce the Laplacian of every
    # polynomial of degree <= 3 (r = 2, |beta| = 2), and no more
    off, w = oracle.dcpse_stencil(h, 3.1)
    x = off * np.asarray(h)
    assert len(w) == 122  # integer offsets with |o| <= 3.1, o != 0
    import itertools
    scale = 1.0 / min(h) ** 2
    worst4 = 0.0
    for deg in range(0, 5):
        for e in itertools.product(range(deg + 1), repeat=3):
            if sum(e) != deg:
                continue
            vals = np.prod(x ** np.array(e), axis=1)
            lap = float(np.sum(w * (vals - (1.0 if deg == 0 else 0.0))))
            if deg <= 3:
                assert abs(lap - _mono_lap_at_0(e)) < 1e-12 * scale * max(1.0, float(np.abs(w * vals).sum())), (e, lap)
            else:
                worst4 = max(worst4, abs(lap - _mono_lap_at_0(e)) / max(h) ** 2)
    assert worst4 > 1e-3


def test_dcpse_weights_symmetric():
    off, w = oracle.dcpse_stencil((1.0, 1.0, 1.0), 3.1)
    table = {tuple(o): wi for o, wi in zip(off.tolist(), w)}
    for o, wi in table.items():
        assert abs(table[(-o[0], -o[1], -o[2])] - wi) < 1e-14 * abs(wi) + 1e-18
        assert abs(table[(o[1], o[2], o[0])] - wi) < 1e-12 * abs(wi) + 1e-16


def test_dcpse_second_order_convergence():
    # Du = 1, v = 0, F = k = 0: the right-hand side is the Laplacian of u;
    # u = sin(2 pi x / L) sin(4 pi y / L) cos(2 pi z / L) has Lap u = -(24 pi^2 / L^2) u
    errs = []
    L = 2.5
    for n in (16, 32):
        p = oracle.GSParams(n, n, n, L=L, Du=1.0, Dv=0.0, F=0.0, k=0.0)
        c = (np.arange(n) + 0.0) * (L / n)
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        u = np.sin(2 * np.pi * X / L) * np.sin(4 * np.pi * Y / L) * np.cos(2 * np.pi * Z / L)
        fu, _ = oracle.gs_dcpse_rhs(p, u.reshape(-1), np.zeros(n ** 3))
        exact = -(24 * np.pi ** 2 / L ** 2) * u.reshape(-1)
        errs.append(np.max(np.abs(np.asarray(fu).reshape(-1) - exact)))
    assert abs(np.log2(errs[0] / errs[1]) - 2.0) < 0.25, errs


def test_dcpse_gs_fixed_point_and_reaction():
    # the uniform state u = 1, v = 0 is a fixed point; a uniform field sees
    # the reaction terms only (the stencil annihilates constants)
    n = 8
    p = oracle.GSParams(n, n, n, L=2.5, Du=2e-4, Dv=1e-4, F=0.053, k=0.014)
    u = np.ones(n ** 3)
    v = np.zeros(n ** 3)
    uo, vo = oracle.gs_dcpse_integrate_const(p, u, v, oracle.RK4, 1.0, 5)
    assert np.array_equal(np.asarray(uo).reshape(-1), u) and np.array_equal(np.asarray(vo).reshape(-1), v)
    u = np.full(n ** 3, 0.4)
    v = np.full(n ** 3, 0.3)
    fu, fv = oracle.gs_dcpse_rhs(p, u, v)
    assert np.allclose(fu, -0.4 * 0.09 + 0.053 * 0.6, rtol=1e-14, atol=1e-17)
    assert np.allclose(fv, 0.4 * 0.09 - 0.067 * 0.3, rtol=1e-14, atol=1e-17)


def test_thread_count_does_not_change_results():
    # the oracle's loops over cells may be shared among threads; every cell's
    # operations and their order stay the same, so results are bit-identical.
    # Run in a child process: OpenMP's thread pool must not meet a later fork.
    import subprocess
    import sys
    code = r"""
import numpy as np, oracle, synthetic_inputs as si
p = oracle.GSParams(24, 20, 18, Du=2e-3, Dv=1e-3)
u0, v0 = si.gs_initial_state(24, 20, 18, seed=3)
out = []
for th in (1, 4):
    oracle.set_threads(th)
    assert oracle.get_threads() == th
    a = oracle.gs_integrate_const(p, u0, v0, oracle.DOPRI5, 0.2, 3)
    b = oracle.gs_integrate_adaptive(p, u0, v0, 0.0, 2.0, 0.1, 1e-7, 1e-7, log_cap=100)
    out.append((a, b))
(a1, b1), (a4, b4) = out
assert all(np.array_equal(x, y) for x, y in zip(a1, a4))
assert np.array_equal(b1["u"], b4["u"]) and np.array_equal(b1["v"], b4["v"])
assert np.array_equal(b1["dts"], b4["dts"]) and b1["n_rej"] == b4["n_rej"]
print("ok")
"""
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
