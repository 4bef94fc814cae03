"""GPU parity of the pointwise ODE path (dx/dt = -x, x(1-x); FP64) and of the
stage algebra against the CPU FP64 oracle, plus closed-form checks at the
full 2^24-element size."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from tests._gpu_common import cuda_or_skip, to_np

pytestmark = pytest.mark.gpu

KINDS = [(0, oracle.PW_EXP_DECAY), (1, oracle.PW_LOGISTIC)]


def _exact(kind, x0, t):
    if kind == 0:
        return x0 * np.exp(-t)
    return x0 / (x0 + (1 - x0) * np.exp(-t))


@pytest.mark.parametrize("kind,okind", KINDS)
@pytest.mark.parametrize("n", [1, 1000, 4099])
def test_adaptive_matches_oracle_run(kind, okind, n):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    x0 = si.ode_initial_values(n, seed=1)
    x = torch.from_numpy(x0.copy()).cuda()
    log = torch.zeros(100000, dtype=torch.float64, device="cuda")
    r = gs.ode_integrate_adaptive(kind, x, 0.0, 10.0, 1e-3, 1e-8, 1e-8, dt_log=log)
    ref = oracle.pw_integrate_adaptive(okind, x0, 0.0, 10.0, 1e-3, 1e-8, 1e-8, log_cap=100000)
    assert r["status"] == 0 and r["t"] == 10.0
    assert (r["n_acc"], r["n_rej"]) == (ref["n_acc"], ref["n_rej"])
    # E is a cancelling sum: FMA vs non-FMA rounding moves it by ~1e-9
    # relative, and the step sequence carries that drift along
    d = to_np(log)[: r["n_acc"]]
    assert np.allclose(d, ref["dts"], rtol=1e-7, atol=0), np.max(np.abs(d / ref["dts"] - 1))
    assert oracle.rel_l2(to_np(x), ref["x"]) < 1e-12


@pytest.mark.parametrize("kind,okind", KINDS)
@pytest.mark.parametrize("method,omethod", [(3, oracle.EULER), (0, oracle.RK4), (1, oracle.DOPRI5)])
def test_fixed_step_matches_oracle(kind, okind, method, omethod):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    x0 = si.ode_initial_values(3001, seed=7)
    x = torch.from_numpy(x0.copy()).cuda()
    gs.ode_integrate_const(kind, method, x, 0.0, 0.05, 200)
    torch.cuda.synchronize()
    ref = oracle.pw_integrate_const(okind, x0, omethod, 0.05, 200)
    assert oracle.rel_l2(to_np(x), ref) < 1e-13


@pytest.mark.parametrize("kind,okind", KINDS)
@pytest.mark.parametrize("nsteps", [0, 1, 2, 3, 4, 50])
def test_ab4_matches_oracle(kind, okind, nsteps):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    x0 = si.ode_initial_values(777, seed=8)
    x = torch.from_numpy(x0.copy()).cuda()
    gs.ode_integrate_ab4(kind, x, 0.0, 0.01, nsteps)
    torch.cuda.synchronize()
    ref = oracle.pw_integrate_ab4(okind, x0, 0.01, nsteps)
    assert oracle.rel_l2(to_np(x), ref) < 1e-13


@pytest.mark.parametrize("kind,okind", KINDS)
def test_full_size_adaptive_closed_form(kind, okind):
    """2^24 elements, Dopri5 with atol = rtol = 1e-8 to t = 10: every element
    within a small multiple of the tolerance of the closed form."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    n = 1 << 24
    x0 = si.ode_initial_values(n, seed=1)
    x = torch.from_numpy(x0).cuda()
    r = gs.ode_integrate_adaptive(kind, x, 0.0, 10.0, 1e-3, 1e-8, 1e-8)
    assert r["status"] == 0 and r["t"] == 10.0
    err = np.max(np.abs(to_np(x) - _exact(kind, x0, 10.0)))
    assert err < 50e-8, err


@pytest.mark.parametrize("kind,okind", KINDS)
def test_full_size_ab4_sampled(kind, okind):
    """2^24 elements, AB4 at dt = 1e-3 for 10^4 steps; 2048 sampled elements
    against the oracle, all against the closed form."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    n = 1 << 24
    x0 = si.ode_initial_values(n, seed=1)
    x = torch.from_numpy(x0).cuda()
    gs.ode_integrate_ab4(kind, x, 0.0, 1e-3, 10000)
    got = to_np(x)
    idx = np.random.default_rng(3).choice(n, 2048, replace=False)
    ref = oracle.pw_integrate_ab4(okind, x0[idx], 1e-3, 10000)
    assert oracle.rel_l2(got[idx], ref) < 1e-12
    assert np.max(np.abs(got - _exact(kind, x0, 10.0))) < 1e-10


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nterms", [1, 2, 7, 15])
@pytest.mark.parametrize("n", [1, 5, 4096, 10007])
def test_axpy_stage(prec, nterms, n):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(nterms * 100 + n)
    xs_np = [rng.standard_normal(n) for _ in range(nterms)]
    coef = rng.standard_normal(nterms)
    if prec == "f32":
        xs_np = [x.astype(np.float32).astype(np.float64) for x in xs_np]
        coef = coef.astype(np.float32).astype(np.float64)
    xs = [torch.from_numpy(x).to("cuda", dt) for x in xs_np]
    y = torch.empty(n, dtype=dt, device="cuda")
    gs.ode_axpy_stage(coef, xs, y)
    ref = oracle.axpy(coef, xs_np)
    tol = 1e-15 if prec == "f64" else 1e-6
    scale = sum(abs(c) * np.abs(x) for c, x in zip(coef, xs_np))
    assert np.all(np.abs(to_np(y) - ref) <= tol * nterms * scale + 1e-300)
    # aliasing: y is one of the operands
    gs.ode_axpy_stage(coef, xs, xs[0])
    assert np.array_equal(to_np(xs[0]), to_np(y))


def test_axpy_exact_integers():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    xs_np = [np.arange(1001.0) * (j + 1) for j in range(15)]
    coef = np.array([(-1.0) ** j * (j + 1) for j in range(15)])
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    y = torch.empty(1001, dtype=torch.float64, device="cuda")
    gs.ode_axpy_stage(coef, xs, y)
    assert np.array_equal(to_np(y), oracle.axpy(coef, xs_np))


def test_fp64_peak_probe_is_positive():
    cuda_or_skip()
    import paper_2309_05331_b300 as gs
    v = gs.gs_measure_fp64_peak()
    assert 0.1 < v < 200.0
