"""Pins for the oracle's error-controlled Dormand-Prince 5(4) driver.

The paper specifies an error stepper, a tolerance and (usually) an
L-infinity norm, but no controller formula; the controller is this build's
reading.  What the mathematics fixes, and what is checked here:

* global error at t_end on closed-form problems stays within a small multiple
  of the tolerance, and shrinks as the tolerance shrinks;
* the number of accepted steps grows like tol^(-1/5) (fifth-order method);
* the final step is clipped so t lands exactly on t_end;
* dt-replay: re-running the accepted step sizes as fixed steps reproduces the
  adaptive result bit for bit (the replay used by GPU parity tests);
* failure statuses: non-finite state, unreachable tolerance.
"""
import math

import numpy as np
import pytest

import oracle


def _exact(kind, x0, t):
    if kind == oracle.PW_EXP_DECAY:
        return x0 * np.exp(-t)
    e = np.exp(-t)
    return x0 / (x0 + (1 - x0) * e)


@pytest.mark.parametrize("kind", [oracle.PW_EXP_DECAY, oracle.PW_LOGISTIC])
def test_error_within_tolerance_multiple(kind):
    x0 = np.linspace(0.01, 0.99, 33)
    errs, steps = [], []
    for tol in (1e-6, 1e-8, 1e-10):
        r = oracle.pw_integrate_adaptive(kind, x0, 0.0, 10.0, 1e-3, tol, tol)
        assert r["status"] == oracle.OK
        assert r["t"] == 10.0
        e = oracle.linf(r["x"] - _exact(kind, x0, 10.0))
        assert e < 50 * tol, (tol, e)
        errs.append(e)
        steps.append(r["n_acc"])
    assert errs[0] > errs[1] > errs[2]
    # accepted steps ~ tol^(-1/5): a factor 100 in tol gives 100^(1/5) = 2.5
    for a, b in zip(steps, steps[1:]):
        assert 1.8 < b / a < 3.5, steps


def test_replay_reproduces_adaptive_run_bitwise():
    x0 = np.linspace(0.05, 0.95, 11)
    r = oracle.pw_integrate_adaptive(oracle.PW_LOGISTIC, x0, 0.0, 10.0, 1e-3, 1e-8, 1e-8, log_cap=10000)
    assert r["n_acc"] == len(r["dts"])
    x = oracle.pw_integrate_replay(oracle.PW_LOGISTIC, x0, oracle.DOPRI5, r["dts"])
    assert np.array_equal(x, r["x"])


def test_max_accepted_mode():
    x0 = np.array([0.3, 0.6])
    r = oracle.pw_integrate_adaptive(oracle.PW_EXP_DECAY, x0, 0.0, math.inf, 1e-3, 1e-8, 1e-8,
                                     max_acc=25)
    assert r["status"] == oracle.OK and r["n_acc"] == 25 and r["t"] < math.inf


def test_step_growth_is_bounded():
    # from a tiny dt0 the controller may grow dt by at most 4.5x per step
    x0 = np.array([0.5])
    r = oracle.pw_integrate_adaptive(oracle.PW_EXP_DECAY, x0, 0.0, 1.0, 1e-9, 1e-6, 1e-6, log_cap=1000)
    d = r["dts"]
    assert np.all(d[1:] / d[:-1] <= 4.5 * (1 + 1e-12))
    assert abs(np.sum(d) - 1.0) < 1e-12


def test_nonfinite_state_is_reported():
    x0 = np.array([0.5, np.nan, 0.2])
    r = oracle.pw_integrate_adaptive(oracle.PW_EXP_DECAY, x0, 0.0, 1.0, 1e-3, 1e-8, 1e-8)
    assert r["status"] == oracle.ERR_NONFINITE


def test_unreachable_tolerance_underflows():
    x0 = np.array([0.5, 0.7])
    r = oracle.pw_integrate_adaptive(oracle.PW_LOGISTIC, x0, 0.0, 1.0, 1e-1, 0.0, 1e-300, max_rej=50)
    assert r["status"] == oracle.ERR_STEP_UNDERFLOW


def test_gs_adaptive_small_grid_consistency():
    # adaptive GS on 8^3: error vs a fine fixed-step RK4 solution is O(tol)
    import synthetic_inputs as si
    p = oracle.GSParams(8, 8, 8, Du=2e-3, Dv=1e-3)
    u0, v0 = si.gs_initial_state(8, 8, 8, seed=2)
    ref = oracle.gs_integrate_const(p, u0, v0, oracle.RK4, 0.01, 500)
    r = oracle.gs_integrate_adaptive(p, u0, v0, 0.0, 5.0, 0.1, 1e-7, 1e-7, log_cap=1000)
    assert r["status"] == oracle.OK and r["t"] == 5.0
    err = oracle.rel_l2([r["u"], r["v"]], list(ref))
    assert err < 1e-6
    # replay of the accepted steps is bitwise identical
    u, v = oracle.gs_integrate_replay(p, u0, v0, oracle.DOPRI5, r["dts"])
    assert np.array_equal(u, r["u"]) and np.array_equal(v, r["v"])
