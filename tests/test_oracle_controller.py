"""Pins for the oracle's error norm and step-size controller (section
"Architecture and nomenclature of Boost Odeint": an error stepper, an
L-infinity norm and a controller; Table 1: Dormand-Prince 5(4)).

The paper gives the controller only in words.  The reading both the oracle
and the CUDA library implement (error order q = 4, propagated order p = 5):

    E = max_i |err_i| / (atol + rtol (|y_i| + h |k1_i|))    (y: state at the
                                                             start of the attempt)
    E > 1          reject,  dt = h max(0.9 E^(-1/(q-1)), 0.2)
    E < 0.5        accept,  dt = h 0.9 max(E, 5^-p)^(-1/p)
    0.5 <= E <= 1  accept,  dt = h
    the attempt size is clipped to t_end - t when t + dt >= t_end.

On the scalar linear problem dx/dt = -x every quantity of an attempt has a
closed form.  With z = -h, one Dormand-Prince attempt gives
    x5  = x R(z),            R(z)  = 1 + sum_k z^(k+1) b^T A^k 1,
    err = x (R - Rhat)(z),   Rhat(z) = 1 + sum_k z^(k+1) bhat^T A^k 1,
    k1  = -x,
with R, Rhat the stability polynomials of the two weight vectors, computed
here in exact rational arithmetic from the published tableau (Dormand and
Prince 1980) through the Neumann series of the nilpotent A -- a different
computation from the oracle's stage-by-stage evaluation.

Three checks per run, on runs chosen to contain a rejection with the 0.2 floor
active, a rejection without it, a kept step (0.5 <= E <= 1), growth with the
5^-5 floor active, growth without it and a clipped last step:
  1. every attempt's E against the closed form at the oracle's own h and
     state, within the rounding bound of the oracle's stage sums;
  2. every decision and the next attempt size from the oracle's own (h, E),
     to 1e-15 relative (an exact replay of the stated controller);
  3. the whole sequence simulated from the closed form alone: same
     accept/reject pattern, step sizes within the rounding growth.
Each constant of the reading, perturbed in a copy, makes check 1 or 2 fail.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

EPS = np.finfo(np.float64).eps

# Dormand-Prince 5(4) (Dormand & Prince 1980), rows of A, weights b (order 5,
# propagated) and bhat (order 4, embedded); row 7 of A equals b (FSAL).
_A = [[Fr(0)] * 7 for _ in range(7)]
_A[1][:1] = [Fr(1, 5)]
_A[2][:2] = [Fr(3, 40), Fr(9, 40)]
_A[3][:3] = [Fr(44, 45), Fr(-56, 15), Fr(32, 9)]
_A[4][:4] = [Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)]
_A[5][:5] = [Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)]
_A[6][:6] = [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)]
_B = [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), Fr(0)]
_BH = [Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200), Fr(187, 2100), Fr(1, 40)]


def _stability_poly(w):
    """Coefficients c_0..c_7 of 1 + sum_k z^(k+1) w^T A^k 1 (A^7 = 0)."""
    v = [Fr(1)] * 7
    c = [Fr(1)]
    for _ in range(7):
        c.append(sum(wi * vi for wi, vi in zip(w, v)))
        v = [sum(_A[i][j] * v[j] for j in range(7)) for i in range(7)]
    return c


_R = _stability_poly(_B)
_RH = _stability_poly(_BH)
_PERR = [a - b for a, b in zip(_R, _RH)]


def _peval(c, z):
    """Exact value of the polynomial at the binary64 number z, rounded once."""
    zf = Fr(z)
    return float(sum(ci * zf ** i for i, ci in enumerate(c)))


def test_stability_polynomials_known_forms():
    # R(z) = sum_{k<=5} z^k/k! + z^6/600 (Hairer-Norsett-Wanner I, IV.2), and the
    # embedded solution agrees with exp to order 4, so R - Rhat starts at z^5
    assert _R[:6] == [Fr(1, math.factorial(k)) for k in range(6)]
    assert _R[6] == Fr(1, 600) and _R[7] == 0
    assert all(c == 0 for c in _PERR[:5]) and _PERR[5] != 0
    assert sum(_B) == 1 and sum(_BH) == 1


# ---------------------------------------------------------------- the reading
def _scale(x, h, atol, rtol):
    return atol + rtol * (abs(x) + h * abs(-x))


def _controller(h, E, *, safety=0.9, rej_exp=-1.0 / 3.0, rej_floor=0.2, hold=0.5, grow_floor=5.0 ** -5,
                grow_exp=-1.0 / 5.0):
    """(accepted, next dt) of the stated controller from one attempt."""
    if E > 1.0:
        return False, h * max(safety * E ** rej_exp, rej_floor)
    if E < hold:
        return True, h * safety * max(E, grow_floor) ** grow_exp
    return True, h


def _replay_states(x0, h, acc):
    """x_n before every attempt, from the oracle's own accepted sizes."""
    xs, x = [], x0
    for hi, a in zip(h, acc):
        xs.append(x)
        if a:
            x = x * _peval(_R, -hi)
    return xs, x


def _rounding_bound(x, h, E, sc):
    # the oracle forms err = h sum_j e_j k_j over stages whose magnitudes stay
    # within a few |x| (|R_j(-h)| <= 3 for h <= 3), with |e_j| summing to < 0.2:
    # |err| carries a rounding error below 64 eps h |x|, plus E's own rounding.
    return 64 * EPS * h * abs(x) / sc + 8 * EPS * E


_RUNS = [
    # x0, t_end, dt0, atol, rtol
    (1.0, 2.0, 2.0, 1e-7, 1e-6),
    (1.0, 3.0, 3.0, 1e-6, 1e-6),
    (-0.8, 3.0, 1e-3, 1e-7, 1e-6),
    (0.6, 5.0, 2.5, 1e-6, 1e-7),
]


def _oracle_run(x0, t_end, dt0, atol, rtol):
    r = oracle.pw_integrate_adaptive_trace(oracle.PW_EXP_DECAY, np.array([x0]), 0.0, t_end, dt0, atol, rtol)
    assert r["status"] == oracle.OK and r["t"] == t_end
    return r


def _branches(h, E, acc):
    kinds = set()
    for e, a in zip(E, acc):
        if not a:
            kinds.add("reject_floor" if 0.9 * e ** (-1 / 3) < 0.2 else "reject")
        elif e >= 0.5:
            kinds.add("keep")
        else:
            kinds.add("grow_floor" if e < 5.0 ** -5 else "grow")
    return kinds


def test_runs_cover_every_branch():
    kinds = set()
    for run in _RUNS:
        r = _oracle_run(*run)
        kinds |= _branches(r["h"], r["E"], r["accepted"])
    assert kinds == {"reject_floor", "reject", "keep", "grow_floor", "grow"}


@pytest.mark.parametrize("run", _RUNS)
def test_norm_matches_closed_form(run):
    x0, t_end, dt0, atol, rtol = run
    r = _oracle_run(*run)
    xs, xend = _replay_states(x0, r["h"], r["accepted"])
    for x, h, E in zip(xs, r["h"], r["E"]):
        sc = _scale(x, h, atol, rtol)
        E_cf = abs(x * _peval(_PERR, -h)) / sc
        assert abs(E - E_cf) <= _rounding_bound(x, h, E, sc), (h, E, E_cf)
    # the state after the accepted steps is x0 prod R(-h) (1e-14 relative)
    assert abs(r["x"][0] - xend) <= 1e-14 * abs(xend)


@pytest.mark.parametrize("run", _RUNS)
def test_controller_replays_exactly(run):
    x0, t_end, dt0, atol, rtol = run
    r = _oracle_run(*run)
    h, E, acc = r["h"], r["E"], r["accepted"]
    assert h[0] == min(dt0, t_end)
    t = 0.0
    for a in range(len(h)):
        ok, dt_next = _controller(h[a], E[a])
        assert ok == bool(acc[a]), (a, E[a])
        if ok:
            t = t_end if t + h[a] >= t_end else t + h[a]
        if a + 1 < len(h):
            expect = t_end - t if t + dt_next >= t_end else dt_next
            assert abs(h[a + 1] - expect) <= 1e-15 * expect, (a, h[a + 1], expect)
        else:
            assert t == t_end
            assert abs(r["dt"] - dt_next) <= 1e-15 * dt_next
    # the last attempt was clipped: its size is below the controller's proposal
    assert r["h"][-1] < _controller(h[-2], E[-2])[1]


@pytest.mark.parametrize("run", _RUNS)
def test_sequence_from_closed_form_alone(run):
    """Simulate the whole run from x0, the polynomials and the reading only."""
    x0, t_end, dt0, atol, rtol = run
    r = _oracle_run(*run)
    x, t, dt, hs, accs = x0, 0.0, dt0, [], []
    while t < t_end:
        h = t_end - t if t + dt >= t_end else dt
        E = abs(x * _peval(_PERR, -h)) / _scale(x, h, atol, rtol)
        ok, dt = _controller(h, E)
        hs.append(h)
        accs.append(ok)
        if ok:
            t = t_end if t + h >= t_end else t + h
            x = x * _peval(_R, -h)
    assert accs == list(r["accepted"])
    # step sizes follow E^(-1/5) of numbers carrying the stage-sum rounding
    # (relative 1e-10 at most here); the clipped last step t_end - t inherits
    # the accumulated difference of t, absolute against t_end
    assert np.allclose(hs[:-1], r["h"][:-1], rtol=1e-10, atol=0)
    assert abs(hs[-1] - r["h"][-1]) <= 1e-10 * t_end


# --------------------------------------------------- sensitivity of the pins
_PERTURBED_CONTROLLERS = {
    "safety 0.8": dict(safety=0.8),
    "reject exponent -1/q": dict(rej_exp=-1.0 / 4.0),
    "reject floor 0.1": dict(rej_floor=0.1),
    "no reject floor": dict(rej_floor=0.0),
    "keep band from 1.0 (always grow)": dict(hold=1.0),
    "keep band from 0.25": dict(hold=0.25),
    "growth floor 10^-5": dict(grow_floor=1e-5),
    "no growth floor": dict(grow_floor=0.0),
    "growth exponent -1/q": dict(grow_exp=-1.0 / 4.0),
}


def _controller_replay_holds(r, t_end, **kw):
    h, E, acc = r["h"], r["E"], r["accepted"]
    t = 0.0
    for a in range(len(h)):
        ok, dt_next = _controller(h[a], E[a], **kw)
        if ok != bool(acc[a]):
            return False
        if ok:
            t = t_end if t + h[a] >= t_end else t + h[a]
        nxt = h[a + 1] if a + 1 < len(h) else r["dt"]
        expect = dt_next if a + 1 == len(h) else (t_end - t if t + dt_next >= t_end else dt_next)
        if abs(nxt - expect) > 1e-15 * expect:
            return False
    return True


@pytest.mark.parametrize("name", sorted(_PERTURBED_CONTROLLERS))
def test_each_controller_constant_is_pinned(name):
    kw = _PERTURBED_CONTROLLERS[name]
    held = [_controller_replay_holds(_oracle_run(*run), run[1], **kw) for run in _RUNS]
    assert not all(held), name


_PERTURBED_SCALES = {
    "new state instead of the old": lambda x, x5, h, atol, rtol: atol + rtol * (abs(x5) + h * abs(x)),
    "derivative term dropped": lambda x, x5, h, atol, rtol: atol + rtol * abs(x),
    "derivative term without h": lambda x, x5, h, atol, rtol: atol + rtol * (abs(x) + abs(x)),
    "atol and rtol swapped": lambda x, x5, h, atol, rtol: rtol + atol * (abs(x) + h * abs(x)),
    "max instead of sum": lambda x, x5, h, atol, rtol: max(atol, rtol * (abs(x) + h * abs(x))),
}


@pytest.mark.parametrize("name", sorted(_PERTURBED_SCALES))
def test_each_norm_choice_is_pinned(name):
    scale = _PERTURBED_SCALES[name]
    caught = False
    for run in _RUNS:
        x0, t_end, dt0, atol, rtol = run
        r = _oracle_run(*run)
        xs, _ = _replay_states(x0, r["h"], r["accepted"])
        for x, h, E in zip(xs, r["h"], r["E"]):
            sc = scale(x, x * _peval(_R, -h), h, atol, rtol)
            E_alt = abs(x * _peval(_PERR, -h)) / sc
            if abs(E - E_alt) > _rounding_bound(x, h, E, sc):
                caught = True
    assert caught, name


def test_error_estimate_sign_and_weights_are_pinned():
    # the embedded weights of the order-4 solution, not the order-5 ones, and
    # |err| rather than err: a dropped stage-7 term (non-FSAL reading) changes E
    r = _oracle_run(*_RUNS[0])
    xs, _ = _replay_states(_RUNS[0][0], r["h"], r["accepted"])
    bh_no7 = list(_BH[:6]) + [Fr(0)]
    perr_alt = [a - b for a, b in zip(_R, _stability_poly(bh_no7))]
    diffs = []
    for x, h, E in zip(xs, r["h"], r["E"]):
        sc = _scale(x, h, *_RUNS[0][3:])
        diffs.append(abs(E - abs(x * _peval(perr_alt, -h)) / sc) > _rounding_bound(x, h, E, sc))
    assert any(diffs)
