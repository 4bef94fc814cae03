"""Pins for the oracle's steppers (Table 1) against mathematics, not itself.

* Butcher order conditions, generated from rooted trees (Butcher's theory of
  order: sum_i b_i Phi_i(t) = 1/gamma(t) for every tree t with |t| <= p).
* Stability polynomials R(z) of RK4 (sum_{k<=4} z^k/k!) and Dormand-Prince 5
  (sum_{k<=5} z^k/k! + z^6/600, Hairer-Norsett-Wanner Vol. I): on dx/dt = -x
  one step multiplies x by R(-dt) exactly.
* Observed orders of convergence on closed-form solutions, as in the paper's
  accuracy benchmarks (Fig. 2, Eq. 1a and 1b): Euler 1, RK4 4, Dopri5 5,
  AB4 4; the embedded estimate's local error is O(dt^5).
"""
import math

import numpy as np
import pytest

import oracle


# ---------------------------------------------------------------- rooted trees
def _trees(order):
    """All rooted trees with `order` nodes, as sorted tuples of child subtrees."""
    if order == 1:
        return [()]
    out = set()

    def partitions(n, maxpart):
        if n == 0:
            yield []
            return
        for p in range(min(n, maxpart), 0, -1):
            for rest in partitions(n - p, p):
                yield [p] + rest

    for parts in partitions(order - 1, order - 1):
        # choose a tree for each part (multisets)
        def build(idx, acc):
            if idx == len(parts):
                out.add(tuple(sorted(acc)))
                return
            for t in _trees(parts[idx]):
                build(idx + 1, acc + [t])
        build(0, [])
    return sorted(out)


def _size(t):
    return 1 + sum(_size(c) for c in t)


def _gamma(t):
    g = _size(t)
    for c in t:
        g *= _gamma(c)
    return g


def _phi(t, A):
    """Elementary weight vector Phi_i(t) = prod_children (A @ Phi(child))_i."""
    s = A.shape[0]
    v = np.ones(s)
    for c in t:
        v = v * (A @ _phi(c, A))
    return v


def test_tree_enumeration_counts():
    # number of rooted trees: 1, 1, 2, 4, 9, 20 (OEIS A000081)
    assert [len(_trees(n)) for n in range(1, 7)] == [1, 1, 2, 4, 9, 20]


@pytest.mark.parametrize("method,weights,order", [
    (oracle.EULER, "b", 1),
    (oracle.RK4, "b", 4),
    (oracle.DOPRI5, "b", 5),
    (oracle.DOPRI5, "bhat", 4),
    (oracle.MIDPOINT, "b", 2),
])
def test_order_conditions(method, weights, order):
    T = oracle.tableau(method)
    A, b = T["A"], T[weights]
    # row-sum condition c_i = sum_j a_ij
    assert np.allclose(A.sum(axis=1), T["c"], atol=1e-15, rtol=0)
    for p in range(1, order + 1):
        for t in _trees(p):
            assert abs(b @ _phi(t, A) - 1.0 / _gamma(t)) < 1e-14, (p, t)
    # and the method is NOT of the next order (some condition fails)
    worst = max(abs(b @ _phi(t, A) - 1.0 / _gamma(t)) for t in _trees(order + 1))
    assert worst > 1e-6


def test_dopri5_fsal_and_error_weights():
    T = oracle.tableau(oracle.DOPRI5)
    A, b, bh = T["A"], T["b"], T["bhat"]
    assert np.array_equal(A[6, :], b)  # last stage evaluates F at the new solution
    assert abs(np.sum(b - bh)) < 1e-16


# ------------------------------------------------------- stability polynomials
def _R_rk4(z):
    return sum(z ** k / math.factorial(k) for k in range(5))


def _R_dopri5(z):
    return sum(z ** k / math.factorial(k) for k in range(6)) + z ** 6 / 600.0


def _R_midpoint(z):
    # two substeps of h = dt/2 on x' = lambda x, written out: z1 = (1 + z/2) x,
    # z2 = x + z z1, x' = (z1 + z2 + (z/2) z2) / 2  ->  1 + z + z^2/2 + z^3/8
    z1 = 1 + z / 2
    z2 = 1 + z * z1
    return (z1 + z2 + z / 2 * z2) / 2


@pytest.mark.parametrize("method,R", [(oracle.RK4, _R_rk4), (oracle.DOPRI5, _R_dopri5),
                                      (oracle.EULER, lambda z: 1 + z), (oracle.MIDPOINT, _R_midpoint)])
def test_exact_discrete_solution_decay(method, R):
    x0 = np.array([0.1, 0.5, 0.9, 1.7])
    for dt in (0.05, 0.3, 1.0):
        n = 20
        x = oracle.pw_integrate_const(oracle.PW_EXP_DECAY, x0, method, dt, n)
        expect = x0 * R(-dt) ** n
        assert np.allclose(x, expect, rtol=1e-13, atol=0)


# ------------------------------------------------------------ convergence order
def _closed_form(kind, x0, t0, t1, coef=None):
    if kind == oracle.PW_EXP_DECAY:
        return x0 * np.exp(-(t1 - t0))
    if kind == oracle.PW_LOGISTIC:
        e = np.exp(-(t1 - t0))
        return x0 / (x0 + (1 - x0) * e)
    if kind == oracle.PW_PAPER_EXP:  # u = c e^t
        return coef * np.exp(t1)
    if kind == oracle.PW_PAPER_SIGMOID:  # u = sigma(t)
        return 1.0 / (1.0 + np.exp(-t1))
    raise ValueError


def _family(kind):
    """Initial data and interval of each benchmark family."""
    if kind in (oracle.PW_EXP_DECAY, oracle.PW_LOGISTIC):
        x0 = np.linspace(0.05, 0.95, 7)
        return x0, 0.0, 10.0, None
    if kind == oracle.PW_PAPER_EXP:
        # Eq. 1a on a 4x4 grid of (x, y) in [0,1]^2, t from -5 to 5
        g = np.linspace(0.0, 1.0, 4)
        coef = np.outer(g, g).reshape(-1)
        return coef * np.exp(-5.0), -5.0, 5.0, coef
    x0 = np.array([1.0 / (1.0 + np.exp(5.0))])
    return x0, -5.0, 5.0, None


@pytest.mark.parametrize("kind", [oracle.PW_EXP_DECAY, oracle.PW_LOGISTIC, oracle.PW_PAPER_EXP,
                                  oracle.PW_PAPER_SIGMOID])
@pytest.mark.parametrize("method,order,nbase", [(oracle.EULER, 1, 400), (oracle.RK4, 4, 40),
                                                (oracle.DOPRI5, 5, 40), (oracle.MIDPOINT, 2, 200)])
def test_observed_order(kind, method, order, nbase):
    x0, t0, t1, coef = _family(kind)
    exact = _closed_form(kind, x0, t0, t1, coef)
    errs = []
    for m in (nbase, 2 * nbase):
        dt = (t1 - t0) / m
        x = oracle.pw_integrate_const(kind, x0, method, dt, m, t0=t0, coef=coef)
        errs.append(oracle.linf(x - exact))
    ratio = errs[0] / errs[1]
    if kind == oracle.PW_PAPER_SIGMOID and order % 2 == 1:
        # Eq. 1b is a quadrature of an even integrand over the symmetric
        # interval [-5, 5].  A composite rule's error expands in terms
        # dt^j (f^(j-1)(5) - f^(j-1)(-5)), which vanish for odd j: an odd
        # order p shows as p + 1 (Euler 2, Dopri5 6).
        order += 1
    assert abs(math.log2(ratio) - order) < 0.35, (errs, ratio)


@pytest.mark.parametrize("kind", [oracle.PW_EXP_DECAY, oracle.PW_LOGISTIC, oracle.PW_PAPER_EXP,
                                  oracle.PW_PAPER_SIGMOID])
def test_ab4_observed_order(kind):
    x0, t0, t1, coef = _family(kind)
    exact = _closed_form(kind, x0, t0, t1, coef)
    errs = []
    for m in (100, 200):
        dt = (t1 - t0) / m
        x = oracle.pw_integrate_ab4(kind, x0, dt, m, t0=t0, coef=coef)
        errs.append(oracle.linf(x - exact))
    assert abs(math.log2(errs[0] / errs[1]) - 4) < 0.35, errs


@pytest.mark.parametrize("kind", [oracle.PW_EXP_DECAY, oracle.PW_LOGISTIC])
def test_embedded_error_estimate_is_local_order_5(kind):
    x0 = np.array([0.2, 0.6, 0.8])
    ests = []
    for dt in (0.2, 0.1):
        _, err, _ = oracle.pw_dopri5_attempt(kind, x0, dt, 1e-8, 1e-8)
        ests.append(np.max(np.abs(err)))
    assert abs(math.log2(ests[0] / ests[1]) - 5) < 0.3, ests


def test_embedded_error_matches_difference_of_solutions():
    # err = y5 - y4 where y4 uses bhat; on -x both are polynomials in z=-dt
    x0 = np.array([1.0])
    dt = 0.25
    y5, err, _ = oracle.pw_dopri5_attempt(oracle.PW_EXP_DECAY, x0, dt, 1e-8, 1e-8)
    T = oracle.tableau(oracle.DOPRI5)
    # y4 = R_hat(z) x0 where R_hat(z) = 1 + z bhat^T (I - zA)^-1 1
    z = -dt
    I = np.eye(7)
    Rhat = 1 + z * T["bhat"] @ np.linalg.solve(I - z * T["A"], np.ones(7))
    assert abs(y5[0] - _R_dopri5(z)) < 1e-15
    assert abs(err[0] - (_R_dopri5(z) - Rhat)) < 1e-15


# ------------------------------------------------------------------- algebra
def test_axpy_exact_and_limits():
    xs = [np.arange(10.0) * (j + 1) for j in range(15)]
    coef = np.array([(-1.0) ** j * (j + 1) for j in range(15)])
    y = oracle.axpy(coef, xs)
    expect = np.arange(10.0) * sum((-1) ** j * (j + 1) ** 2 for j in range(15))
    assert np.array_equal(y, expect)
    with pytest.raises(ValueError):
        oracle.axpy(np.ones(16), [np.ones(3)] * 16)


# ------------------------------------------- Table 1: Cash-Karp 5(4), Fehlberg 7(8)
@pytest.mark.parametrize("method,weights,order", [
    (oracle.CK54, "b", 5),
    (oracle.CK54, "bhat", 4),
    (oracle.RKF78, "b", 8),
    (oracle.RKF78, "bhat", 7),
])
def test_order_conditions_ck54_rkf78(method, weights, order):
    # same conditions; the tolerance scales with the coefficient magnitudes
    # (Fehlberg's rows hold entries up to 15.6, summed over 13 stages)
    T = oracle.tableau(method)
    A, b = T["A"], T[weights]
    scale = 1.0 + float(np.abs(A).sum())
    assert np.allclose(A.sum(axis=1), T["c"], atol=1e-16 * scale, rtol=0)
    for p in range(1, order + 1):
        for t in _trees(p):
            assert abs(b @ _phi(t, A) - 1.0 / _gamma(t)) < 1e-15 * scale, (p, t)
    worst = max(abs(b @ _phi(t, A) - 1.0 / _gamma(t)) for t in _trees(order + 1))
    assert worst > 1e-9


def test_rkf78_error_estimate_vanishes_for_time_only_rhs():
    # b - bhat = 41/840 (-1, 0..0, -1, +1, +1) on stages 1, 11, 12, 13 with
    # c = 0, 1, 0, 1: for f = f(t) the four stages pair up and the estimate is 0
    T = oracle.tableau(oracle.RKF78)
    d = T["b"] - T["bhat"]
    assert np.allclose(d[[0, 10, 11, 12]], np.array([-1, -1, 1, 1]) * 41 / 840, rtol=1e-15, atol=0)
    assert np.all(d[1:10] == 0)
    assert (T["c"][0], T["c"][10], T["c"][11], T["c"][12]) == (0.0, 1.0, 0.0, 1.0)
    assert oracle.pair_orders(oracle.RKF78) == (8, 7)
    assert oracle.pair_orders(oracle.CK54) == (5, 4) == oracle.pair_orders(oracle.DOPRI5)


@pytest.mark.parametrize("kind", [oracle.PW_EXP_DECAY, oracle.PW_LOGISTIC, oracle.PW_PAPER_EXP,
                                  oracle.PW_PAPER_SIGMOID])
@pytest.mark.parametrize("method,order,nbase", [(oracle.CK54, 5, 40), (oracle.RKF78, 8, 12)])
def test_observed_order_ck54_rkf78(kind, method, order, nbase):
    x0, t0, t1, coef = _family(kind)
    exact = _closed_form(kind, x0, t0, t1, coef)
    errs = []
    for m in (nbase, 2 * nbase):
        x = oracle.pw_integrate_const(kind, x0, method, (t1 - t0) / m, m, t0=t0, coef=coef)
        errs.append(oracle.linf(x - exact))
    if errs[1] < 1e-13:
        # Eq. 1b: the order-8 rule is at round-off already; check accuracy only
        assert kind == oracle.PW_PAPER_SIGMOID and errs[0] < 1e-9, errs
        return
    ratio = errs[0] / errs[1]
    if kind == oracle.PW_PAPER_SIGMOID and order % 2 == 1:
        order += 1  # even integrand on a symmetric interval (see test_observed_order)
    assert abs(math.log2(ratio) - order) < 0.7, (errs, ratio)


# ------------------------------------------------ Adams-Bashforth 1..8 (Fig. 2c,d)
@pytest.mark.parametrize("steps", range(1, 9))
def test_ab_coefficients_exact_on_polynomials(steps):
    # an s-step Adams-Bashforth rule integrates polynomials of degree < s
    # exactly: sum_j beta_j (-j)^k = 1 / (k + 1) for k = 0 .. s-1
    beta = oracle.ab_coefficients(steps)
    j = np.arange(steps)
    for k in range(steps):
        lhs = float(np.sum(beta * (-j) ** k)) if k else float(np.sum(beta))
        assert abs(lhs - 1.0 / (k + 1)) < 1e-12 * max(1.0, float(np.sum(np.abs(beta * j ** k)))), (k, lhs)
    # and not of degree s (the next moment fails)
    assert abs(float(np.sum(beta * (-j) ** steps)) - 1.0 / (steps + 1)) > 1e-6


def test_ab_coefficients_known_rules():
    assert np.allclose(oracle.ab_coefficients(1), [1.0], rtol=0, atol=0)
    assert np.allclose(oracle.ab_coefficients(2), [1.5, -0.5], rtol=1e-15, atol=0)
    assert np.allclose(oracle.ab_coefficients(4), np.array([55, -59, 37, -9]) / 24, rtol=1e-14, atol=0)


def test_ab4_generic_matches_ab4():
    x0, t0, t1, coef = _family(oracle.PW_PAPER_EXP)
    a = oracle.pw_integrate_ab(4, oracle.PW_PAPER_EXP, x0, 0.05, 200, t0=t0, coef=coef)
    b = oracle.pw_integrate_ab4(oracle.PW_PAPER_EXP, x0, 0.05, 200, t0=t0, coef=coef)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("steps", range(1, 9))
def test_ab_observed_order_exponential_family(steps):
    # Fig. 2c: the exponential family (Eq. 1a) with 1..8 steps shows order s
    x0, t0, t1, coef = _family(oracle.PW_PAPER_EXP)
    exact = _closed_form(oracle.PW_PAPER_EXP, x0, t0, t1, coef)
    errs = []
    for m in (200, 400):
        x = oracle.pw_integrate_ab(steps, oracle.PW_PAPER_EXP, x0, (t1 - t0) / m, m, t0=t0, coef=coef)
        errs.append(oracle.linf(x - exact))
    assert abs(math.log2(errs[0] / errs[1]) - steps) < 0.4, errs


@pytest.mark.parametrize("steps", range(1, 6))
def test_ab_observed_order_decay(steps):
    x0, t0, t1, coef = _family(oracle.PW_EXP_DECAY)
    exact = _closed_form(oracle.PW_EXP_DECAY, x0, t0, t1, coef)
    errs = []
    for m in (100, 200):
        x = oracle.pw_integrate_ab(steps, oracle.PW_EXP_DECAY, x0, (t1 - t0) / m, m, t0=t0)
        errs.append(oracle.linf(x - exact))
    assert abs(math.log2(errs[0] / errs[1]) - steps) < 0.45, errs


# -------------------------------- adaptive: any embedded pair; per-element steps
@pytest.mark.parametrize("method", [oracle.DOPRI5, oracle.CK54, oracle.RKF78])
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_adaptive_each_closed_form_and_independent_steps(method, tol):
    # every element of dx/dt = -x integrated with its own step size: the
    # closed form within C * tol, and elements of different size take
    # different numbers of steps (x0 = 0 stays 0 and takes the fewest)
    x0 = np.linspace(0.0, 1.0, 11)
    r = oracle.pw_integrate_adaptive_each(oracle.PW_EXP_DECAY, x0, 0.0, 10.0, 0.1, tol, tol, method=method)
    exact = x0 * np.exp(-10.0)
    assert np.all(r["status"] == oracle.OK) and np.all(r["t"] == 10.0)
    assert np.max(np.abs(r["x"] - exact) / (1.0 + np.abs(exact))) < 5 * tol
    assert r["x"][0] == 0.0
    assert r["n_acc"][0] == r["n_acc"].min() and r["n_acc"][0] < r["n_acc"][-1]
    assert len(set(r["n_acc"].tolist())) > 3


def test_adaptive_each_higher_order_takes_fewer_steps():
    x0 = np.linspace(0.1, 0.9, 5)  # (x = 1 is a fixed point of the logistic)
    n = {}
    for m in (oracle.DOPRI5, oracle.RKF78):
        r = oracle.pw_integrate_adaptive_each(oracle.PW_LOGISTIC, x0, 0.0, 10.0, 0.1, 1e-10, 1e-10, method=m)
        n[m] = r["n_acc"]
    assert np.all(n[oracle.RKF78] * 2 < n[oracle.DOPRI5])


@pytest.mark.parametrize("method", [oracle.DOPRI5, oracle.CK54])
def test_adaptive_global_norm_any_pair_closed_form(method):
    x0, t0, t1, coef = _family(oracle.PW_PAPER_EXP)
    exact = _closed_form(oracle.PW_PAPER_EXP, x0, t0, t1, coef)
    r = oracle.pw_integrate_adaptive(oracle.PW_PAPER_EXP, x0, t0, t1, 0.1, 1e-9, 1e-9, coef=coef, method=method)
    assert r["status"] == oracle.OK and r["t"] == t1
    assert np.max(np.abs(r["x"] - exact) / (1.0 + np.abs(exact))) < 5e-9


# ------------------------------------------- Adams-Bashforth-Moulton (Table 1)
@pytest.mark.parametrize("steps", range(1, 9))
def test_am_coefficients_exact_on_polynomials(steps):
    # the Adams-Moulton rule with s nodes t_{m+1}, ..., t_{m+2-s} integrates
    # polynomials of degree < s over [t_m, t_{m+1}] exactly:
    # sum_j beta*_j (1 - j)^k = 1 / (k + 1) for k = 0 .. s-1, not for k = s
    beta = oracle.am_coefficients(steps)
    node = 1.0 - np.arange(steps)
    for k in range(steps):
        lhs = float(np.sum(beta * node ** k))
        assert abs(lhs - 1.0 / (k + 1)) < 1e-12 * max(1.0, float(np.sum(np.abs(beta * node ** k)))), (k, lhs)
    assert abs(float(np.sum(beta * node ** steps)) - 1.0 / (steps + 1)) > 1e-6


def test_am_coefficients_known_rules():
    # implicit Euler, the trapezoidal rule and the 4-node Adams-Moulton rule
    assert np.array_equal(oracle.am_coefficients(1), [1.0])
    assert np.allclose(oracle.am_coefficients(2), [0.5, 0.5], rtol=1e-15, atol=0)
    assert np.allclose(oracle.am_coefficients(3), np.array([5, 8, -1]) / 12, rtol=1e-14, atol=0)
    assert np.allclose(oracle.am_coefficients(4), np.array([9, 19, -5, 1]) / 24, rtol=1e-14, atol=0)


def test_abm_one_pece_step_by_hand():
    # s = 2 on dx/dt = -x with the history seeded by one RK4 step: the
    # predictor, the evaluation and the corrector written out
    x0, dt = 0.8, 0.1
    x1 = x0 * (1 - dt + dt ** 2 / 2 - dt ** 3 / 6 + dt ** 4 / 24)  # RK4 on -x
    f0, f1 = -x0, -x1
    xp = x1 + dt * (1.5 * f1 - 0.5 * f0)
    x2 = x1 + dt * (0.5 * (-xp) + 0.5 * f1)
    got = oracle.pw_integrate_abm(2, oracle.PW_EXP_DECAY, np.array([x0]), dt, 2)
    assert abs(got[0] - x2) < 1e-15
    # and differs from plain Adams-Bashforth 2 (the corrector acts)
    ab = oracle.pw_integrate_ab(2, oracle.PW_EXP_DECAY, np.array([x0]), dt, 2)
    assert abs(ab[0] - x2) > 1e-6


@pytest.mark.parametrize("steps", range(1, 9))
def test_abm_observed_order_exponential_family(steps):
    # the exponential family (Eq. 1a) with 1..8 steps shows order s
    x0, t0, t1, coef = _family(oracle.PW_PAPER_EXP)
    exact = _closed_form(oracle.PW_PAPER_EXP, x0, t0, t1, coef)
    errs = []
    for m in (100, 200):
        x = oracle.pw_integrate_abm(steps, oracle.PW_PAPER_EXP, x0, (t1 - t0) / m, m, t0=t0, coef=coef)
        errs.append(oracle.linf(x - exact))
    assert abs(math.log2(errs[0] / errs[1]) - steps) < 0.4, errs


@pytest.mark.parametrize("steps", range(1, 7))
def test_abm_observed_order_decay(steps):
    x0, t0, t1, coef = _family(oracle.PW_EXP_DECAY)
    exact = _closed_form(oracle.PW_EXP_DECAY, x0, t0, t1, coef)
    errs = []
    for m in (200, 400):
        x = oracle.pw_integrate_abm(steps, oracle.PW_EXP_DECAY, x0, (t1 - t0) / m, m, t0=t0)
        errs.append(oracle.linf(x - exact))
    assert abs(math.log2(errs[0] / errs[1]) - steps) < 0.45, errs


@pytest.mark.parametrize("steps", [2, 4, 6])
def test_abm_more_accurate_than_ab(steps):
    # the corrector's error constant is smaller than the predictor's (e.g.
    # 1/24 against 251/720 at s = 4): same order, smaller error
    x0, t0, t1, coef = _family(oracle.PW_LOGISTIC)
    exact = _closed_form(oracle.PW_LOGISTIC, x0, t0, t1, coef)
    m = 200
    e_ab = oracle.linf(oracle.pw_integrate_ab(steps, oracle.PW_LOGISTIC, x0, (t1 - t0) / m, m, t0=t0) - exact)
    e_abm = oracle.linf(oracle.pw_integrate_abm(steps, oracle.PW_LOGISTIC, x0, (t1 - t0) / m, m, t0=t0) - exact)
    assert e_abm < 0.5 * e_ab, (e_abm, e_ab)
