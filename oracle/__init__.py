"""CPU FP64 oracle for explicit time stepping of du/dt = F(t,u) (test infrastructure).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The CUDA library never
loads it, and it never loads the CUDA library; the two share no code.

The arithmetic lives in ``oracle.c`` (plain loops, IEEE FP64, no FMA
contraction); this module only marshals numpy arrays into it.  Function names
follow the paper's vocabulary: a *System* F(t,u) (Listing 2), fixed-step
``integrate_const`` (Listing 3), error-controlled ``integrate_adaptive``
(section "Architecture and nomenclature of Boost Odeint"), and the steppers
of Table 1.

Parity status of each function (pins live in tests/test_oracle_*.py):
  gs_rhs / gs_laplacian        pinned: Fourier eigenvalues, zero sum, uniform
                               fixed points of the reaction (closed forms)
  integrate_const (Euler/RK4/  pinned: exact discrete solutions of du/dt = -x,
  Dopri5)                      polynomial exactness, observed orders
  dopri5 error estimate        pinned: local error order 5 (ratio ~32)
  integrate_adaptive           pinned: closed-form error within C*tol; tol
                               scaling; every attempt (h, E, accept) of runs on
                               dx/dt = -x against the stability polynomials of
                               the tableau and the stated controller reading
                               (paper silent on the formula), each constant of
                               which a perturbed copy must fail to reproduce
  integrate_ab4                pinned: cubic exactness, observed order 4
  CK54 / RKF78 tableaux        pinned: Butcher order conditions (orders 5/4,
                               8/7) and observed orders
  integrate_adaptive (any      pinned: closed-form error within C*tol per
  pair), per element           element; elements with different dynamics take
                               different step counts
  ab_coefficients / AB 1..8    pinned: exactness on polynomials of degree
                               s - 1, the AB2/AB4 coefficients, observed
                               orders 1..8
  am_coefficients / ABM 1..8   pinned: exactness on polynomials of degree
                               s - 1 (not s), the trapezoidal and AM4
                               weights, observed orders 1..8, exact
                               quadrature of polynomial right-hand sides
  axpy                         pinned: exact small-integer sums
  dcpse_stencil / gs_dcpse_*   pinned: exact Laplacian of every polynomial of
                               degree <= 3 (not 4), second-order convergence
                               on periodic trigonometric fields, reflection
                               symmetry; kernel parameters are this build's
                               reading (paper cites the method only)
  conv3d fwd/dgrad/wgrad       pinned: FP64 central differences of a scalar
                               loss, 1x1x1-equivalent reduction to a matmul
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

EULER, RK4, DOPRI5, CK54, RKF78, MIDPOINT = 0, 1, 2, 3, 4, 5
PW_EXP_DECAY, PW_LOGISTIC, PW_PAPER_EXP, PW_PAPER_SIGMOID = 0, 1, 2, 3

OK, ERR_INVALID, ERR_NOMEM, ERR_STEP_UNDERFLOW, ERR_MAX_STEPS, ERR_NONFINITE = 0, 1, 3, 4, 5, 6

_lib = None
_dp = C.POINTER(C.c_double)


class _GS(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("Du", C.c_double), ("Dv", C.c_double), ("F", C.c_double), ("k", C.c_double)]


class _Tableau(C.Structure):
    _fields_ = [("s", C.c_int), ("a", C.c_double * 169), ("b", C.c_double * 13),
                ("bhat", C.c_double * 13), ("c", C.c_double * 13), ("has_bhat", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_get_tableau.argtypes = [C.c_int, C.POINTER(_Tableau)]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_gs_laplacian.argtypes = [C.POINTER(_GS), _dp, _dp]
        L.orc_gs_rhs_full.argtypes = [C.POINTER(_GS), _dp, _dp]
        L.orc_gs_integrate_const.argtypes = [C.POINTER(_GS), C.c_int, _dp, C.c_double, C.c_double, C.c_long]
        L.orc_gs_integrate_replay.argtypes = [C.POINTER(_GS), C.c_int, _dp, C.c_double, _dp, C.c_long]
        L.orc_gs_integrate_adaptive.argtypes = [C.POINTER(_GS), _dp, _dp, C.c_double, _dp, C.c_double,
                                                C.c_double, C.c_long, C.c_long, C.POINTER(C.c_long),
                                                C.POINTER(C.c_long), _dp, C.c_long]
        L.orc_gs_integrate_ab4.argtypes = [C.POINTER(_GS), _dp, C.c_double, C.c_double, C.c_long]
        L.orc_gs_integrate_adaptive_m.argtypes = [C.POINTER(_GS), C.c_int, _dp, _dp, C.c_double, _dp, C.c_double,
                                                  C.c_double, C.c_long, C.c_long, C.POINTER(C.c_long),
                                                  C.POINTER(C.c_long), _dp, C.c_long]
        L.orc_gs_dcpse_integrate_adaptive_m.argtypes = [C.POINTER(_GS), C.c_double, C.c_int, _dp, _dp, C.c_double,
                                                        _dp, C.c_double, C.c_double, C.c_long, C.c_long,
                                                        C.POINTER(C.c_long), C.POINTER(C.c_long), _dp, C.c_long]
        L.orc_gs_dopri5_attempt.argtypes = [C.POINTER(_GS), C.c_double, C.c_double, _dp, _dp, _dp,
                                            C.c_double, C.c_double]
        L.orc_gs_dopri5_attempt.restype = C.c_double
        L.orc_pw_rhs.argtypes = [C.c_int, _dp, C.c_double, C.c_long, _dp, _dp]
        L.orc_pw_integrate_const.argtypes = [C.c_int, _dp, C.c_int, C.c_long, _dp, C.c_double, C.c_double, C.c_long]
        L.orc_pw_integrate_replay.argtypes = [C.c_int, _dp, C.c_int, C.c_long, _dp, C.c_double, _dp, C.c_long]
        L.orc_pw_integrate_adaptive.argtypes = [C.c_int, _dp, C.c_long, _dp, _dp, C.c_double, _dp,
                                                C.c_double, C.c_double, C.c_long, C.c_long,
                                                C.POINTER(C.c_long), C.POINTER(C.c_long), _dp, C.c_long]
        L.orc_pw_integrate_ab4.argtypes = [C.c_int, _dp, C.c_long, _dp, C.c_double, C.c_double, C.c_long]
        L.orc_pw_dopri5_attempt.argtypes = [C.c_int, _dp, C.c_long, C.c_double, C.c_double, _dp, _dp, _dp,
                                            C.c_double, C.c_double]
        L.orc_pw_dopri5_attempt.restype = C.c_double
        L.orc_pw_integrate_ab.argtypes = [C.c_int, C.c_int, _dp, C.c_long, _dp, C.c_double, C.c_double,
                                          C.c_long]
        L.orc_pw_integrate_adaptive_m.argtypes = [C.c_int, C.c_int, _dp, C.c_long, _dp, _dp, C.c_double, _dp,
                                                  C.c_double, C.c_double, C.c_long, C.c_long,
                                                  C.POINTER(C.c_long), C.POINTER(C.c_long), _dp, C.c_long]
        _lp = C.POINTER(C.c_long)
        L.orc_pw_integrate_adaptive_trace.argtypes = [C.c_int, C.c_int, _dp, C.c_long, _dp, _dp, C.c_double, _dp,
                                                      C.c_double, C.c_double, C.c_long, C.c_long, _lp, _lp, _dp,
                                                      _dp, C.POINTER(C.c_int), C.c_long, _lp]
        L.orc_pw_integrate_adaptive_each.argtypes = [C.c_int, C.c_int, _dp, C.c_long, _dp, C.c_double,
                                                     C.c_double, C.c_double, C.c_double, C.c_double, C.c_long,
                                                     C.c_long, _dp, _dp, _lp, _lp, C.POINTER(C.c_int)]
        L.orc_ab_coefficients.argtypes = [C.c_int, _dp]
        L.orc_am_coefficients.argtypes = [C.c_int, _dp]
        L.orc_pw_integrate_abm.argtypes = [C.c_int, C.c_int, _dp, C.c_long, _dp, C.c_double, C.c_double,
                                           C.c_long]
        L.orc_gs_integrate_abm.argtypes = [C.POINTER(_GS), C.c_int, _dp, C.c_double, C.c_double, C.c_long]
        L.orc_pair_orders.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_dcpse_stencil.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int), _dp,
                                         C.c_int]
        L.orc_gs_dcpse_rhs_full.argtypes = [C.POINTER(_GS), C.c_double, _dp, _dp]
        L.orc_gs_dcpse_integrate_const.argtypes = [C.POINTER(_GS), C.c_double, C.c_int, _dp, C.c_double,
                                                   C.c_double, C.c_long]
        L.orc_gs_dcpse_integrate_adaptive.argtypes = [C.POINTER(_GS), C.c_double, _dp, _dp, C.c_double, _dp,
                                                      C.c_double, C.c_double, C.c_long, C.c_long,
                                                      C.POINTER(C.c_long), C.POINTER(C.c_long), _dp, C.c_long]
        L.orc_axpy.argtypes = [C.c_long, C.c_int, _dp, C.POINTER(_dp), _dp]
        L.orc_conv3d_fwd.argtypes = [C.c_int] * 5 + [_dp, _dp, _dp, _dp]
        L.orc_conv3d_dgrad.argtypes = [C.c_int] * 5 + [_dp, _dp, _dp]
        L.orc_conv3d_wgrad.argtypes = [C.c_int] * 5 + [_dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    """Threads for the oracle's loops over cells and elements (default 1).
    Each element's arithmetic is identical for every thread count.  Call it
    only in a process that will not fork afterwards (OpenMP's thread pool does
    not survive a fork)."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def max_threads() -> int:
    """Processors available to this process."""
    return int(lib().orc_max_threads())


# --------------------------------------------------------------------------
# Tableaux (Table 1)
# --------------------------------------------------------------------------
def tableau(method: int):
    T = _Tableau()
    if lib().orc_get_tableau(method, C.byref(T)) != 0:
        raise ValueError(method)
    s = T.s
    A = np.array(T.a[: s * s]).reshape(s, s)
    return {"s": s, "A": A, "b": np.array(T.b[:s]), "bhat": np.array(T.bhat[:s]) if T.has_bhat else None,
            "c": np.array(T.c[:s])}


# --------------------------------------------------------------------------
# Gray-Scott (Eq. 2)
# --------------------------------------------------------------------------
class GSParams:
    """Grid and physics of one Gray-Scott problem (periodic box L^3)."""

    def __init__(self, nx, ny, nz, L=2.5, Du=2e-5, Dv=1e-5, F=0.053, k=0.014, Ly=None, Lz=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.Lx = float(L)
        self.Ly = float(L if Ly is None else Ly)
        self.Lz = float(L if Lz is None else Lz)
        self.Du, self.Dv, self.F, self.k = float(Du), float(Dv), float(F), float(k)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def _c(self):
        return _GS(self.nx, self.ny, self.nz, self.Lx, self.Ly, self.Lz, self.Du, self.Dv, self.F, self.k)


def _pack(p: GSParams, u, v):
    y = np.empty(2 * p.ncell, dtype=np.float64)
    y[: p.ncell] = np.asarray(u, dtype=np.float64).reshape(-1)
    y[p.ncell:] = np.asarray(v, dtype=np.float64).reshape(-1)
    return y


def _unpack(p: GSParams, y):
    shape = (p.nz, p.ny, p.nx)
    return y[: p.ncell].reshape(shape).copy(), y[p.ncell:].reshape(shape).copy()


def gs_laplacian(p: GSParams, w):
    w = _f64(w).reshape(-1)
    out = np.empty_like(w)
    lib().orc_gs_laplacian(C.byref(p._c()), _p(w), _p(out))
    return out.reshape(p.nz, p.ny, p.nx)


def gs_rhs(p: GSParams, u, v):
    """F(t,u) of the Gray-Scott System (Listing 2): returns (du/dt, dv/dt)."""
    y = _pack(p, u, v)
    f = np.empty_like(y)
    lib().orc_gs_rhs_full(C.byref(p._c()), _p(y), _p(f))
    return _unpack(p, f)


def gs_integrate_const(p: GSParams, u, v, method: int, dt: float, nsteps: int, t0: float = 0.0):
    y = _pack(p, u, v)
    st = lib().orc_gs_integrate_const(C.byref(p._c()), method, _p(y), t0, dt, nsteps)
    if st:
        raise RuntimeError(f"oracle status {st}")
    return _unpack(p, y)


def gs_integrate_replay(p: GSParams, u, v, method: int, dts, t0: float = 0.0):
    y = _pack(p, u, v)
    dts = _f64(dts)
    st = lib().orc_gs_integrate_replay(C.byref(p._c()), method, _p(y), t0, _p(dts), len(dts))
    if st:
        raise RuntimeError(f"oracle status {st}")
    return _unpack(p, y)


def gs_integrate_adaptive(p: GSParams, u, v, t0, t_end, dt0, atol, rtol, max_acc=-1, max_rej=500,
                          log_cap=0, method=DOPRI5):
    y = _pack(p, u, v)
    t = C.c_double(t0)
    dt = C.c_double(dt0)
    na, nr = C.c_long(0), C.c_long(0)
    log = np.zeros(max(log_cap, 1))
    st = lib().orc_gs_integrate_adaptive_m(C.byref(p._c()), method, _p(y), C.byref(t), t_end, C.byref(dt), atol,
                                           rtol, max_acc, max_rej, C.byref(na), C.byref(nr),
                                           _p(log) if log_cap else None, log_cap)
    u1, v1 = _unpack(p, y)
    return {"u": u1, "v": v1, "t": t.value, "dt": dt.value, "n_acc": na.value, "n_rej": nr.value,
            "status": st, "dts": log[: min(na.value, log_cap)].copy() if log_cap else None}


def gs_integrate_ab4(p: GSParams, u, v, dt, nsteps, t0=0.0):
    y = _pack(p, u, v)
    lib().orc_gs_integrate_ab4(C.byref(p._c()), _p(y), t0, dt, nsteps)
    return _unpack(p, y)


def gs_dopri5_attempt(p: GSParams, u, v, dt, atol, rtol, t=0.0):
    """One Dopri5 attempt: returns (u5, v5, err_u, err_v, E)."""
    y = _pack(p, u, v)
    yo = np.empty_like(y)
    err = np.empty_like(y)
    E = lib().orc_gs_dopri5_attempt(C.byref(p._c()), t, dt, _p(y), _p(yo), _p(err), atol, rtol)
    u5, v5 = _unpack(p, yo)
    eu, ev = _unpack(p, err)
    return u5, v5, eu, ev, E


# --------------------------------------------------------------------------
# Pointwise ODE families (closed-form benchmarks, Eq. 1a / 1b, and the
# decay / logistic ensembles)
# --------------------------------------------------------------------------
def dcpse_stencil(h=(1.0, 1.0, 1.0), rc_over_h=3.1):
    """DC-PSE Laplacian stencil: (offsets [m, 3] in spacings, weights [m])."""
    cap = 4096
    off = (C.c_int * (3 * cap))()
    w = np.zeros(cap)
    m = lib().orc_dcpse_stencil(h[0], h[1], h[2], rc_over_h, off, _p(w), cap)
    if m < 0:
        raise ValueError("DC-PSE moment system failed")
    return np.array(off[: 3 * m], dtype=np.int64).reshape(m, 3), w[:m].copy()


def gs_dcpse_rhs(p: GSParams, u, v, rc_over_h=3.1):
    y = _pack(p, u, v)
    f = np.empty_like(y)
    if lib().orc_gs_dcpse_rhs_full(C.byref(p._c()), rc_over_h, _p(y), _p(f)) != 0:
        raise ValueError("DC-PSE moment system failed")
    return _unpack(p, f)


def gs_dcpse_integrate_const(p: GSParams, u, v, method: int, dt: float, nsteps: int, t0: float = 0.0,
                             rc_over_h=3.1):
    y = _pack(p, u, v)
    if lib().orc_gs_dcpse_integrate_const(C.byref(p._c()), rc_over_h, method, _p(y), t0, dt, nsteps) != 0:
        raise ValueError("DC-PSE integration failed")
    return _unpack(p, y)


def gs_dcpse_integrate_adaptive(p: GSParams, u, v, t0, t_end, dt0, atol, rtol, max_acc=-1, max_rej=500,
                                rc_over_h=3.1, log_cap=0, method=DOPRI5):
    y = _pack(p, u, v)
    t = C.c_double(t0)
    dt = C.c_double(dt0)
    na, nr = C.c_long(0), C.c_long(0)
    log = np.zeros(max(log_cap, 1))
    st = lib().orc_gs_dcpse_integrate_adaptive_m(C.byref(p._c()), rc_over_h, method, _p(y), C.byref(t), t_end,
                                                 C.byref(dt), atol, rtol, max_acc, max_rej, C.byref(na),
                                                 C.byref(nr), _p(log) if log_cap else None, log_cap)
    u2, v2 = _unpack(p, y)
    return {"u": u2, "v": v2, "t": t.value, "dt": dt.value, "n_acc": na.value, "n_rej": nr.value, "status": st,
            "dts": log[: min(na.value, log_cap)].copy() if log_cap else None}


def pw_rhs(kind, x, t=0.0, coef=None):
    x = _f64(x)
    f = np.empty_like(x)
    c = _f64(coef) if coef is not None else None
    lib().orc_pw_rhs(kind, _p(c), t, x.size, _p(x), _p(f))
    return f


def pw_integrate_const(kind, x, method, dt, nsteps, t0=0.0, coef=None):
    x = _f64(x).copy()
    c = _f64(coef) if coef is not None else None
    lib().orc_pw_integrate_const(kind, _p(c), method, x.size, _p(x), t0, dt, nsteps)
    return x


def pw_integrate_replay(kind, x, method, dts, t0=0.0, coef=None):
    x = _f64(x).copy()
    c = _f64(coef) if coef is not None else None
    dts = _f64(dts)
    lib().orc_pw_integrate_replay(kind, _p(c), method, x.size, _p(x), t0, _p(dts), len(dts))
    return x


def pw_integrate_adaptive(kind, x, t0, t_end, dt0, atol, rtol, max_acc=-1, max_rej=500, coef=None,
                          log_cap=0, method=DOPRI5):
    """One state vector, one step size (global L-infinity norm)."""
    x = _f64(x).copy()
    c = _f64(coef) if coef is not None else None
    t = C.c_double(t0)
    dt = C.c_double(dt0)
    na, nr = C.c_long(0), C.c_long(0)
    log = np.zeros(max(log_cap, 1))
    st = lib().orc_pw_integrate_adaptive_m(method, kind, _p(c), x.size, _p(x), C.byref(t), t_end, C.byref(dt),
                                           atol, rtol, max_acc, max_rej, C.byref(na), C.byref(nr),
                                           _p(log) if log_cap else None, log_cap)
    return {"x": x, "t": t.value, "dt": dt.value, "n_acc": na.value, "n_rej": nr.value, "status": st,
            "dts": log[: min(na.value, log_cap)].copy() if log_cap else None}


def pw_integrate_adaptive_trace(kind, x, t0, t_end, dt0, atol, rtol, max_acc=-1, max_rej=500, coef=None,
                                method=DOPRI5, cap=100000):
    """pw_integrate_adaptive plus the record of every attempt: arrays h, E
    and accepted (bool), one entry per attempt in order."""
    x = _f64(x).copy()
    c = _f64(coef) if coef is not None else None
    t = C.c_double(t0)
    dt = C.c_double(dt0)
    na, nr, natt = C.c_long(0), C.c_long(0), C.c_long(0)
    th = np.zeros(cap)
    tE = np.zeros(cap)
    ta = np.zeros(cap, dtype=np.int32)
    st = lib().orc_pw_integrate_adaptive_trace(method, kind, _p(c), x.size, _p(x), C.byref(t), t_end, C.byref(dt),
                                               atol, rtol, max_acc, max_rej, C.byref(na), C.byref(nr), _p(th),
                                               _p(tE), ta.ctypes.data_as(C.POINTER(C.c_int)), cap, C.byref(natt))
    m = min(natt.value, cap)
    return {"x": x, "t": t.value, "dt": dt.value, "n_acc": na.value, "n_rej": nr.value, "status": st,
            "h": th[:m].copy(), "E": tE[:m].copy(), "accepted": ta[:m].astype(bool)}


def pw_integrate_ab4(kind, x, dt, nsteps, t0=0.0, coef=None):
    x = _f64(x).copy()
    c = _f64(coef) if coef is not None else None
    lib().orc_pw_integrate_ab4(kind, _p(c), x.size, _p(x), t0, dt, nsteps)
    return x


def pw_integrate_adaptive_each(kind, x, t0, t_end, dt0, atol, rtol, method=DOPRI5, max_acc=-1, max_rej=500,
                               coef=None):
    """Every element its own step size and controller."""
    x = _f64(x).copy()
    n = x.size
    c = _f64(coef) if coef is not None else None
    t = np.zeros(n)
    dt = np.zeros(n)
    na = np.zeros(n, dtype=np.int64)
    nr = np.zeros(n, dtype=np.int64)
    stv = np.zeros(n, dtype=np.int32)
    _lp = C.POINTER(C.c_long)
    st = lib().orc_pw_integrate_adaptive_each(method, kind, _p(c), n, _p(x), t0, t_end, dt0, atol, rtol, max_acc,
                                              max_rej, _p(t), _p(dt), na.ctypes.data_as(_lp),
                                              nr.ctypes.data_as(_lp), stv.ctypes.data_as(C.POINTER(C.c_int)))
    if st != OK:
        raise ValueError(st)
    return {"x": x, "t": t, "dt": dt, "n_acc": na, "n_rej": nr, "status": stv}


def ab_coefficients(steps):
    beta = np.zeros(steps)
    if lib().orc_ab_coefficients(steps, _p(beta)) != OK:
        raise ValueError(steps)
    return beta


def pw_integrate_ab(steps, kind, x, dt, nsteps, t0=0.0, coef=None):
    x = _f64(x).copy()
    c = _f64(coef) if coef is not None else None
    if lib().orc_pw_integrate_ab(steps, kind, _p(c), x.size, _p(x), t0, dt, nsteps) != OK:
        raise ValueError(steps)
    return x


def am_coefficients(steps):
    """Adams-Moulton weights beta*_0..beta*_{s-1} (node t_{m+1} first)."""
    beta = np.zeros(steps)
    if lib().orc_am_coefficients(steps, _p(beta)) != OK:
        raise ValueError(steps)
    return beta


def pw_integrate_abm(steps, kind, x, dt, nsteps, t0=0.0, coef=None):
    """Adams-Bashforth-Moulton (PECE) with `steps` steps."""
    x = _f64(x).copy()
    c = _f64(coef) if coef is not None else None
    if lib().orc_pw_integrate_abm(steps, kind, _p(c), x.size, _p(x), t0, dt, nsteps) != OK:
        raise ValueError(steps)
    return x


def gs_integrate_abm(p: GSParams, u, v, steps, dt, nsteps, t0=0.0):
    y = _pack(p, u, v)
    if lib().orc_gs_integrate_abm(C.byref(p._c()), steps, _p(y), t0, dt, nsteps) != OK:
        raise ValueError(steps)
    return _unpack(p, y)


def pair_orders(method):
    p, q = C.c_int(0), C.c_int(0)
    if lib().orc_pair_orders(method, C.byref(p), C.byref(q)) != 0:
        raise ValueError(method)
    return p.value, q.value


def pw_dopri5_attempt(kind, x, dt, atol, rtol, t=0.0, coef=None):
    x = _f64(x)
    c = _f64(coef) if coef is not None else None
    yo = np.empty_like(x)
    err = np.empty_like(x)
    E = lib().orc_pw_dopri5_attempt(kind, _p(c), x.size, t, dt, _p(x), _p(yo), _p(err), atol, rtol)
    return yo, err, E


def axpy(coef, xs):
    """y = sum_j coef[j] * xs[j] (the Algebra's n-ary for_each, n <= 15)."""
    xs = [_f64(x).reshape(-1) for x in xs]
    coef = _f64(coef)
    n = xs[0].size
    y = np.empty(n)
    arr = (_dp * len(xs))(*[_p(x) for x in xs])
    st = lib().orc_axpy(n, len(xs), _p(coef), arr, _p(y))
    if st:
        raise ValueError("nterms must be in 1..15")
    return y


# --------------------------------------------------------------------------
# 3D periodic convolution (surrogate)
# --------------------------------------------------------------------------
def conv3d_fwd(x, w, b=None):
    """x: (D,H,W,Cin), w: (27,Cin,Cout) taps ordered (dz,dy,dx), b: (Cout,)."""
    x = _f64(x)
    w = _f64(w)
    D, H, W, Cin = x.shape
    Cout = w.shape[2]
    y = np.empty((D, H, W, Cout))
    lib().orc_conv3d_fwd(D, H, W, Cin, Cout, _p(x), _p(w), _p(_f64(b)) if b is not None else None, _p(y))
    return y


def conv3d_dgrad(dy, w):
    dy = _f64(dy)
    w = _f64(w)
    D, H, W, Cout = dy.shape
    Cin = w.shape[1]
    dx = np.empty((D, H, W, Cin))
    lib().orc_conv3d_dgrad(D, H, W, Cin, Cout, _p(dy), _p(w), _p(dx))
    return dx


def conv3d_wgrad(x, dy):
    x = _f64(x)
    dy = _f64(dy)
    D, H, W, Cin = x.shape
    Cout = dy.shape[3]
    dw = np.empty((27, Cin, Cout))
    db = np.empty(Cout)
    lib().orc_conv3d_wgrad(D, H, W, Cin, Cout, _p(x), _p(dy), _p(dw), _p(db))
    return dw, db


# --------------------------------------------------------------------------
# Error norms of the accuracy benchmarks (section "Accuracy Benchmarks")
# --------------------------------------------------------------------------
def linf(e):
    return float(np.max(np.abs(np.asarray(e, dtype=np.float64))))


def l2(e):
    e = np.asarray(e, dtype=np.float64).reshape(-1)
    return float(np.sqrt(np.sum(e * e)))


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 over all components, a and b sequences of arrays."""
    if not isinstance(a, (list, tuple)):
        a, b = [a], [b]
    num = sum(float(np.sum((np.asarray(x, np.float64) - np.asarray(y, np.float64)) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(np.asarray(y, np.float64) ** 2)) for y in b)
    return float(np.sqrt(num / den))


# --------------------------------------------------------------------------
# Learned surrogate: 4-layer 3D conv network (2 -> 32 -> 32 -> 32 -> 2,
# 3^3 periodic kernels, ReLU), composed from the convolutions above.  With
# emulate_bf16 the tensors the GPU stores in BF16 (normalised input, weights,
# hidden activations, gradients of layer outputs) are rounded to BF16
# (round-to-nearest-even) at the same points; all arithmetic is FP64.
# --------------------------------------------------------------------------
SURROGATE_LAYERS = [(2, 32), (32, 32), (32, 32), (32, 2)]


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    b = f.view(np.uint32)
    b += ((b >> 16) & np.uint32(1)) + np.uint32(0x7FFF)
    b &= np.uint32(0xFFFF0000)
    return f.astype(np.float64)


def surrogate_unpack(params):
    """[(W[27,cin,cout], b[cout])] from the flat parameter vector."""
    p = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for cin, cout in SURROGATE_LAYERS:
        nw = 27 * cin * cout
        out.append((p[off:off + nw].reshape(27, cin, cout), p[off + nw:off + nw + cout]))
        off += nw + cout
    return out


def surrogate_param_count():
    return sum(27 * a * b + b for a, b in SURROGATE_LAYERS)


def surrogate_forward(params, u, v, mean, sd, scale, emulate_bf16=True):
    """Prediction of the state 16 RK4 steps ahead, u, v shaped (D, H, W)."""
    r = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = surrogate_unpack(params)
    x = r(np.stack([(u - mean[0]) / sd[0], (v - mean[1]) / sd[1]], axis=-1))
    for l, (w, b) in enumerate(layers):
        z = conv3d_fwd(x, r(w), b)
        x = r(np.maximum(z, 0.0)) if l < 3 else z
    return u + scale[0] * x[..., 0], v + scale[1] * x[..., 1]


def surrogate_loss_grad(params, u, v, ut, vt, mean, sd, scale, emulate_bf16=True):
    """Loss = mean over cells and the 2 channels of (y - (target - state)/scale)^2
    and its gradient w.r.t. the flat parameter vector (backpropagation with
    the oracle's dgrad / wgrad)."""
    r = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = surrogate_unpack(params)
    acts = [r(np.stack([(u - mean[0]) / sd[0], (v - mean[1]) / sd[1]], axis=-1))]
    for l, (w, b) in enumerate(layers):
        z = conv3d_fwd(acts[-1], r(w), b)
        acts.append(r(np.maximum(z, 0.0)) if l < 3 else z)
    y = acts[-1]
    tgt = np.stack([(ut - u) / scale[0], (vt - v) / scale[1]], axis=-1)
    n = y.size
    diff = y - tgt
    loss = float(np.sum(diff * diff) / n)
    dy = r(2.0 * diff / n)
    grads = [None] * 4
    for l in range(3, -1, -1):
        w, b = layers[l]
        dw, db = conv3d_wgrad(acts[l], dy)
        grads[l] = (dw, db)
        if l > 0:
            dx = conv3d_dgrad(dy, r(w))
            dy = r(dx * (acts[l] > 0))
    flat = np.concatenate([np.concatenate([g[0].reshape(-1), g[1]]) for g in grads])
    return loss, flat
