"""The Observer of the integrate functions (the user functor called before
each time step; section "Architecture and nomenclature of Boost Odeint"):
when and on what it is called, that a nonzero return stops the integration,
and that an observed run takes the steps of the same call without one (bit
for bit), on the stencil path (fixed steps of every method, error-controlled
Dormand-Prince with and without the stage pairs) and on the DC-PSE path."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from tests._gpu_common import assert_parity, cuda_or_skip, to_np

pytestmark = pytest.mark.gpu


def _gs(torch, dims, prec, seed, **phys):
    import paper_2309_05331_b300 as gs
    u0, v0 = si.gs_initial_state(*dims, seed=seed)
    g = gs.GrayScott(*dims, prec=prec, **phys)
    g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    gs.gs_set_small_grid_path(g.ctx, 0)  # RK4 on the per-stage graph in every run compared here
    return g, u0, v0


def _recorder(log, stop_at=None):
    def fn(t, u, v):
        log.append((t, to_np(u).copy(), to_np(v).copy()))
        return stop_at is not None and len(log) == stop_at
    return fn


METHODS = ["euler", "rk4", "dopri5", "ab4"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("method", METHODS)
def test_observer_fixed_steps(prec, method):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    m = {"euler": gs.GS_EULER, "rk4": gs.GS_RK4, "dopri5": gs.GS_DOPRI5, "ab4": gs.GS_AB4}[method]
    dims, t0, dt, n = (20, 12, 9), 0.25, 0.5, 7
    ref, u0, v0 = _gs(torch, dims, prec, 71)
    states = {}
    for k in (0, 3, n):  # unobserved runs of k steps from the same state
        ref.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
        if k:
            assert ref.step(m, t0, dt, k) == t0 + k * dt
        states[k] = (to_np(ref.u).copy(), to_np(ref.v).copy())
    ref.close()
    g, _, _ = _gs(torch, dims, prec, 71)
    log = []
    g.set_observer(_recorder(log))
    assert g.step(m, t0, dt, n) == t0 + n * dt
    # called before every step and once after the last, at t0 + j dt
    assert [e[0] for e in log] == [t0 + j * dt for j in range(n + 1)]
    for k in (0, 3, n):
        assert np.array_equal(log[k][1], states[k][0]) and np.array_equal(log[k][2], states[k][1])
    assert np.array_equal(to_np(g.u), states[n][0]) and np.array_equal(to_np(g.v), states[n][1])
    # a nonzero return stops before the next step
    g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    log2 = []
    g.set_observer(_recorder(log2, stop_at=4))
    assert g.step(m, t0, dt, n) == t0 + 3 * dt
    assert len(log2) == 4
    assert np.array_equal(to_np(g.u), states[3][0]) and np.array_equal(to_np(g.v), states[3][1])
    # removed: no calls
    g.set_observer(None)
    g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    g.step(m, t0, dt, 2)
    assert len(log2) == 4
    g.close()


@pytest.mark.parametrize("prec,fusion", [(0, -1), (1, 0), (1, 1)])
def test_observer_adaptive(prec, fusion):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (24, 16, 20)
    tol = 1e-8 if prec == 0 else 1e-5
    t_end = 40.0
    ref, u0, v0 = _gs(torch, dims, prec, 72)
    if fusion >= 0:
        gs.gs_set_dopri5_fusion(ref.ctx, fusion)
    gs.gs_set_step_log(ref.ctx, 10000)
    r = ref.integrate_adaptive(tol, tol, 0.0, t_end, 0.5)
    dts, cnt = gs.gs_get_step_log(ref.ctx, 10000)
    final = (to_np(ref.u).copy(), to_np(ref.v).copy())
    ref.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    r3 = ref.integrate_adaptive(tol, tol, 0.0, t_end, 0.5, max_accepted=3)
    after3 = (to_np(ref.u).copy(), to_np(ref.v).copy())
    ref.close()
    assert r["n_acc"] > 5 and cnt == r["n_acc"]

    g, _, _ = _gs(torch, dims, prec, 72)
    if fusion >= 0:
        gs.gs_set_dopri5_fusion(g.ctx, fusion)
    log = []
    g.set_observer(_recorder(log))
    ro = g.integrate_adaptive(tol, tol, 0.0, t_end, 0.5)
    assert (ro["n_acc"], ro["n_rej"], ro["t"], ro["dt"]) == (r["n_acc"], r["n_rej"], r["t"], r["dt"])
    # at the start time and after every accepted step, at the accepted times
    times = [0.0]
    for h in dts:
        times.append(times[-1] + h)
    times[-1] = t_end  # the last step is clipped to end exactly at t_end
    assert [e[0] for e in log] == times
    assert np.array_equal(to_np(g.u), final[0]) and np.array_equal(to_np(g.v), final[1])
    assert np.array_equal(log[-1][1], final[0])
    # stop after the third accepted step: the state of max_accepted = 3
    g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    log2 = []
    g.set_observer(_recorder(log2, stop_at=4))
    rs = g.integrate_adaptive(tol, tol, 0.0, t_end, 0.5)
    assert (rs["n_acc"], rs["n_rej"], rs["t"], rs["dt"]) == (r3["n_acc"], r3["n_rej"], r3["t"], r3["dt"])
    assert np.array_equal(to_np(g.u), after3[0]) and np.array_equal(to_np(g.v), after3[1])
    g.close()


def test_observer_dcpse():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (16, 12, 10)
    phys = dict(Du=2e-4, Dv=1e-4, F=0.053, k=0.014)
    runs = []
    for observed in (False, True):
        g, u0, v0 = _gs(torch, dims, gs.GS_FP64, 73, **phys)
        gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
        log = []
        if observed:
            g.set_observer(_recorder(log))
        t = g.step(gs.GS_RK4, 0.0, 1.0, 3)
        r = g.integrate_adaptive(1e-8, 1e-8, t, 10.0, 1.0)
        runs.append((to_np(g.u).copy(), to_np(g.v).copy(), r, log))
        g.close()
    (u_a, v_a, ra, _), (u_b, v_b, rb, log) = runs
    assert np.array_equal(u_a, u_b) and np.array_equal(v_a, v_b)
    assert (ra["n_acc"], ra["n_rej"], ra["t"]) == (rb["n_acc"], rb["n_rej"], rb["t"])
    # 4 calls of the fixed-step run (t = 0, 1, 2, 3), then the start and every accepted step
    assert [e[0] for e in log[:4]] == [0.0, 1.0, 2.0, 3.0]
    assert len(log) == 4 + 1 + rb["n_acc"] and log[-1][0] == 10.0
    # the observed fixed-step states are the oracle's
    p = oracle.GSParams(*dims, **phys)
    ou, ov = oracle.gs_dcpse_integrate_const(p, u0, v0, oracle.RK4, 1.0, 2)
    assert_parity([log[2][1], log[2][2]], [ou, ov], 1e-12)
