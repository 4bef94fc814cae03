"""Times the FP64-bound paths whose kernels are launched directly (no graph),
so that a profiler sees each launch.

    python -m paper_2309_05331_b300.kernel_timing dcpse --grid 64 --method rk4 --steps 20
    python -m paper_2309_05331_b300.kernel_timing dp5 --n 1048576 --rhs 0
    python -m paper_2309_05331_b300.kernel_timing ab4 --n 16777216 --rhs 1 --steps 1000
    python -m paper_2309_05331_b300.kernel_timing batch --count 512 [--pairs 12 [--lanes 0]]
    python -m paper_2309_05331_b300.kernel_timing each --n 16777216 --rhs 0
    python -m paper_2309_05331_b300.kernel_timing rk4 --grid 256 --steps 50

dcpse: the Gray-Scott run with the DC-PSE Laplacian (Du = 2e-4, Dv = 1e-4,
F = 0.053, k = 0.014, FP64, fixed steps of dt = 1).  dp5: error-controlled
Dormand-Prince on n independent elements through the allocation-free entry
point (whose attempts are launched one by one), atol = rtol = 1e-8, t: 0 -> 10.
ab4: Adams-Bashforth 4, dt = 1e-3.  batch: the ensemble of `count` uneven
Gray-Scott instances (FP32) and the batched integrator's autotuner, whose
timing rounds launch every Dormand-Prince stage of the whole batch directly
(with --pairs TY: the k1 stage and the three stage-pair steps, ring depth 2,
tile height TY for the instances with one cell per lane; --lanes 1, the
default: 2 or 4 cells per lane where an instance's rows allow, tile height 7
for those; --lanes 0: one cell per lane for every instance).
each: Dormand-Prince with every element its own step size (one launch),
atol = rtol = 1e-8, t: 0 -> 10.
rk4: the Gray-Scott grid (Du = 2e-5, Dv = 1e-5, FP32) autotuned (its timing
launches every stage and stage-pair kernel directly, the RK4 pairs among
them), then `steps` fixed RK4 steps of dt = 0.1; reports the pair shapes
chosen and the steps' time.
Seeded synthetic inputs; prints one JSON line with the wall time (after a
warm-up run) of the call.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import time


def main(argv=None):
    import torch

    import synthetic_inputs as si

    from . import GS_DOPRI5, GS_FP64, GS_LAP_DCPSE, GS_RK4, GrayScott, gs_set_laplacian, lib, ode_integrate_ab4

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("what", choices=["dcpse", "dp5", "ab4", "batch", "each", "rk4"])
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--method", choices=["rk4", "dopri5"], default="rk4")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--rhs", type=int, default=0, help="0: dx/dt = -x, 1: x (1 - x)")
    ap.add_argument("--pairs", type=int, default=0, help="batch: stage pairs of this tile height (0: single stages)")
    ap.add_argument("--lanes", type=int, default=1, help="batch pairs: 1 = 2 or 4 cells per lane where rows allow, 0 = one")
    a = ap.parse_args(argv)
    res = {"what": a.what}
    if a.what == "dcpse":
        n = a.grid
        u0, v0 = si.gs_initial_state(n, n, n, seed=2)
        g = GrayScott(n, n, n, Du=2e-4, Dv=1e-4, F=0.053, k=0.014, prec=GS_FP64)
        gs_set_laplacian(g.ctx, GS_LAP_DCPSE, 3.1)
        m = GS_RK4 if a.method == "rk4" else GS_DOPRI5

        def run():
            g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.step(m, 0.0, 1.0, a.steps)
            return (time.perf_counter() - t0) * 1e3
        run()
        res.update(grid=n, method=a.method, steps=a.steps, ms=run())
        g.close()
    elif a.what == "dp5":
        x0 = torch.from_numpy(si.ode_initial_values(a.n, seed=1)).cuda()

        def run():
            x = x0.clone()
            tt, dd = C.c_double(0.0), C.c_double(1e-3)
            na, nr = C.c_long(0), C.c_long(0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = lib().ode_integrate_adaptive_noalloc(a.rhs, a.n, x.data_ptr(), C.byref(tt), 10.0, C.byref(dd),
                                                      1e-8, 1e-8, -1, C.byref(na), C.byref(nr), None)
            ms = (time.perf_counter() - t0) * 1e3
            assert st == 0, st
            return ms, na.value, nr.value
        run()
        ms, na, nr = run()
        res.update(n=a.n, rhs=a.rhs, ms=ms, accepted=na, rejected=nr)
    elif a.what == "batch":
        from . import GS_FP32, GrayScottBatch
        insts = si.batch_instances(a.count, seed=3)
        b = GrayScottBatch(insts, L=2.5, Du=2e-5, Dv=1e-5, prec=GS_FP32)
        for i, d in enumerate(insts):
            u, v = si.gs_initial_state(d["nx"], d["ny"], d["nz"], seed=1000 + i)
            b.set_instance(i, torch.from_numpy(u), torch.from_numpy(v))
        if a.pairs:
            b.set_pairs(True, a.pairs, 2)
            b.set_pair_lanes(a.lanes)
        t0 = time.perf_counter()
        ty, zc, ms = b.autotune()
        if a.pairs:
            ty = a.pairs
        res.update(pairs=bool(a.pairs), lanes=b.pair_lanes()[2] if a.pairs else None, count=a.count, cells=int(sum(d["nx"] * d["ny"] * d["nz"] for d in insts)), tile=[ty, zc],
                   round_ms=ms, ms=(time.perf_counter() - t0) * 1e3)
        b.close()
    elif a.what == "rk4":
        from . import GS_FP32, GS_RK4, GrayScott, gs_autotune, gs_get_pair_configs, gs_get_rk4_fusion
        n = a.grid
        u0, v0 = si.gs_initial_state(n, n, n, seed=2)
        g = GrayScott(n, n, n, prec=GS_FP32)
        g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
        gs_autotune(g.ctx)
        g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
        g.step(GS_RK4, 0.0, 0.1, 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(GS_RK4, 0.2, 0.1, a.steps)
        torch.cuda.synchronize()
        res.update(grid=n, steps=a.steps, ms=(time.perf_counter() - t0) * 1e3, rk4_pairs=gs_get_rk4_fusion(g.ctx),
                   pair_configs=gs_get_pair_configs(g.ctx))
        g.close()
    elif a.what == "each":
        from . import ODE_TAB_DOPRI5, ode_integrate_adaptive_each
        x0 = torch.from_numpy(si.ode_initial_values(a.n, seed=1)).cuda()

        def run():
            x = x0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = ode_integrate_adaptive_each(a.rhs, ODE_TAB_DOPRI5, x, 0.0, 10.0, 1e-3, 1e-8, 1e-8)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) * 1e3, int(r["n_acc"].sum()), int(r["n_rej"].sum())
        run()
        ms, na, nr = run()
        res.update(n=a.n, rhs=a.rhs, ms=ms, accepted=na, rejected=nr)
    else:
        x0 = torch.from_numpy(si.ode_initial_values(a.n, seed=1)).cuda()

        def run():
            x = x0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ode_integrate_ab4(a.rhs, x, 0.0, 1e-3, a.steps)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) * 1e3
        run()
        res.update(n=a.n, rhs=a.rhs, steps=a.steps, ms=run())
    print(json.dumps(res))


if __name__ == "__main__":
    main()
