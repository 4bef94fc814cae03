"""GPU parity of the Gray-Scott path (Eq. 2 + Table 1 steppers) against the
CPU FP64 oracle, element by element on the same seeded inputs.

Tolerances (relative L2 over both components): FP64 path <= 1e-12, FP32 path
<= 1e-5 (against the FP64 oracle started from the same FP32-rounded state).
"""
import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from tests._gpu_common import assert_parity, cuda_or_skip, periodic_box, to_np

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def _gs(torch, dims, prec, u0, v0, **phys):
    import paper_2309_05331_b300 as gs
    nx, ny, nz = dims
    g = gs.GrayScott(nx, ny, nz, prec=prec, **phys)
    g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    return g


def _round32(a):
    return a.astype(np.float32).astype(np.float64)


DIMS = [(8, 8, 8), (9, 6, 5), (33, 17, 40), (64, 31, 30), (1, 1, 1), (2, 3, 1), (61, 14, 3), (32, 32, 32)]


@pytest.mark.parametrize("dims", DIMS)
def test_rhs_fp64(dims):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    u0, v0 = si.gs_initial_state(*dims, seed=11)
    phys = dict(L=2.5, Ly=1.9, Lz=3.3, Du=2e-3, Dv=1e-3)
    g = _gs(torch, dims, gs.GS_FP64, u0, v0, **phys)
    fu, fv = g.rhs()
    torch.cuda.synchronize()
    eu, ev = oracle.gs_rhs(oracle.GSParams(*dims, **phys), u0, v0)
    assert_parity([to_np(fu), to_np(fv)], [eu, ev], 1e-14)
    g.close()


@pytest.mark.parametrize("dims", [(8, 8, 8), (33, 17, 40), (61, 14, 3)])
def test_rhs_fp32(dims):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    u0, v0 = si.gs_initial_state(*dims, seed=12)
    u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, dims, gs.GS_FP32, u0, v0)
    fu, fv = g.rhs()
    torch.cuda.synchronize()
    eu, ev = oracle.gs_rhs(oracle.GSParams(*dims), u0, v0)
    assert_parity([to_np(fu), to_np(fv)], [eu, ev], 1e-6)
    g.close()


def test_rk4_32cubed_fp64_100_steps():
    """Gray-Scott 32^3, dt = 0.1, 100 RK4 steps, FP64 (the small fixed-step workload)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    n = 32
    u0, v0 = si.gs_initial_state(n, n, n, seed=0)
    g = _gs(torch, (n, n, n), gs.GS_FP64, u0, v0)
    t = g.step(gs.GS_RK4, 0.0, 0.1, 100)
    assert t == pytest.approx(10.0, abs=1e-12)
    ou, ov = oracle.gs_integrate_const(oracle.GSParams(n, n, n), u0, v0, oracle.RK4, 0.1, 100)
    assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], FP64_TOL)
    g.close()


def test_rk4_32cubed_fp32():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    n = 32
    u0, v0 = si.gs_initial_state(n, n, n, seed=0)
    u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, (n, n, n), gs.GS_FP32, u0, v0)
    g.step(gs.GS_RK4, 0.0, 0.1, 100)
    ou, ov = oracle.gs_integrate_const(oracle.GSParams(n, n, n), u0, v0, oracle.RK4, 0.1, 100)
    err = assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], FP32_TOL)
    g.close()


@pytest.mark.parametrize("dims", [(37, 10, 7), (36, 10, 7)])  # generic / vectorised kernel
@pytest.mark.parametrize("method", ["euler", "rk4", "dopri5", "ab4"])
@pytest.mark.parametrize("nsteps", [1, 2, 3, 4, 7])
def test_fixed_step_methods_fp64(dims, method, nsteps):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    phys = dict(Du=3e-3, Dv=1.5e-3)
    u0, v0 = si.gs_initial_state(*dims, seed=21)
    g = _gs(torch, dims, gs.GS_FP64, u0, v0, **phys)
    dt = 0.2
    m = {"euler": gs.GS_EULER, "rk4": gs.GS_RK4, "dopri5": gs.GS_DOPRI5, "ab4": gs.GS_AB4}[method]
    g.step(m, 0.0, dt, nsteps)
    p = oracle.GSParams(*dims, **phys)
    if method == "ab4":
        ou, ov = oracle.gs_integrate_ab4(p, u0, v0, dt, nsteps)
    else:
        om = {"euler": oracle.EULER, "rk4": oracle.RK4, "dopri5": oracle.DOPRI5}[method]
        ou, ov = oracle.gs_integrate_const(p, u0, v0, om, dt, nsteps)
    assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], FP64_TOL)
    g.close()


# (dims, L): the domain grows with the grid so the explicit step stays stable
@pytest.mark.parametrize("dims,L", [((45, 29, 19), 2.5), ((44, 29, 19), 2.5), ((264, 9, 5), 2.5 * 264 / 45)])
@pytest.mark.parametrize("tile", [(2, 1), (4, 3), (6, 32), (8, 5), (14, 64), (7, 0), (11, 0)])
@pytest.mark.parametrize("variant", [0, 4])
def test_tile_shape_does_not_change_results(dims, L, tile, variant):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    u0, v0 = si.gs_initial_state(*dims, seed=31)
    res = []
    if variant == 4 and dims[0] % 2:
        pytest.skip("the staged form needs whole 16-byte rows")
    for i, (ty, zc) in enumerate([(6, 32), tile]):
        g = _gs(torch, dims, gs.GS_FP64, u0, v0, L=L, Du=2e-3, Dv=1e-3)
        if variant:
            gs.gs_set_kernel_variant(g.ctx, variant)
            gs.gs_set_stage_depth(g.ctx, 1 + (ty + zc + i) % 3)
        gs.gs_set_tile(g.ctx, ty, zc)
        g.step(gs.GS_DOPRI5, 0.0, 0.3, 3)
        res.append((to_np(g.u), to_np(g.v)))
        g.close()
    assert np.all(np.isfinite(res[0][0]))
    for r in res[1:]:
        assert np.array_equal(res[0][0], r[0]) and np.array_equal(res[0][1], r[1])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(64, 20, 12), (132, 7, 9), (4, 4, 4), (260, 3, 2), (70, 5, 6)])
def test_kernel_variants_match_oracle(prec, dims):
    """The generic (one cell per thread), vectorised (16-byte rows; FP32 also
    8-byte rows) and staged (16-byte rows, inputs copied 1..3 planes ahead)
    stencil kernels on the same grid, each against the oracle, Dopri5 and RK4
    steps."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    # x spacing at least 2.5/45 keeps dt * lambda_max well inside the
    # stability region of both steppers at dt = 0.25
    phys = dict(Du=3e-3, Dv=1.5e-3, L=max(2.5, dims[0] * 2.5 / 45))
    u0, v0 = si.gs_initial_state(*dims, seed=41)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    p = oracle.GSParams(*dims, **phys)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    for method, om in ((gs.GS_DOPRI5, oracle.DOPRI5), (gs.GS_RK4, oracle.RK4)):
        ou, ov = oracle.gs_integrate_const(p, u0, v0, om, 0.25, 3)
        runs = [(1, 0), (2, 0)] + ([(3, 0)] if prec == 1 else []) + [(4, d) for d in (1, 2, 3)]
        for variant, depth in runs:
            vx = {1: 1, 2: 2 if prec == 0 else 4, 3: 2, 4: 2 if prec == 0 else 4}[variant]
            if dims[0] % vx:
                continue
            g = _gs(torch, dims, prec, u0, v0, **phys)
            gs.gs_set_kernel_variant(g.ctx, variant)
            if depth:
                gs.gs_set_stage_depth(g.ctx, depth)
                assert gs.gs_get_kernel_variant(g.ctx) == 4
                assert gs.gs_get_stage_depths(g.ctx) == [depth] * 7
            g.step(method, 0.0, 0.25, 3)
            got = [to_np(g.u), to_np(g.v)]
            g.close()
            assert_parity(got, [ou, ov], tol, (variant, depth, method))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(64, 20, 12), (132, 7, 9), (4, 4, 4), (260, 3, 2)])
def test_split_stages_match_unsplit_and_oracle(prec, dims):
    """Fixed Dopri5 steps with stages 6/7 split and unsplit: both against the
    oracle, and against each other (FP64: 1e-13; the split sums y5 and the
    error terms in another order)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    phys = dict(Du=3e-3, Dv=1.5e-3, L=max(2.5, dims[0] * 2.5 / 45))
    u0, v0 = si.gs_initial_state(*dims, seed=43)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    if dims[0] % (2 if prec == 0 else 4):
        pytest.skip("the split exists in the staged form only")
    ou, ov = oracle.gs_integrate_const(oracle.GSParams(*dims, **phys), u0, v0, oracle.DOPRI5, 0.25, 3)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    res = []
    for split in (1, 0):
        g = _gs(torch, dims, prec, u0, v0, **phys)
        gs.gs_set_dopri5_fusion(g.ctx, 0)
        gs.gs_set_dopri5_split(g.ctx, split)
        g.step(gs.GS_DOPRI5, 0.0, 0.25, 3)
        res.append((to_np(g.u), to_np(g.v)))
        assert_parity(list(res[-1]), [ou, ov], tol, split)
        g.close()
    if prec == 0:
        assert_parity(list(res[0]), list(res[1]), 1e-13)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nsteps,ctas", [(7, 0), (8, 1), (5, 3), (20, 37), (6, 600), (4, 5000)])
def test_rk4_small_grid_path_matches_graph_path(prec, nsteps, ctas):
    """Fixed-step RK4 in one cooperative launch (grid barrier between stages)
    against the four-kernel graph path and the oracle; odd and even step
    counts (copy-back), CTA counts that do and do not divide the cells, and
    CTA counts far above the cells' need, up to the resident limit the launch
    caps 5000 to."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (20, 12, 9)
    phys = dict(Du=2e-3, Dv=1e-3)
    u0, v0 = si.gs_initial_state(*dims, seed=51)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    res = []
    for mode in (1, 0):
        g = _gs(torch, dims, prec, u0, v0, **phys)
        gs.gs_set_small_grid_path(g.ctx, mode, ctas)
        assert gs.gs_get_small_grid_path(g.ctx) == mode
        t = g.step(gs.GS_RK4, 0.0, 0.2, nsteps)
        assert abs(t - 0.2 * nsteps) < 1e-12
        res.append((to_np(g.u), to_np(g.v)))
        g.close()
    ou, ov = oracle.gs_integrate_const(oracle.GSParams(*dims, **phys), u0, v0, oracle.RK4, 0.2, nsteps)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    for r in res:
        assert_parity(list(r), [ou, ov], tol)
    if prec == 0:
        assert_parity(list(res[0]), list(res[1]), 1e-14)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(64, 20, 12), (132, 7, 9), (4, 4, 4), (260, 3, 2), (8, 1, 1), (136, 13, 5)])
@pytest.mark.parametrize("ty,depth", [(7, 2), (1, 1), (3, 3), (5, 1)])
def test_pairs_match_single_stages_and_oracle(prec, dims, ty, depth):
    """Fixed Dopri5 steps with the stages in pairs (2+3, 4+5, 6+7 in one
    launch each, the first stage recomputed on a one-cell ring) against the
    oracle and against the single-stage kernels; ragged x tiles (132, 136,
    260), tile heights that do and do not divide ny, single-plane z, every
    ring depth.  FP64: pairs and single stages agree to 1e-13 (Y_{i+1} is
    summed in another order)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    phys = dict(Du=3e-3, Dv=1.5e-3, L=max(2.5, dims[0] * 2.5 / 45))
    u0, v0 = si.gs_initial_state(*dims, seed=47)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    ou, ov = oracle.gs_integrate_const(oracle.GSParams(*dims, **phys), u0, v0, oracle.DOPRI5, 0.25, 3)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    res = []
    for fusion in (1, 0):
        g = _gs(torch, dims, prec, u0, v0, **phys)
        gs.gs_set_dopri5_fusion(g.ctx, fusion)
        gs.gs_set_pair_config(g.ctx, -1, ty, depth)
        assert gs.gs_get_dopri5_fusion(g.ctx) == fusion
        assert gs.gs_get_pair_configs(g.ctx) == [(ty, depth)] * 5
        t = g.step(gs.GS_DOPRI5, 0.0, 0.25, 3)
        assert abs(t - 0.75) < 1e-15
        res.append((to_np(g.u), to_np(g.v)))
        assert_parity(list(res[-1]), [ou, ov], tol, fusion)
        g.close()
    if prec == 0:
        assert_parity(list(res[0]), list(res[1]), 1e-13)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(64, 20, 12), (132, 7, 9), (4, 4, 4), (260, 3, 2), (8, 1, 1), (136, 13, 5)])
@pytest.mark.parametrize("ty,depth,nsteps", [(7, 2, 3), (1, 1, 2), (3, 3, 5)])
def test_rk4_pairs_match_single_stages_and_oracle(prec, dims, ty, depth, nsteps):
    """Fixed-step RK4 as two pair launches (k1 and k2 from u; k3, k4 and the
    update without storing k3, k4) against the oracle and the four
    single-stage kernels; odd and even step counts (the state ends in either
    buffer), ragged tiles, single-plane z, every ring depth.  FP64: pairs and
    single stages agree to 1e-13 (the update is summed in another order)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    phys = dict(Du=3e-3, Dv=1.5e-3, L=max(2.5, dims[0] * 2.5 / 45))
    u0, v0 = si.gs_initial_state(*dims, seed=53)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    ou, ov = oracle.gs_integrate_const(oracle.GSParams(*dims, **phys), u0, v0, oracle.RK4, 0.2, nsteps)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    res = []
    for fusion in (1, 0):
        g = _gs(torch, dims, prec, u0, v0, **phys)
        gs.gs_set_small_grid_path(g.ctx, 0)
        gs.gs_set_dopri5_fusion(g.ctx, fusion)
        gs.gs_set_pair_config(g.ctx, -1, ty, depth)
        assert gs.gs_get_rk4_fusion(g.ctx) == fusion
        t = g.step(gs.GS_RK4, 0.0, 0.2, nsteps)
        assert abs(t - 0.2 * nsteps) < 1e-12
        res.append((to_np(g.u), to_np(g.v)))
        assert_parity(list(res[-1]), [ou, ov], tol, fusion)
        g.close()
    if prec == 0:
        assert_parity(list(res[0]), list(res[1]), 1e-13)


def test_pairs_per_pair_configs_and_timing():
    """Different launch shapes per pair give the same result; gs_time_pairs
    times k1 and the three pair kernels without touching the state."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (68, 23, 11)
    u0, v0 = si.gs_initial_state(*dims, seed=5)
    res = []
    for cfgs in ([(7, 1), (2, 3), (4, 2), (5, 1), (2, 2)], [(3, 2), (6, 1), (1, 3), (7, 3), (4, 1)],
                 [(11, 3), (7, 2), (9, 1), (10, 1), (8, 2)]):
        g = _gs(torch, dims, gs.GS_FP64, u0, v0, Du=2e-3, Dv=1e-3)
        gs.gs_set_dopri5_fusion(g.ctx, 1)
        for pi, (ty, d) in enumerate(cfgs):
            gs.gs_set_pair_config(g.ctx, pi, ty, d)
        assert gs.gs_get_pair_configs(g.ctx) == cfgs
        used = gs.gs_get_pair_depths_in_use(g.ctx)
        assert all(1 <= u <= d for u, (_, d) in zip(used, cfgs))
        ms = gs.gs_time_pairs(g.ctx, reps=2)
        assert len(ms) == 4 and all(m > 0 for m in ms)
        assert np.array_equal(to_np(g.u), u0) and np.array_equal(to_np(g.v), v0)
        g.step(gs.GS_DOPRI5, 0.0, 0.2, 2)
        res.append((to_np(g.u), to_np(g.v)))
        g.close()
    for r in res[1:]:
        assert np.array_equal(res[0][0], r[0]) and np.array_equal(res[0][1], r[1])


def test_pairs_more_columns_than_ctas_bit_identical():
    """More tile columns than resident CTAs (256 x 160 x 8 FP64 at tile height
    2: 4 x 80 columns): the pair kernels then take linear shares of the
    (column, z) space, several partial columns per CTA, instead of the
    column-split schedule; FP64 results are bit-identical to a run whose
    columns fit the GPU (heights 7 and 11), for Dormand-Prince and RK4."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (256, 160, 8)
    u0, v0 = si.gs_initial_state(*dims, seed=71)
    res = []
    for cfg in ([(2, 1)] * 5, [(11, 2), (7, 1), (11, 1), (11, 2), (11, 1)]):
        g = _gs(torch, dims, gs.GS_FP64, u0, v0, Du=2e-5, Dv=1e-5)
        gs.gs_set_small_grid_path(g.ctx, 0)
        gs.gs_set_dopri5_fusion(g.ctx, 1)
        for pi, (ty, d) in enumerate(cfg):
            gs.gs_set_pair_config(g.ctx, pi, ty, d)
        g.step(gs.GS_DOPRI5, 0.0, 0.2, 2)
        g.step(gs.GS_RK4, 0.4, 0.2, 2)
        res.append((to_np(g.u), to_np(g.v)))
        g.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(64, 20, 12), (132, 23, 9), (136, 8, 5), (8, 1, 1)])
@pytest.mark.parametrize("ty,depth", [(11, 3), (8, 1), (10, 2)])
def test_tall_pairs_match_oracle(prec, dims, ty, depth):
    """Tile heights 8..11 (CTAs of 16 warps) for the Dormand-Prince pairs 2+3
    and 6+7 and both RK4 pairs, stages 4+5 at 7 rows: fixed Dopri5 and RK4
    steps against the oracle; tiles that do and do not divide ny, a tile
    taller than the grid."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    phys = dict(Du=3e-3, Dv=1.5e-3, L=max(2.5, dims[0] * 2.5 / 45))
    u0, v0 = si.gs_initial_state(*dims, seed=61)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    for method, om, dt, n in ((gs.GS_DOPRI5, oracle.DOPRI5, 0.25, 3), (gs.GS_RK4, oracle.RK4, 0.2, 3)):
        ou, ov = oracle.gs_integrate_const(oracle.GSParams(*dims, **phys), u0, v0, om, dt, n)
        g = _gs(torch, dims, prec, u0, v0, **phys)
        gs.gs_set_small_grid_path(g.ctx, 0)
        gs.gs_set_dopri5_fusion(g.ctx, 1)
        for pi in (0, 2, 3, 4):
            gs.gs_set_pair_config(g.ctx, pi, ty, depth)
        gs.gs_set_pair_config(g.ctx, 1, 7, 1)
        assert [c[0] for c in gs.gs_get_pair_configs(g.ctx)] == [ty, 7, ty, ty, ty]
        g.step(method, 0.0, dt, n)
        assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], tol, method)
        g.close()


def test_pairs_rejected_without_staged_form():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    g = _gs(torch, (9, 4, 4), gs.GS_FP32, *si.gs_initial_state(9, 4, 4))
    assert gs.gs_get_dopri5_fusion(g.ctx) == 0
    with pytest.raises(RuntimeError):
        gs.gs_set_dopri5_fusion(g.ctx, 1)
    with pytest.raises(RuntimeError):
        gs.gs_time_pairs(g.ctx)
    g.close()
    g = _gs(torch, (8, 4, 4), gs.GS_FP32, *si.gs_initial_state(8, 4, 4))
    # tile heights: 1..11, but 1..7 for stages 6+7 (pair 2), so -1 (all) takes 1..7
    for bad in [(0, 0, 1), (0, 12, 1), (1, 8, 1), (-1, 8, 1), (0, 3, 0), (0, 3, 4), (5, 3, 1), (-2, 3, 1)]:
        with pytest.raises(RuntimeError):
            gs.gs_set_pair_config(g.ctx, *bad)
    with pytest.raises(RuntimeError):
        gs.gs_set_dopri5_fusion(g.ctx, 2)
    g.close()


def test_split_rejected_without_staged_form():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    g = _gs(torch, (9, 4, 4), gs.GS_FP32, *si.gs_initial_state(9, 4, 4))
    assert gs.gs_get_dopri5_split(g.ctx) == 0
    with pytest.raises(gs.GSError):
        gs.gs_set_dopri5_split(g.ctx, 1)
    gs.gs_set_dopri5_split(g.ctx, 0)
    for bad in (-2, 2):
        with pytest.raises(gs.GSError):
            gs.gs_set_dopri5_split(g.ctx, bad)
    g.close()


def test_vectorised_variant_rejects_unaligned_rows():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    # nx = 10 (FP32): 10 = 5 x 2 cells, so the 8-byte rows apply and variant 2
    # falls back to them; nx = 9 admits no vectorised form
    g = _gs(torch, (10, 4, 4), gs.GS_FP32, *si.gs_initial_state(10, 4, 4))
    gs.gs_set_kernel_variant(g.ctx, 2)
    gs.gs_set_kernel_variant(g.ctx, 3)
    gs.gs_set_kernel_variant(g.ctx, 1)
    g.close()
    g = _gs(torch, (9, 4, 4), gs.GS_FP32, *si.gs_initial_state(9, 4, 4))
    for variant in (2, 3, 4):
        with pytest.raises(gs.GSError):
            gs.gs_set_kernel_variant(g.ctx, variant)
    g.close()
    g = _gs(torch, (10, 4, 4), gs.GS_FP64, *si.gs_initial_state(10, 4, 4))
    with pytest.raises(gs.GSError):
        gs.gs_set_kernel_variant(g.ctx, 3)  # 8-byte rows exist for FP32 only
    for depth in (0, 4):  # the staged ring holds 1..3 planes
        with pytest.raises(gs.GSError):
            gs.gs_set_stage_depth(g.ctx, depth)
    with pytest.raises(gs.GSError):
        gs.gs_set_kernel_variant(g.ctx, 5)
    g.close()


@pytest.mark.parametrize("fusion,split", [(1, 1), (0, 1), (0, 0)])
def test_adaptive_fp64_matches_oracle_run(fusion, split):
    """Error-controlled Dopri5 on 16^3 FP64: same accepted/rejected counts and
    step sizes as the oracle's own adaptive run, final state within 1e-12;
    with the stages in pairs (stages 6+7 reduce the error norm in one
    launch), and single stages with stages 6/7 split (stage 6 forms y5 and
    the error terms of k1..k6) and unsplit."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (16, 16, 16)
    phys = dict(Du=2e-3, Dv=1e-3)
    u0, v0 = si.gs_initial_state(*dims, seed=2)
    g = _gs(torch, dims, gs.GS_FP64, u0, v0, **phys)
    gs.gs_set_dopri5_fusion(g.ctx, fusion)
    gs.gs_set_dopri5_split(g.ctx, split)
    assert gs.gs_get_dopri5_fusion(g.ctx) == fusion
    assert gs.gs_get_dopri5_split(g.ctx) == split
    gs.gs_set_step_log(g.ctx, 10000)
    r = g.integrate_adaptive(1e-8, 1e-8, 0.0, 20.0, 0.1)
    dts, cnt = gs.gs_get_step_log(g.ctx, 10000)
    ref = oracle.gs_integrate_adaptive(oracle.GSParams(*dims, **phys), u0, v0, 0.0, 20.0, 0.1, 1e-8, 1e-8,
                                       log_cap=10000)
    assert ref["status"] == 0 and r["status"] == 0
    assert r["t"] == 20.0 and ref["t"] == 20.0
    assert (r["n_acc"], r["n_rej"]) == (ref["n_acc"], ref["n_rej"])
    # E is a cancelling sum: FMA vs non-FMA rounding moves it by ~1e-9 relative
    assert np.allclose(dts, ref["dts"], rtol=1e-7, atol=0), np.max(np.abs(dts / ref["dts"] - 1))
    assert_parity([to_np(g.u), to_np(g.v)], [ref["u"], ref["v"]], FP64_TOL)
    g.close()


def test_adaptive_fp32_against_fp64_oracle():
    """FP32 stage arithmetic with FP64 control vs the FP64 oracle (32^3, tol 1e-6)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    n = 32
    u0, v0 = si.gs_initial_state(n, n, n, seed=2)
    u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, (n, n, n), gs.GS_FP32, u0, v0)
    r = g.integrate_adaptive(1e-6, 1e-6, 0.0, 50.0, 0.1)
    ref = oracle.gs_integrate_adaptive(oracle.GSParams(n, n, n), u0, v0, 0.0, 50.0, 0.1, 1e-6, 1e-6)
    assert r["status"] == 0 and r["t"] == 50.0
    assert abs(r["n_acc"] - ref["n_acc"]) <= max(1, 0.01 * ref["n_acc"])
    err = assert_parity([to_np(g.u), to_np(g.v)], [ref["u"], ref["v"]], FP32_TOL)
    g.close()


def test_adaptive_max_accepted_and_time_accounting():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (20, 12, 9)
    u0, v0 = si.gs_initial_state(*dims, seed=4)
    g = _gs(torch, dims, gs.GS_FP32, u0, v0)
    gs.gs_set_step_log(g.ctx, 100)
    r = g.integrate_adaptive(1e-6, 1e-6, 1.5, math.inf, 0.1, max_accepted=7)
    dts, cnt = gs.gs_get_step_log(g.ctx, 100)
    assert r["n_acc"] == 7 and cnt == 7
    assert r["t"] == pytest.approx(1.5 + float(np.sum(dts)), rel=1e-15)
    g.close()


def test_nonfinite_state_is_reported():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (12, 12, 12)
    u0, v0 = si.gs_initial_state(*dims, seed=5)
    u0[3, 4, 5] = np.nan
    g = _gs(torch, dims, gs.GS_FP64, u0, v0)
    r = g.integrate_adaptive(1e-6, 1e-6, 0.0, 1.0, 0.1, check=False)
    assert r["status"] == gs.GS_ERR_NONFINITE
    g.close()


@pytest.mark.parametrize("prec,rtol", [(0, 1e-300), (1, 1e-30)])
def test_unreachable_tolerance_underflows(prec, rtol):
    """atol = 0 and a tolerance no step can meet.  The problem is autonomous,
    so it starts at t = 1e12, where t + dt == t once dt < 6e-5: rejections
    shrink dt by 5x each (0.1, 0.02, ...) and STEP_UNDERFLOW follows after a
    handful of attempts, while every attempted step still changes the state
    (so the error estimate stays far above the tolerance)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (8, 8, 8)
    u0, v0 = si.gs_initial_state(*dims, seed=6)
    g = _gs(torch, dims, prec, u0, v0)
    before = to_np(g.u)
    r = g.integrate_adaptive(0.0, rtol, 1e12, 2e12, 0.1, check=False)
    assert r["status"] == gs.GS_ERR_STEP_UNDERFLOW
    assert r["n_acc"] == 0 and 2 <= r["n_rej"] <= 10, r
    # rejected attempts leave the state untouched
    assert np.array_equal(to_np(g.u), before)
    g.close()


def test_invalid_calls():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    g = _gs(torch, (8, 8, 8), gs.GS_FP64, *si.gs_initial_state(8, 8, 8))
    with pytest.raises(gs.GSError):
        g.step(17, 0.0, 0.1, 1)
    with pytest.raises(gs.GSError):
        g.step(gs.GS_RK4, 0.0, 0.1, -1)
    for ty, zc in ((1, 0), (15, 0), (6, -1), (6, 1025)):
        with pytest.raises(gs.GSError):
            gs.gs_set_tile(g.ctx, ty, zc)
    assert g.step(gs.GS_RK4, 0.0, 0.1, 0) == 0.0
    g.close()


def _light_cone_check(state_after, u0, v0, dims, method, dt, nsteps, radius, centers, tol):
    """Oracle values of sampled cells computed on periodic boxes around them
    (the dependence cone of nsteps steps lies inside the box).  Each sampled
    cell is checked on its own (|gpu - oracle| <= tol * max |oracle| over the
    samples, per component) and the samples pooled by relative L2."""
    gu, gv = state_after
    h = [2.5 / n for n in dims]
    e = 2 * radius + 1
    p = oracle.GSParams(e, e, e, L=e * h[0], Ly=e * h[1], Lz=e * h[2])
    got, ref = [], []
    for c in centers:
        bu, bv = periodic_box(u0, c, radius), periodic_box(v0, c, radius)
        ou, ov = oracle.gs_integrate_const(p, bu, bv, method, dt, nsteps)
        ref.append([ou[radius, radius, radius], ov[radius, radius, radius]])
        got.append([gu[c], gv[c]])
    got, ref = np.array(got), np.array(ref)
    assert_parity([got[:, 0], got[:, 1]], [ref[:, 0], ref[:, 1]], tol, "sampled cells")


def _seam_centers(n, ty, rng, count=64):
    """Sample cells (z, y, x) of an n^3 grid on the places a tiling can get
    wrong: x at the periodic seam and at the 128-cell row boundaries, y at the
    periodic seam and at the tile-height boundaries of every height in ty (an
    int or several), z at the seam and at the middle (where two z-bands of the
    column-split schedule meet), plus random cells; count in total."""
    xs = sorted({0, 1, 126, 127, 128, 129, n - 2, n - 1})
    ys = {0, n - 1}
    for t in ([ty] if isinstance(ty, int) else ty):
        ys |= {t - 1, t, 2 * t - 1, 2 * t, (n // t) * t - 1, (n // t) * t}
    ys = sorted(ys - {n})
    zs = sorted({0, n // 2 - 1, n // 2, n // 4, n - 1})
    grid = [(z, y, x) for z in zs for y in ys for x in xs]
    pick = rng.choice(len(grid), size=min(count - 16, len(grid)), replace=False)
    centers = [grid[i] for i in sorted(pick)]
    centers += [tuple(int(a) for a in rng.integers(0, n, 3)) for _ in range(count - len(centers))]
    return centers


@pytest.mark.parametrize("fusion", [1, 0])
def test_full_size_256cubed_fp32_dopri5_sampled(fusion):
    """256^3 FP32 (the large adaptive workload's grid and kernels, autotuned
    launch shapes; stage pairs and single stages): 3 fixed Dopri5 steps, 64
    sampled cells -- on the periodic seams, the row and tile-height
    boundaries and the z-band joins -- each against the oracle on its
    dependence cone (radius 6 per step)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    n = 256
    u0, v0 = si.gs_initial_state(n, n, n, seed=2)
    u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, (n, n, n), gs.GS_FP32, u0, v0)
    gs.gs_autotune(g.ctx)
    gs.gs_set_dopri5_fusion(g.ctx, fusion)  # the tuned launch shapes of either path
    g.step(gs.GS_DOPRI5, 0.0, 0.5, 3)
    gu, gv = to_np(g.u), to_np(g.v)
    # the tile heights of all three pair kernels (2+3 and 4+5 may run 16-warp tiles)
    ty = [c[0] for c in gs.gs_get_pair_configs(g.ctx)[:3]] if fusion else gs.gs_get_stage_configs(g.ctx)[6][1]
    centers = _seam_centers(n, ty, np.random.default_rng(0))
    assert len(centers) == 64
    oracle.set_threads(oracle.max_threads())
    try:
        _light_cone_check((gu, gv), u0, v0, (n, n, n), oracle.DOPRI5, 0.5, 3, 19, centers, FP32_TOL)
    finally:
        oracle.set_threads(1)
    g.close()


def test_full_size_256cubed_adaptive_properties():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    n = 256
    u0, v0 = si.gs_initial_state(n, n, n, seed=2)
    g = _gs(torch, (n, n, n), gs.GS_FP32, u0, v0)
    gs.gs_set_step_log(g.ctx, 100)
    r = g.integrate_adaptive(1e-6, 1e-6, 0.0, math.inf, 0.1, max_accepted=10)
    dts, cnt = gs.gs_get_step_log(g.ctx, 100)
    assert r["status"] == 0 and r["n_acc"] == 10 and cnt == 10
    assert r["t"] == pytest.approx(float(np.sum(dts)), rel=1e-14)
    assert bool(torch.isfinite(g.u).all()) and bool(torch.isfinite(g.v).all())
    # the accepted steps replayed by the oracle (fixed Dormand-Prince steps of
    # the logged sizes) on the dependence cones of sampled cells: radius 6 per
    # step (y5 uses k1..k6), 10 steps
    gu, gv = to_np(g.u), to_np(g.v)
    g.close()
    u32, v32 = _round32(u0), _round32(v0)
    radius = 61
    e = 2 * radius + 1
    p = oracle.GSParams(e, e, e, L=e * 2.5 / n)
    centers = [(0, 0, 0), (255, 130, 127), (128, 7, 128), (96, 251, 255), (160, 160, 96), (31, 200, 64)]
    oracle.set_threads(oracle.max_threads())
    got, ref = [], []
    try:
        for c in centers:
            bu, bv = periodic_box(u32, c, radius), periodic_box(v32, c, radius)
            ou, ov = oracle.gs_integrate_replay(p, bu, bv, oracle.DOPRI5, dts)
            ref.append([ou[radius, radius, radius], ov[radius, radius, radius]])
            got.append([gu[c], gv[c]])
    finally:
        oracle.set_threads(1)
    got, ref = np.array(got), np.array(ref)
    assert_parity([got[:, 0], got[:, 1]], [ref[:, 0], ref[:, 1]], FP32_TOL, "adaptive 256^3 sampled cells")


# ------------------------------------------------------------ DC-PSE Laplacian
PAPER_GS = dict(Du=2e-4, Dv=1e-4, F=0.053, k=0.014)  # the paper's constants


def test_dcpse_stencil_matches_oracle():
    """The library's weights (Cholesky of the moment system) against the
    oracle's (Gaussian elimination), isotropic and anisotropic grids."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    for dims, L in (((64, 64, 64), (2.5, 2.5, 2.5)), ((20, 12, 9), (2.5, 1.5, 3.0))):
        g = gs.GrayScott(*dims, L=L[0], Ly=L[1], Lz=L[2], prec=gs.GS_FP64, **PAPER_GS)
        gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
        off, w = gs.gs_get_dcpse_stencil(g.ctx)
        h = (L[0] / dims[0], L[1] / dims[1], L[2] / dims[2])
        ooff, ow = oracle.dcpse_stencil(h, 3.1)
        mine = {tuple(o): x for o, x in zip(off.tolist(), w)}
        ref = {tuple(o): x for o, x in zip(ooff.tolist(), ow)}
        assert mine.keys() == ref.keys() and len(mine) == 122
        scale = max(abs(x) for x in ref.values())
        assert max(abs(mine[k] - ref[k]) for k in ref) < 1e-11 * scale
        g.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(16, 12, 20), (9, 8, 7), (4, 4, 4), (64, 64, 64)])
def test_dcpse_rhs_matches_oracle(prec, dims):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    u0, v0 = si.gs_initial_state(*dims, seed=61)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, dims, prec, u0, v0, **PAPER_GS)
    gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
    fu, fv = g.rhs()
    ou, ov = oracle.gs_dcpse_rhs(oracle.GSParams(*dims, **PAPER_GS), u0, v0)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    assert_parity([to_np(fu), to_np(fv)], [ou, ov], tol)
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("method,omethod", [("euler", oracle.EULER), ("rk4", oracle.RK4), ("dopri5", oracle.DOPRI5)])
def test_dcpse_fixed_steps_match_oracle(prec, method, omethod):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (16, 12, 10)
    u0, v0 = si.gs_initial_state(*dims, seed=62)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, dims, prec, u0, v0, **PAPER_GS)
    gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
    m = {"euler": gs.GS_EULER, "rk4": gs.GS_RK4, "dopri5": gs.GS_DOPRI5}[method]
    t = g.step(m, 0.0, 1.0, 4)
    assert t == 4.0
    ou, ov = oracle.gs_dcpse_integrate_const(oracle.GSParams(*dims, **PAPER_GS), u0, v0, omethod, 1.0, 4)
    tol = FP64_TOL if prec == 0 else FP32_TOL
    assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], tol)
    with pytest.raises(RuntimeError):
        g.step(gs.GS_AB4, 0.0, 1.0, 4)
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_dcpse_tile_depths_agree(prec):
    """Tiles of 8 x 8 x 4 and 8 x 8 x 8 cells give bit-identical states (every
    cell's sums run in the same order), on a ragged grid, for RK4 steps and
    an adaptive Dormand-Prince run, and both match the oracle."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (20, 12, 9)
    u0, v0 = si.gs_initial_state(*dims, seed=63)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    tol = 1e-8 if prec == 0 else 1e-5
    runs = {}
    for tz in (4, 8):
        g = _gs(torch, dims, prec, u0, v0, **PAPER_GS)
        gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
        gs.gs_set_dcpse_tile(g.ctx, tz)
        g.step(gs.GS_RK4, 0.0, 1.0, 3)
        mid = (to_np(g.u).copy(), to_np(g.v).copy())
        r = g.integrate_adaptive(tol, tol, 3.0, 6.0, 1.0)
        runs[tz] = (mid, to_np(g.u).copy(), to_np(g.v).copy(), r["n_acc"], r["n_rej"])
        with pytest.raises(RuntimeError):
            gs.gs_set_dcpse_tile(g.ctx, 6)
        g.close()
    assert runs[4][3:] == runs[8][3:]
    for a, b in ((runs[4][0][0], runs[8][0][0]), (runs[4][0][1], runs[8][0][1]), (runs[4][1], runs[8][1]),
                 (runs[4][2], runs[8][2])):
        assert np.array_equal(a, b)
    p = oracle.GSParams(*dims, **PAPER_GS)
    ou, ov = oracle.gs_dcpse_integrate_const(p, u0, v0, oracle.RK4, 1.0, 3)
    bar = FP64_TOL if prec == 0 else FP32_TOL
    assert_parity(list(runs[4][0]), [ou, ov], bar)
    if prec == 0:  # the FP64 run takes the oracle's steps
        ref = oracle.gs_dcpse_integrate_adaptive(p, ou, ov, 3.0, 6.0, 1.0, tol, tol)
        assert (ref["n_acc"], ref["n_rej"]) == runs[4][3:]
        assert_parity([runs[4][1], runs[4][2]], [ref["u"], ref["v"]], bar)


def test_dcpse_adaptive_fp64_matches_oracle_run():
    """Error-controlled Dopri5 with the DC-PSE Laplacian (host controller):
    same accepted / rejected counts and step sizes as the oracle's run."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (16, 16, 16)
    u0, v0 = si.gs_initial_state(*dims, seed=2)
    g = _gs(torch, dims, gs.GS_FP64, u0, v0, **PAPER_GS)
    gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
    gs.gs_set_step_log(g.ctx, 1000)
    r = g.integrate_adaptive(1e-8, 1e-8, 0.0, 20.0, 1.0)
    dts, cnt = gs.gs_get_step_log(g.ctx, 1000)
    ref = oracle.gs_dcpse_integrate_adaptive(oracle.GSParams(*dims, **PAPER_GS), u0, v0, 0.0, 20.0, 1.0, 1e-8, 1e-8,
                                             log_cap=1000)
    assert r["status"] == 0 and ref["status"] == 0 and r["t"] == 20.0
    assert (r["n_acc"], r["n_rej"]) == (ref["n_acc"], ref["n_rej"]) and cnt == r["n_acc"]
    assert np.allclose(dts, ref["dts"], rtol=1e-7, atol=0)
    assert_parity([to_np(g.u), to_np(g.v)], [ref["u"], ref["v"]], FP64_TOL)
    g.close()


def test_dcpse_paper_workload_64cubed_rk4():
    """The paper's Gray-Scott run: 64^3 on [0,2.5]^3, d1 = 2e-4, d2 = 1e-4,
    F = 0.053, K = 0.014, DC-PSE Laplacian, RK4 with dt = 1 to t_f = 20, FP64:
    against the oracle, and the 7-point path differs (the operators differ)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (64, 64, 64)
    u0, v0 = si.gs_initial_state(*dims, seed=2)
    g = _gs(torch, dims, gs.GS_FP64, u0, v0, **PAPER_GS)
    gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
    g.step(gs.GS_RK4, 0.0, 1.0, 20)
    ou, ov = oracle.gs_dcpse_integrate_const(oracle.GSParams(*dims, **PAPER_GS), u0, v0, oracle.RK4, 1.0, 20)
    assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], FP64_TOL)
    g.close()


# ---------------------------------- Cash-Karp 5(4) and Fehlberg 7(8) (Table 1)
TAB_METHODS = [("ck54", oracle.CK54), ("rkf78", oracle.RKF78)]


def _tab_run_oracle(lap, dims, phys, u0, v0, omethod, dt, n):
    p = oracle.GSParams(*dims, **phys)
    if lap == "dcpse":
        return oracle.gs_dcpse_integrate_const(p, u0, v0, omethod, dt, n)
    return oracle.gs_integrate_const(p, u0, v0, omethod, dt, n)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("lap", ["7point", "dcpse"])
@pytest.mark.parametrize("method,omethod", TAB_METHODS + [("midpoint", oracle.MIDPOINT)])
@pytest.mark.parametrize("dims", [(16, 12, 10), (9, 5, 4), (20, 8, 1)])
def test_tableau_path_fixed_steps_match_oracle(prec, lap, method, omethod, dims):
    """Cash-Karp and Fehlberg fixed steps on the Gray-Scott grid (the tableau
    path: one tiled stage kernel per stage, 13 stages for Fehlberg), with the
    7-point and the DC-PSE Laplacian, ragged tiles and a single plane,
    against the oracle's generic tableau step."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    phys = PAPER_GS if lap == "dcpse" else dict(Du=3e-3, Dv=1.5e-3)
    dt = 1.0 if lap == "dcpse" else 0.25
    u0, v0 = si.gs_initial_state(*dims, seed=71)
    if prec == 1:
        u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, dims, prec, u0, v0, **phys)
    if lap == "dcpse":
        gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
    m = {"ck54": gs.GS_CK54, "rkf78": gs.GS_RKF78, "midpoint": gs.GS_MIDPOINT}[method]
    t = g.step(m, 0.0, dt, 3)
    assert t == 3 * dt
    ou, ov = _tab_run_oracle(lap, dims, phys, u0, v0, omethod, dt, 3)
    assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], FP64_TOL if prec == 0 else FP32_TOL, (lap, method))
    g.close()


@pytest.mark.parametrize("lap", ["7point", "dcpse"])
@pytest.mark.parametrize("method,omethod", TAB_METHODS)
def test_tableau_path_adaptive_fp64_matches_oracle_run(lap, method, omethod):
    """Error-controlled Cash-Karp 5(4) and Fehlberg 7(8) (controller with the
    pair's orders p, q): the oracle's accepted / rejected counts and step
    sizes, the state within the FP64 bound."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (16, 12, 10)
    phys = PAPER_GS if lap == "dcpse" else dict(Du=3e-3, Dv=1.5e-3)
    u0, v0 = si.gs_initial_state(*dims, seed=72)
    g = _gs(torch, dims, gs.GS_FP64, u0, v0, **phys)
    if lap == "dcpse":
        gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
    gs.gs_set_step_log(g.ctx, 1000)
    pair = {"ck54": gs.GS_CK54, "rkf78": gs.GS_RKF78}[method]
    r = g.integrate_adaptive(1e-9, 1e-9, 0.0, 20.0, 1.0, pair=pair)
    dts, cnt = gs.gs_get_step_log(g.ctx, 1000)
    p = oracle.GSParams(*dims, **phys)
    run = oracle.gs_dcpse_integrate_adaptive if lap == "dcpse" else oracle.gs_integrate_adaptive
    ref = run(p, u0, v0, 0.0, 20.0, 1.0, 1e-9, 1e-9, log_cap=1000, method=omethod)
    assert r["status"] == 0 and ref["status"] == 0 and r["t"] == 20.0
    assert (r["n_acc"], r["n_rej"]) == (ref["n_acc"], ref["n_rej"]) and cnt == r["n_acc"]
    assert ref["n_acc"] > 3  # the controller really worked
    # Fehlberg's error estimate is dt 41/840 (k1 + k11 - k12 - k13), a
    # difference of four nearly equal stage values (|k| ~ 1e-2, |err| ~ 1e-9
    # here): stage values that differ by 1e-15 relative (FMA, the order of
    # the stencil sums) move E by ~1e-5 relative, and dt follows E^(-1/8);
    # the clipped last step inherits the accumulated difference of t.
    # Cash-Karp's estimate cancels far less.
    if method == "rkf78":
        assert np.allclose(dts[:-1], ref["dts"][:-1], rtol=1e-4, atol=0)
        assert abs(dts[-1] - ref["dts"][-1]) <= 1e-4 * 20.0
    else:
        assert np.allclose(dts, ref["dts"], rtol=1e-7, atol=0)
    assert_parity([to_np(g.u), to_np(g.v)], [ref["u"], ref["v"]], FP64_TOL)
    g.close()


def test_tableau_path_adaptive_fp32_and_invalid():
    """FP32 state with the FP64 controller against the FP64 oracle (1e-5);
    pairs without an embedded solution are rejected."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (24, 16, 12)
    u0, v0 = si.gs_initial_state(*dims, seed=73)
    u0, v0 = _round32(u0), _round32(v0)
    g = _gs(torch, dims, gs.GS_FP32, u0, v0, Du=3e-3, Dv=1.5e-3)
    r = g.integrate_adaptive(1e-6, 1e-6, 0.0, 5.0, 0.2, pair=gs.GS_RKF78)
    ref = oracle.gs_integrate_adaptive(oracle.GSParams(*dims, Du=3e-3, Dv=1.5e-3), u0, v0, 0.0, 5.0, 0.2, 1e-6, 1e-6,
                                       method=oracle.RKF78)
    assert r["t"] == 5.0 and abs(r["n_acc"] - ref["n_acc"]) <= 1
    assert_parity([to_np(g.u), to_np(g.v)], [ref["u"], ref["v"]], FP32_TOL)
    for bad in (gs.GS_RK4, gs.GS_EULER, gs.GS_AB4, gs.GS_MIDPOINT, 17):
        with pytest.raises(RuntimeError):
            g.integrate_adaptive(1e-6, 1e-6, 5.0, 6.0, 0.2, pair=bad)
    g.close()


def test_dcpse_paper_workload_64cubed_rkf78():
    """The paper's Gray-Scott run with its third stepper: 64^3, d1 = 2e-4,
    d2 = 1e-4, DC-PSE, Fehlberg 7(8) with dt = 1 to t_f = 20, FP64, against
    the oracle."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    dims = (64, 64, 64)
    u0, v0 = si.gs_initial_state(*dims, seed=2)
    g = _gs(torch, dims, gs.GS_FP64, u0, v0, **PAPER_GS)
    gs.gs_set_laplacian(g.ctx, gs.GS_LAP_DCPSE, 3.1)
    g.step(gs.GS_RKF78, 0.0, 1.0, 20)
    oracle.set_threads(oracle.max_threads())
    try:
        ou, ov = oracle.gs_dcpse_integrate_const(oracle.GSParams(*dims, **PAPER_GS), u0, v0, oracle.RKF78, 1.0, 20)
    finally:
        oracle.set_threads(1)
    assert_parity([to_np(g.u), to_np(g.v)], [ou, ov], FP64_TOL)
    g.close()
