"""GPU parity of the batched ensemble (uneven grids, per-instance F, k and
per-instance adaptive Dormand-Prince) against the oracle run instance by
instance, against single-grid runs, and at the full 512-instance size."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from tests._gpu_common import assert_parity, cuda_or_skip, to_np

pytestmark = pytest.mark.gpu

SMALL = [dict(nx=12, ny=9, nz=7, F=0.03, k=0.05), dict(nx=5, ny=16, nz=3, F=0.045, k=0.061),
         dict(nx=33, ny=4, nz=10, F=0.053, k=0.014), dict(nx=1, ny=1, nz=1, F=0.04, k=0.06),
         dict(nx=8, ny=8, nz=8, F=0.025, k=0.055), dict(nx=17, ny=23, nz=5, F=0.058, k=0.065),
         dict(nx=40, ny=2, nz=1, F=0.035, k=0.045)]
PHYS = dict(Du=2e-3, Dv=1e-3)


def _inits(insts, seed0=100, round32=False):
    out = []
    for i, d in enumerate(insts):
        u, v = si.gs_initial_state(d["nx"], d["ny"], d["nz"], seed=seed0 + i)
        if round32:
            u, v = u.astype(np.float32).astype(np.float64), v.astype(np.float32).astype(np.float64)
        out.append((u, v))
    return out


def _batch(torch, insts, inits, prec):
    import paper_2309_05331_b300 as gs
    b = gs.GrayScottBatch(insts, L=2.5, prec=prec, **PHYS)
    for i, (u, v) in enumerate(inits):
        b.set_instance(i, torch.from_numpy(u), torch.from_numpy(v))
    return b


def _oracle_adaptive(d, u, v, t_end, tol, max_acc=-1, log_cap=0):
    p = oracle.GSParams(d["nx"], d["ny"], d["nz"], F=d["F"], k=d["k"], **PHYS)
    return oracle.gs_integrate_adaptive(p, u, v, 0.0, t_end, 0.1, tol, tol, max_acc=max_acc, log_cap=log_cap)


def test_batched_fp64_matches_oracle_per_instance():
    torch = cuda_or_skip()
    inits = _inits(SMALL)
    b = _batch(torch, SMALL, inits, 0)
    b.set_step_log(200)
    r = b.integrate_adaptive(1e-8, 1e-8, 0.0, 5.0, 0.1)
    logs = b.step_log()
    for i, d in enumerate(SMALL):
        ref = _oracle_adaptive(d, *inits[i], 5.0, 1e-8, log_cap=200)
        assert r["t"][i] == 5.0 and ref["t"] == 5.0
        assert (r["n_acc"][i], r["n_rej"][i]) == (ref["n_acc"], ref["n_rej"]), i
        assert np.allclose(logs[i], ref["dts"], rtol=1e-7, atol=0), i
        gu, gv = b.view(i)
        assert_parity([to_np(gu), to_np(gv)], [ref["u"], ref["v"]], 1e-12, i)
    b.close()


def test_batched_fp32_against_fp64_oracle():
    torch = cuda_or_skip()
    inits = _inits(SMALL, round32=True)
    b = _batch(torch, SMALL, inits, 1)
    r = b.integrate_adaptive(1e-6, 1e-6, 0.0, 8.0, 0.1)
    for i, d in enumerate(SMALL):
        ref = _oracle_adaptive(d, *inits[i], 8.0, 1e-6)
        assert abs(int(r["n_acc"][i]) - ref["n_acc"]) <= 1
        gu, gv = b.view(i)
        assert_parity([to_np(gu), to_np(gv)], [ref["u"], ref["v"]], 1e-5, i)
    b.close()


def test_failure_of_one_instance_is_isolated():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    inits = _inits(SMALL)
    inits[2][0][1, 2, 3] = np.nan
    b = _batch(torch, SMALL, inits, 0)
    r = b.integrate_adaptive(1e-8, 1e-8, 0.0, 2.0, 0.1, check=False)
    assert r["status"] == gs.GS_ERR_NONFINITE
    assert r["statuses"][2] == gs.GS_ERR_NONFINITE
    for i, d in enumerate(SMALL):
        if i == 2:
            continue
        assert r["statuses"][i] == gs.GS_OK and r["t"][i] == 2.0
        ref = _oracle_adaptive(d, *inits[i], 2.0, 1e-8)
        gu, gv = b.view(i)
        assert_parity([to_np(gu), to_np(gv)], [ref["u"], ref["v"]], 1e-12, i)
    b.close()


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_batched_equals_single_grid_runs(depth):
    """Batched ensemble (vectorised segment code, or staged with ring depth
    1, 2) against single-grid runs of each instance: same step counts, FP64
    states within 1e-13."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    insts = SMALL[:3] + SMALL[4:]
    inits = _inits(insts, seed0=7)
    b = _batch(torch, insts, inits, 0)
    b.set_stage_depth(depth)
    r = b.integrate_adaptive(1e-8, 1e-8, 0.0, 3.0, 0.1)
    for i, d in enumerate(insts):
        g = gs.GrayScott(d["nx"], d["ny"], d["nz"], L=2.5, F=d["F"], k=d["k"], prec=gs.GS_FP64, **PHYS)
        g.set_state(torch.from_numpy(inits[i][0]), torch.from_numpy(inits[i][1]))
        rs = g.integrate_adaptive(1e-8, 1e-8, 0.0, 3.0, 0.1)
        assert (rs["n_acc"], rs["n_rej"]) == (r["n_acc"][i], r["n_rej"][i])
        gu, gv = b.view(i)
        assert_parity([to_np(gu), to_np(gv)], [to_np(g.u), to_np(g.v)], 1e-13)
        g.close()
    b.close()


@pytest.mark.parametrize("tile", [(2, 1), (4, 5), (14, 64)])
def test_batched_segment_shape_does_not_change_results(tile):
    torch = cuda_or_skip()
    inits = _inits(SMALL, seed0=11)
    res = []
    for ty, zc in [(6, 16), tile]:
        b = _batch(torch, SMALL, inits, 0)
        b.set_tile(ty, zc)
        b.integrate_adaptive(1e-7, 1e-7, 0.0, 1.0, 0.1)
        res.append([to_np(x) for i in range(len(SMALL)) for x in b.view(i)])
        b.close()
    for a, c in zip(*res):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("group_cells", [1, 2000, 30000, 0])
def test_instance_grouping_does_not_change_results(group_cells):
    """Stages run group by group (cache blocking): every grouping, from one
    instance per group to a single group, gives bit-identical results (each
    instance's arithmetic and max-norm are independent of the order)."""
    torch = cuda_or_skip()
    inits = _inits(SMALL, seed0=17)
    res = []
    for gc in (0, group_cells):
        b = _batch(torch, SMALL, inits, 0)
        b.set_grouping(gc)
        budget, ngroups = b.grouping()
        if gc == 1:
            assert ngroups == len(SMALL)  # at least one instance per group
        if gc == 0:
            assert ngroups == 1
        r = b.integrate_adaptive(1e-7, 1e-7, 0.0, 1.0, 0.1)
        res.append(([to_np(x) for i in range(len(SMALL)) for x in b.view(i)], r["n_acc"].copy(), r["n_rej"].copy()))
        b.close()
    (a0, acc0, rej0), (a1, acc1, rej1) = res
    assert np.array_equal(acc0, acc1) and np.array_equal(rej0, rej1)
    for a, c in zip(a0, a1):
        assert np.array_equal(a, c)


def test_grouping_rejects_invalid_budget():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    inits = _inits(SMALL, seed0=1)
    b = _batch(torch, SMALL, inits, 0)
    with pytest.raises(gs.GSError):
        b.set_grouping(-2)
    b.set_grouping(-1)
    budget, ngroups = b.grouping()
    assert budget > 0 and ngroups >= 1
    b.close()


def test_batched_max_accepted_and_per_instance_times():
    torch = cuda_or_skip()
    inits = _inits(SMALL, seed0=3)
    b = _batch(torch, SMALL, inits, 1)
    t0 = np.linspace(0.0, 3.0, len(SMALL))
    r = b.integrate_adaptive(1e-6, 1e-6, t0, np.inf, 0.1, max_accepted=4)
    assert np.all(r["n_acc"] == 4) and np.all(r["t"] > t0)
    b.close()


@pytest.mark.parametrize("ty,depth", [(7, 2), (3, 1), (1, 3), (12, 2), (9, 1)])
def test_batched_pairs_fp64_match_oracle(ty, depth):
    """The batch's stage pairs (stages 2+3, 4+5, 6+7 each one launch, one cell
    per lane, any nx): every instance takes the oracle's accepted / rejected
    steps and step sizes and matches its state element by element; odd and
    tiny grids (1^3, nx = 5, 17, 33), tile heights above ny."""
    torch = cuda_or_skip()
    inits = _inits(SMALL, seed0=300)
    b = _batch(torch, SMALL, inits, 0)
    b.set_pairs(1, ty, depth)
    assert b.pairs() == (1, ty, depth)
    b.set_step_log(200)
    r = b.integrate_adaptive(1e-8, 1e-8, 0.0, 5.0, 0.1)
    logs = b.step_log()
    for i, d in enumerate(SMALL):
        ref = _oracle_adaptive(d, *inits[i], 5.0, 1e-8, log_cap=200)
        assert r["t"][i] == 5.0 and ref["t"] == 5.0
        assert (r["n_acc"][i], r["n_rej"][i]) == (ref["n_acc"], ref["n_rej"]), i
        assert np.allclose(logs[i], ref["dts"], rtol=1e-7, atol=0), i
        gu, gv = b.view(i)
        assert_parity([to_np(gu), to_np(gv)], [ref["u"], ref["v"]], 1e-12, i)
    b.close()


def test_batched_pairs_fp32_match_oracle_replay_and_single_stages():
    """FP32 batch with the stage pairs: every instance against the FP64 oracle
    replaying its logged step sizes (1e-5), and against the same batch run
    with the single-stage kernels (the same formulas in another order)."""
    torch = cuda_or_skip()
    inits = _inits(SMALL, seed0=310, round32=True)
    res = []
    for pairs in (1, 0):
        b = _batch(torch, SMALL, inits, 1)
        b.set_pairs(pairs, 5, 2)
        b.set_step_log(200)
        r = b.integrate_adaptive(1e-6, 1e-6, 0.0, 4.0, 0.1)
        assert np.all(r["statuses"] == 0) and np.all(r["t"] == 4.0)
        logs = b.step_log()
        states = [tuple(to_np(x) for x in b.view(i)) for i in range(len(SMALL))]
        res.append((logs, states, r["n_acc"].copy()))
        b.close()
    for i, d in enumerate(SMALL):
        p = oracle.GSParams(d["nx"], d["ny"], d["nz"], F=d["F"], k=d["k"], **PHYS)
        ou, ov = oracle.gs_integrate_replay(p, *inits[i], oracle.DOPRI5, res[0][0][i])
        assert_parity(list(res[0][1][i]), [ou, ov], 1e-5, i)
        if res[0][2][i] == res[1][2][i] and np.allclose(res[0][0][i], res[1][0][i], rtol=1e-5):
            assert_parity(list(res[0][1][i]), list(res[1][1][i]), 1e-5, ("pairs vs stages", i))


# instances whose rows allow 4 (FP32: nx > 64, a multiple of 4) or 2 (nx > 32,
# even) cells per lane in the stage pairs, with partial last columns (100 of
# 128 cells; 130 = 64 + 64 + 2), and two that keep one cell per lane
WIDE = [dict(nx=96, ny=9, nz=5, F=0.03, k=0.05), dict(nx=68, ny=13, nz=3, F=0.045, k=0.061),
        dict(nx=100, ny=4, nz=6, F=0.053, k=0.014), dict(nx=130, ny=5, nz=4, F=0.04, k=0.06),
        dict(nx=66, ny=7, nz=5, F=0.025, k=0.055), dict(nx=34, ny=3, nz=9, F=0.058, k=0.065),
        dict(nx=35, ny=6, nz=4, F=0.035, k=0.045), dict(nx=12, ny=9, nz=7, F=0.05, k=0.06)]


@pytest.mark.parametrize("tyw,depth", [(7, 2), (3, 1), (5, 3)])
def test_batched_pairs_wide_lanes_fp64_match_oracle_and_one_cell_lanes(tyw, depth):
    """FP64 batch with the stage pairs at 2 cells (16 bytes) per lane where nx
    is even and above 32: every instance takes the oracle's accepted /
    rejected steps and step sizes and matches its state element by element,
    and the run is bit-identical to the one with one cell per lane
    everywhere (the per-cell arithmetic does not depend on the lane width)."""
    torch = cuda_or_skip()
    inits = _inits(WIDE, seed0=400)
    res = []
    for mode in (1, 0):
        b = _batch(torch, WIDE, inits, 0)
        b.set_pairs(1, 7, depth)
        b.set_pair_lanes(mode, tyw)
        assert b.pair_lanes() == (mode, tyw, [2, 6, 0] if mode else [8, 0, 0])
        b.set_step_log(1000)
        r = b.integrate_adaptive(1e-8, 1e-8, 0.0, 1.0, 0.1)
        res.append((b.step_log(), [tuple(to_np(x) for x in b.view(i)) for i in range(len(WIDE))],
                    r["n_acc"].copy(), r["n_rej"].copy()))
        b.close()
    logs, states, nacc, nrej = res[0]
    for i, d in enumerate(WIDE):
        ref = _oracle_adaptive(d, *inits[i], 1.0, 1e-8, log_cap=1000)
        assert (nacc[i], nrej[i]) == (ref["n_acc"], ref["n_rej"]) and nacc[i] <= 1000, i
        assert np.allclose(logs[i], ref["dts"], rtol=1e-7, atol=0), i
        assert_parity(list(states[i]), [ref["u"], ref["v"]], 1e-12, i)
        assert np.array_equal(logs[i], res[1][0][i]), i
        assert np.array_equal(states[i][0], res[1][1][i][0]) and np.array_equal(states[i][1], res[1][1][i][1]), i


@pytest.mark.parametrize("tyw,depth", [(7, 1), (4, 2)])
def test_batched_pairs_wide_lanes_fp32_match_oracle_replay(tyw, depth):
    """FP32 batch with the stage pairs at 4 cells per lane (nx > 64, a multiple
    of 4), 2 (nx > 32, even) and 1 (the rest): every instance against the
    FP64 oracle replaying its logged step sizes, cell by cell (1e-5), and
    against the run with one cell per lane everywhere."""
    torch = cuda_or_skip()
    inits = _inits(WIDE, seed0=410, round32=True)
    res = []
    for mode in (1, 0):
        b = _batch(torch, WIDE, inits, 1)
        b.set_pairs(1, 9, depth)
        b.set_pair_lanes(mode, tyw)
        assert b.pair_lanes()[2] == ([2, 3, 3] if mode else [8, 0, 0])
        b.set_step_log(1000)
        r = b.integrate_adaptive(1e-6, 1e-6, 0.0, 1.0, 0.1)
        assert np.all(r["statuses"] == 0) and np.all(r["t"] == 1.0)
        assert np.all(r["n_acc"] <= 1000)
        res.append((b.step_log(), [tuple(to_np(x) for x in b.view(i)) for i in range(len(WIDE))],
                    r["n_acc"].copy()))
        b.close()
    for i, d in enumerate(WIDE):
        p = oracle.GSParams(d["nx"], d["ny"], d["nz"], F=d["F"], k=d["k"], **PHYS)
        ou, ov = oracle.gs_integrate_replay(p, *inits[i], oracle.DOPRI5, res[0][0][i])
        gu, gv = res[0][1][i]
        assert_parity([gu, gv], [ou, ov], 1e-5, i)
        for a, o in ((gu, ou), (gv, ov)):
            assert np.max(np.abs(a - o)) <= 1e-5 * np.max(np.abs(o)), i
        if res[0][2][i] == res[1][2][i] and np.allclose(res[0][0][i], res[1][0][i], rtol=1e-5):
            assert_parity(list(res[0][1][i]), list(res[1][1][i]), 1e-5, ("4/2 vs 1 cells per lane", i))


@pytest.mark.parametrize("group_cells", [1, 6000, 0])
def test_pair_lanes_with_instance_groups_bit_identical(group_cells):
    """Stage pairs at every lane width, run group by group (one launch per
    lane width and group, each from its own counter): the same bits as one
    group, in FP64."""
    torch = cuda_or_skip()
    inits = _inits(WIDE, seed0=420)
    res = []
    for gc in (0, group_cells):
        b = _batch(torch, WIDE, inits, 0)
        b.set_pairs(1, 5, 2)
        b.set_grouping(gc)
        if gc == 1:
            assert b.grouping()[1] == len(WIDE)
        r = b.integrate_adaptive(1e-7, 1e-7, 0.0, 0.5, 0.1)
        res.append(([to_np(x) for i in range(len(WIDE)) for x in b.view(i)], r["n_acc"].copy(), r["n_rej"].copy()))
        b.close()
    (a0, acc0, rej0), (a1, acc1, rej1) = res
    assert np.array_equal(acc0, acc1) and np.array_equal(rej0, rej1)
    for a, c in zip(a0, a1):
        assert np.array_equal(a, c)


def test_pair_lanes_reject_invalid_settings():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    b = _batch(torch, WIDE[:2], _inits(WIDE[:2]), 1)
    for bad in ((2, 7), (-1, 7), (1, 0), (1, 8)):
        with pytest.raises(gs.GSError):
            b.set_pair_lanes(*bad)
    assert b.pair_lanes() == (1, 7, [0, 0, 2])
    b.close()


@pytest.mark.parametrize("pairs", [0, 1])
def test_full_size_512_instance_ensemble(pairs):
    """512 instances, per-axis edges U{16..96}, F in [0.02,0.06], k in
    [0.04,0.07], FP32 state / FP64 control, 3 accepted steps each, single
    stages and stage pairs; EVERY
    instance against the FP64 oracle replaying that instance's logged
    accepted step sizes, cell by cell (an FP32 run takes its own step sizes:
    its error norms carry FP32 rounding, so its own adaptive sequence is
    not the FP64 oracle's)."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    insts = si.batch_instances(512, seed=3)
    b = gs.GrayScottBatch(insts, L=2.5, Du=2e-5, Dv=1e-5, prec=gs.GS_FP32)
    inits = []
    for i, d in enumerate(insts):
        u, v = si.gs_initial_state(d["nx"], d["ny"], d["nz"], seed=1000 + i)
        b.set_instance(i, torch.from_numpy(u), torch.from_numpy(v))
        inits.append((u, v))
    b.autotune()
    b.set_pairs(pairs, 7, 2)
    b.set_step_log(8)
    r = b.integrate_adaptive(1e-6, 1e-6, 0.0, np.inf, 0.1, max_accepted=3)
    assert np.all(r["statuses"] == 0) and np.all(r["n_acc"] == 3)
    logs = b.step_log()
    oracle.set_threads(oracle.max_threads())
    try:
        for i, d in enumerate(insts):
            assert len(logs[i]) == 3 and abs(float(np.sum(logs[i])) - r["t"][i]) <= 1e-12 * r["t"][i]
            u, v = (a.astype(np.float32).astype(np.float64) for a in inits[i])
            p = oracle.GSParams(d["nx"], d["ny"], d["nz"], F=d["F"], k=d["k"], Du=2e-5, Dv=1e-5)
            ou, ov = oracle.gs_integrate_replay(p, u, v, oracle.DOPRI5, logs[i])
            gu, gv = b.view(i)
            assert_parity([to_np(gu), to_np(gv)], [ou, ov], 1e-5, i)
    finally:
        oracle.set_threads(1)
    b.close()


def test_autotune_run_restores_state_and_picks_a_candidate():
    """The run-based tuner integrates the caller's run once per candidate tile
    and restores the bound state: afterwards the state is bit-identical to
    before, the chosen tile is a candidate, and the integration gives the
    same result as on the default tile."""
    torch = cuda_or_skip()
    inits = _inits(SMALL, seed0=23)
    b = _batch(torch, SMALL, inits, 0)
    before = [to_np(x).copy() for i in range(len(SMALL)) for x in b.view(i)]
    ty, zc, ms = b.autotune_run(1e-7, 1e-7, 0.0, 1.0, 0.1)
    pairs = b.pairs()
    if pairs[0]:
        assert (ty, zc) in {(7, 32), (7, 64), (7, 128), (10, 64), (12, 64), (12, 128)} and pairs[1] == ty and ms > 0
    else:
        assert (ty, zc) in {(4, 16), (6, 16), (6, 32), (6, 64), (8, 32), (14, 16), (14, 32)} and ms > 0
    after = [to_np(x) for i in range(len(SMALL)) for x in b.view(i)]
    assert all(np.array_equal(p, q) for p, q in zip(before, after))
    b.integrate_adaptive(1e-7, 1e-7, 0.0, 1.0, 0.1)
    tuned = [to_np(x) for i in range(len(SMALL)) for x in b.view(i)]
    b.close()
    b = _batch(torch, SMALL, inits, 0)
    b.set_pairs(*pairs)  # the same kernels on the default tile
    b.integrate_adaptive(1e-7, 1e-7, 0.0, 1.0, 0.1)
    ref = [to_np(x) for i in range(len(SMALL)) for x in b.view(i)]
    b.close()
    assert all(np.array_equal(p, q) for p, q in zip(tuned, ref))
