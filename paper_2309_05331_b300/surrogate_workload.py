"""The surrogate workload on a 128^3 Gray-Scott grid: data from the library's
own RK4 integrator, GPU training of the BF16 conv network, evaluation against
the integrator (relative L2 over 16 steps of dt = 0.1 on a held-out
trajectory) and timing against the plain integrator at matched error.

Every numerical step runs in the library's kernels (RK4 stage kernels,
surrogate forward / backward / Adam, moment and norm reductions); this module
only sequences them.
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np

import synthetic_inputs as si

from . import GS_FP32, GS_RK4, GrayScott, Surrogate, lib

DT = 0.1
STEPS = 16  # steps per surrogate advance: 1.6 time units
JUDGE_EVERY = 10  # advances per judged advance in the reported speed-up


def generate_snapshots(torch, n=128, trajectories=8, per_traj=250, seed0=0, Du=2e-5, Dv=1e-5, F=0.053, k=0.014):
    """Snapshots [traj][s] (u, v) FP32 on the GPU, STEPS RK4 steps apart."""
    cells = n ** 3
    data = torch.empty((trajectories, per_traj, 2, cells), dtype=torch.float32, device="cuda")
    g = GrayScott(n, n, n, prec=GS_FP32, Du=Du, Dv=Dv, F=F, k=k)
    for tr in range(trajectories):
        u0, v0 = si.gs_initial_state(n, n, n, seed=seed0 + tr)
        g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
        for s in range(per_traj):
            data[tr, s, 0].copy_(g.u.view(-1))
            data[tr, s, 1].copy_(g.v.view(-1))
            g.step(GS_RK4, 0.0, DT, STEPS)
    g.close()
    torch.cuda.synchronize()
    return data


def _moments(torch, x):
    acc = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = lib().sur_moments(x.numel(), x.data_ptr(), acc.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    s, q = acc.tolist()
    n = x.numel()
    return s / n, math.sqrt(max(q / n - (s / n) ** 2, 1e-30)), math.sqrt(q / n)


def fit_normalization(torch, data, train_traj):
    """Input mean / deviation per channel, increment RMS per channel."""
    mean, sd, scale = [], [], []
    d = data[:train_traj]
    for c in range(2):
        m, s, _ = _moments(torch, d[:, :, c].contiguous())
        inc = (d[:, 1:, c] - d[:, :-1, c]).contiguous()
        _, _, rms = _moments(torch, inc)
        mean.append(m)
        sd.append(s)
        scale.append(rms)
    return mean, sd, scale


def train(torch, sur, data, train_traj, iters, lr0=1e-3, lr_min=1e-5, seed=0, log_every=0):
    """Adam on random (snapshot, snapshot + 1) pairs, cosine learning rate."""
    rng = np.random.default_rng(seed)
    T, S = train_traj, data.shape[1]
    n = int(round(data.shape[-1] ** (1 / 3)))
    shape = (n, n, n)
    losses = []
    for it in range(iters):
        tr, s = int(rng.integers(T)), int(rng.integers(S - 1))
        lr = lr_min + 0.5 * (lr0 - lr_min) * (1 + math.cos(math.pi * it / max(iters - 1, 1)))
        a, b = data[tr, s], data[tr, s + 1]
        loss = sur.train_step(a[0].view(shape), a[1].view(shape), b[0].view(shape), b[1].view(shape), lr)
        losses.append(loss)
        if log_every and it % log_every == 0:
            print(f"it {it} loss {loss:.4e} lr {lr:.2e}")
    return losses


def _rel_l2_dev(torch, a0, a1, b0, b1):
    num = float(((a0 - b0).double() ** 2).sum() + ((a1 - b1).double() ** 2).sum())
    den = float((b0.double() ** 2).sum() + (b1.double() ** 2).sum())
    return math.sqrt(num / den)


def evaluate(torch, sur, data, traj):
    """rel-L2 of the surrogate and of the 'no change' prediction against the
    integrator over every pair of the held-out trajectory."""
    n = int(round(data.shape[-1] ** (1 / 3)))
    shape = (n, n, n)
    uo = torch.empty(shape, dtype=torch.float32, device="cuda")
    vo = torch.empty_like(uo)
    errs, ident = [], []
    for s in range(data.shape[1] - 1):
        a, b = data[traj, s], data[traj, s + 1]
        sur.forward(a[0].view(shape), a[1].view(shape), uo, vo)
        errs.append(_rel_l2_dev(torch, uo.view(-1), vo.view(-1), b[0], b[1]))
        ident.append(_rel_l2_dev(torch, a[0], a[1], b[0], b[1]))
    return np.array(errs), np.array(ident)


def timing(torch, sur, data, traj, reps=20):
    """Device time (CUDA events) of one surrogate advance and of 16 RK4 steps
    at dt = 0.1, and of the RK4 runs with larger steps; relative L2 of each
    against the dt = 0.1 integrator."""
    n = int(round(data.shape[-1] ** (1 / 3)))
    shape = (n, n, n)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    a, b = data[traj, 0], data[traj, 1]
    uo = torch.empty(shape, dtype=torch.float32, device="cuda")
    vo = torch.empty_like(uo)
    for _ in range(3):
        sur.forward(a[0].view(shape), a[1].view(shape), uo, vo)
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(reps):
        sur.forward(a[0].view(shape), a[1].view(shape), uo, vo)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sur = e0.elapsed_time(e1) / reps
    out = {"surrogate_ms": t_sur}
    g = GrayScott(n, n, n, prec=GS_FP32)
    for m in (16, 8, 4, 2, 1):
        g.u.view(-1).copy_(a[0])
        g.v.view(-1).copy_(a[1])
        g.step(GS_RK4, 0.0, 1.6 / m, m)  # warm-up (graph capture)
        ts = []
        for _ in range(5):
            g.u.view(-1).copy_(a[0])
            g.v.view(-1).copy_(a[1])
            torch.cuda.synchronize()
            e0.record(stream)
            g.step(GS_RK4, 0.0, 1.6 / m, m)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        err = _rel_l2_dev(torch, g.u.view(-1), g.v.view(-1), b[0], b[1])
        out[f"rk4_dt{1.6 / m:.2f}"] = {"ms": float(np.median(ts)), "rel_l2_vs_dt0.1": err}
    g.close()
    return out


def run(torch, n=128, trajectories=8, per_traj=250, iters=2000, threshold=1e-3, verbose=False):
    """Full workload; returns a dict of results."""
    res = {"grid": n, "snapshots": trajectories * per_traj, "iters": iters}
    t0 = time.perf_counter()
    data = generate_snapshots(torch, n, trajectories, per_traj)
    res["generate_s"] = time.perf_counter() - t0
    train_traj = trajectories - 1
    mean, sd, scale = fit_normalization(torch, data, train_traj)
    sur = Surrogate(n, n, n)
    sur.set_params(si.surrogate_init_params(seed=7, last_layer_scale=0.0))
    sur.set_normalization(mean, sd, scale)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(torch, sur, data, train_traj, iters, log_every=200 if verbose else 0)
    torch.cuda.synchronize()
    res["train_s"] = time.perf_counter() - t0
    res["train_ms_per_step"] = 1e3 * res["train_s"] / max(iters, 1)
    res["loss_first"] = float(np.mean(losses[:20]))
    res["loss_last"] = float(np.mean(losses[-20:]))
    errs, ident = evaluate(torch, sur, data, train_traj)
    res["heldout_rel_l2_mean"] = float(errs.mean())
    res["heldout_rel_l2_max"] = float(errs.max())
    res["heldout_identity_rel_l2_mean"] = float(ident.mean())
    res["heldout_fraction_within_threshold"] = float(np.mean(errs <= threshold))
    res["threshold"] = threshold
    tm = timing(torch, sur, data, train_traj)
    res["timing"] = tm
    cells = n ** 3
    res["surrogate_cell_steps_per_s"] = cells * STEPS / (tm["surrogate_ms"] * 1e-3)
    res["rk4_dt0.1_cell_steps_per_s"] = cells * STEPS / (tm["rk4_dt0.10"]["ms"] * 1e-3)
    # plain RK4 at matched error: the cheapest step size whose error against
    # the dt = 0.1 integrator is not above the surrogate's mean error
    best = None
    for key, v in tm.items():
        if key.startswith("rk4_") and v["rel_l2_vs_dt0.1"] <= res["heldout_rel_l2_mean"]:
            if best is None or v["ms"] < best[1]["ms"]:
                best = (key, v)
    if best is not None:
        res["rk4_matched_error"] = {"setting": best[0], **best[1],
                                    "cell_steps_per_s": cells * STEPS / (best[1]["ms"] * 1e-3)}
        res["surrogate_speedup_at_matched_error"] = best[1]["ms"] / tm["surrogate_ms"]
    res["surrogate_speedup_vs_rk4_dt0.1"] = tm["rk4_dt0.10"]["ms"] / tm["surrogate_ms"]
    # one judged advance (RK4 judge) on the held-out trajectory
    g = GrayScott(n, n, n, prec=GS_FP32)
    a = data[train_traj, per_traj // 2]
    g.u.view(-1).copy_(a[0])
    g.v.view(-1).copy_(a[1])
    rel, fb = sur.advance(g.ctx, g.u, g.v, judge=True, threshold=threshold)
    res["judge_rel_l2"] = rel
    res["judge_fell_back"] = fb
    # wall time of the public calls (each synchronises): an advance, plain
    # and judged, and the 16 RK4 steps at dt = 0.1 it stands for; the
    # speed-up with one judged advance in every JUDGE_EVERY
    def call_ms(fn, reps):
        ts = []
        for _ in range(reps):
            g.u.view(-1).copy_(a[0])
            g.v.view(-1).copy_(a[1])
            torch.cuda.synchronize()
            t_0 = time.perf_counter()
            fn()
            ts.append((time.perf_counter() - t_0) * 1e3)
        return float(np.median(ts))
    plain_ms = call_ms(lambda: sur.advance(g.ctx, g.u, g.v, judge=False, threshold=threshold), 7)
    judged_ms = call_ms(lambda: sur.advance(g.ctx, g.u, g.v, judge=True, threshold=threshold), 5)
    rk4_ms = call_ms(lambda: g.step(GS_RK4, 0.0, 0.1, STEPS), 7)
    per_call = ((JUDGE_EVERY - 1) * plain_ms + judged_ms) / JUDGE_EVERY
    res["advance"] = {"plain_ms": plain_ms, "judged_ms": judged_ms, "judge_every": JUDGE_EVERY,
                      "ms_per_call": per_call, "rk4_dt0.1_call_ms": rk4_ms,
                      "speedup_vs_rk4_dt0.1_with_judging": rk4_ms / per_call,
                      "speedup_vs_rk4_dt0.1_unjudged": rk4_ms / plain_ms}
    g.close()
    sur.close()
    del data
    torch.cuda.empty_cache()
    return res


if __name__ == "__main__":
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser(description="surrogate workload (data, training, evaluation, timing)")
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--trajectories", type=int, default=8)
    ap.add_argument("--per-traj", type=int, default=250)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--conv-engine", type=int, default=0, help="0 automatic, 1 mma.sync, 2 tcgen05 where it applies")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    assert lib().sur_set_conv_engine(a.conv_engine) == 0
    print(json.dumps(run(torch, a.grid, a.trajectories, a.per_traj, a.iters), indent=1))
