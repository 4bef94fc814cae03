"""GPU parity of the learned surrogate's BF16 tensor-core kernels against the
CPU oracle: convolution forward, input gradient and weight gradient on
BF16-rounded inputs (FP32 accumulation on the GPU, FP64 in the oracle), the
whole network's loss gradient against oracle backpropagation with the same
BF16 rounding points, training, and the RK4 judge / fallback."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from tests._gpu_common import cuda_or_skip, to_np

pytestmark = pytest.mark.gpu

ACC_TOL = 1e-5  # FP32 accumulation of exact BF16 products vs FP64


def _pad(c):
    return 8 if c <= 8 else 32


def _rand_bf16(rng, shape, scale=1.0):
    return oracle.bf16_round(scale * rng.standard_normal(shape))


def _dev_act(torch, a, cpad):
    """(D,H,W,c) float64 -> (D,H,W,cpad) BF16 on the GPU (zero padding)."""
    D, H, W, c = a.shape
    full = np.zeros((D, H, W, cpad), dtype=np.float32)
    full[..., :c] = a
    return torch.from_numpy(full).to("cuda", torch.bfloat16).contiguous()


def _packed(torch, gs, w, dgrad):
    cin, cout = w.shape[1], w.shape[2]
    nb = gs.lib().sur_packed_bytes(_pad(cout), _pad(cin)) if dgrad else gs.lib().sur_packed_bytes(_pad(cin), _pad(cout))
    buf = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    wd = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda()
    assert gs.lib().sur_pack_weights(cin, cout, wd.data_ptr(), dgrad, buf.data_ptr(), None) == 0
    return buf, wd


def _rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


SHAPES = [(2, 32), (32, 32), (32, 2)]
GRIDS = [(2, 8, 16), (4, 16, 32)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("cin,cout", SHAPES)
def test_conv_forward(grid, cin, cout):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    D, H, W = grid
    rng = np.random.default_rng(cin * 100 + cout + D)
    x = _rand_bf16(rng, (D, H, W, cin))
    w = _rand_bf16(rng, (27, cin, cout), 0.2)
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    xd = _dev_act(torch, x, _pad(cin))
    wp, _ = _packed(torch, gs, w, 0)
    bd = torch.zeros(_pad(cout), dtype=torch.float32, device="cuda")
    bd[:cout] = torch.from_numpy(b.astype(np.float32))
    out = torch.zeros((D, H, W, _pad(cout)), dtype=torch.float32, device="cuda")
    st = gs.lib().sur_conv3d(D, H, W, _pad(cin), _pad(cout), xd.data_ptr(), wp.data_ptr(), bd.data_ptr(), 3, None,
                             out.data_ptr(), _pad(cout), None)
    assert st == 0
    torch.cuda.synchronize()
    ref = oracle.conv3d_fwd(x, w, b)
    got = to_np(out)
    assert _rel(got[..., :cout], ref) < ACC_TOL
    assert np.all(got[..., cout:] == 0.0)


@pytest.mark.parametrize("cin,cout", [(32, 32), (32, 2)])
def test_conv_input_gradient(cin, cout):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    D, H, W = 4, 8, 16
    rng = np.random.default_rng(11 + cout)
    dy = _rand_bf16(rng, (D, H, W, cout))
    w = _rand_bf16(rng, (27, cin, cout), 0.2)
    dyd = _dev_act(torch, dy, _pad(cout))
    wp, _ = _packed(torch, gs, w, 1)
    out = torch.zeros((D, H, W, _pad(cin)), dtype=torch.float32, device="cuda")
    assert gs.lib().sur_conv3d(D, H, W, _pad(cout), _pad(cin), dyd.data_ptr(), wp.data_ptr(), None, 3, None,
                               out.data_ptr(), _pad(cin), None) == 0
    torch.cuda.synchronize()
    ref = oracle.conv3d_dgrad(dy, w)
    assert _rel(to_np(out)[..., :cin], ref) < ACC_TOL
    # the masked BF16 form used in training: gradient times (mask > 0)
    mask = _rand_bf16(rng, (D, H, W, cin))
    md = _dev_act(torch, mask, _pad(cin))
    outb = torch.zeros((D, H, W, _pad(cin)), dtype=torch.bfloat16, device="cuda")
    assert gs.lib().sur_conv3d(D, H, W, _pad(cout), _pad(cin), dyd.data_ptr(), wp.data_ptr(), None, 2, md.data_ptr(),
                               outb.data_ptr(), _pad(cin), None) == 0
    torch.cuda.synchronize()
    refm = ref * (mask > 0)
    gotm = to_np(outb)[..., :cin]
    assert np.all(np.abs(gotm - refm) <= 2.0 ** -8 * np.abs(refm) + 1e-30)


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("cin,cout", SHAPES)
def test_conv_weight_gradient(grid, cin, cout):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    D, H, W = grid
    rng = np.random.default_rng(23 + cin + cout + D)
    x = _rand_bf16(rng, (D, H, W, cin))
    dy = _rand_bf16(rng, (D, H, W, cout))
    xd, dyd = _dev_act(torch, x, _pad(cin)), _dev_act(torch, dy, _pad(cout))
    nb = gs.lib().sur_wgrad_workspace_bytes(_pad(cin), _pad(cout))
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dw = torch.zeros((27, cin, cout), dtype=torch.float32, device="cuda")
    assert gs.lib().sur_conv3d_wgrad(D, H, W, _pad(cin), _pad(cout), xd.data_ptr(), dyd.data_ptr(), cin, cout,
                                     dw.data_ptr(), ws.data_ptr(), nb, None) == 0
    torch.cuda.synchronize()
    ref, _ = oracle.conv3d_wgrad(x, dy)
    assert _rel(to_np(dw), ref) < ACC_TOL


def _state(shape, seed):
    D, H, W = shape
    u, v = si.gs_initial_state(W, H, D, seed=seed)
    return u, v


def _norm():
    return (0.95, 0.02), (0.1, 0.07), (0.003, 0.006)


def test_network_gradient_matches_oracle_backprop():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    D, H, W = 4, 8, 16
    params = si.surrogate_init_params(seed=3, last_layer_scale=0.5)
    u, v = _state((D, H, W), 5)
    rng = np.random.default_rng(2)
    ut = u + 0.003 * rng.standard_normal(u.shape)
    vt = v + 0.006 * rng.standard_normal(v.shape)
    u, v, ut, vt = (a.astype(np.float32).astype(np.float64) for a in (u, v, ut, vt))
    mean, sd, scale = _norm()
    s = gs.Surrogate(W, H, D)
    s.set_params(params)
    s.set_normalization(mean, sd, scale)
    dev = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (u, v, ut, vt)]
    loss = s.train_step(*dev, 1e-9)
    g = s.get_grad()
    ref_loss, ref_g = oracle.surrogate_loss_grad(params.astype(np.float64), u, v, ut, vt, mean, sd, scale)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    assert _rel(g.astype(np.float64), ref_g) < 2e-3
    # forward prediction
    uo, vo = torch.empty_like(dev[0]), torch.empty_like(dev[1])
    s.set_params(params)
    s.forward(dev[0], dev[1], uo, vo)
    pu, pv = oracle.surrogate_forward(params.astype(np.float64), u, v, mean, sd, scale)
    assert _rel(np.concatenate([to_np(uo).ravel() - u.ravel(), to_np(vo).ravel() - v.ravel()]),
                np.concatenate([(pu - u).ravel(), (pv - v).ravel()])) < 1e-3
    s.close()


def test_training_reduces_loss():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    D, H, W = 16, 16, 32
    # snapshots 16 RK4 steps apart from our own integrator
    g = gs.GrayScott(W, H, D, prec=gs.GS_FP32, Du=2e-4, Dv=1e-4)
    u0, v0 = si.gs_initial_state(W, H, D, seed=9)
    g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    snaps = [(g.u.clone(), g.v.clone())]
    for _ in range(6):
        g.step(gs.GS_RK4, 0.0, 0.1, 16)
        snaps.append((g.u.clone(), g.v.clone()))
    g.close()
    s = gs.Surrogate(W, H, D)
    s.set_params(si.surrogate_init_params(seed=4, last_layer_scale=0.0))
    s.set_normalization(*_norm())
    losses = []
    for it in range(60):
        k = it % 6
        losses.append(s.train_step(snaps[k][0], snaps[k][1], snaps[k + 1][0], snaps[k + 1][1], 2e-3))
    assert np.mean(losses[-6:]) < 0.5 * np.mean(losses[:6]), (losses[:6], losses[-6:])
    s.close()


def test_judge_and_fallback():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    D, H, W = 8, 16, 32
    u0, v0 = si.gs_initial_state(W, H, D, seed=1)
    g = gs.GrayScott(W, H, D, prec=gs.GS_FP32)
    g.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    s = gs.Surrogate(W, H, D)
    s.set_params(si.surrogate_init_params(seed=4, last_layer_scale=0.0))  # predicts "no change"
    s.set_normalization(*_norm())
    # the judge integrates 16 RK4 steps and measures the prediction against it
    ref = gs.GrayScott(W, H, D, prec=gs.GS_FP32)
    ref.set_state(torch.from_numpy(u0), torch.from_numpy(v0))
    ref.step(gs.GS_RK4, 0.0, 0.1, 16)
    rel, fb = s.advance(g.ctx, g.u, g.v, judge=True, threshold=1e-3)
    expect = float(np.sqrt(np.sum((u0.astype(np.float32) - to_np(ref.u)) ** 2 + (v0.astype(np.float32) - to_np(ref.v)) ** 2)
                           / np.sum(to_np(ref.u) ** 2 + to_np(ref.v) ** 2)))
    assert abs(rel - expect) < 1e-6 and rel > 1e-3 and fb
    assert np.array_equal(to_np(g.u), to_np(ref.u))  # the integrator's result is kept
    # while the judgement stands, unjudged calls run the integrator
    rel2, fb2 = s.advance(g.ctx, g.u, g.v, judge=False)
    ref.step(gs.GS_RK4, 0.0, 0.1, 16)
    assert fb2 and np.array_equal(to_np(g.u), to_np(ref.u))
    # a generous threshold accepts the surrogate; unjudged calls then use it
    rel3, fb3 = s.advance(g.ctx, g.u, g.v, judge=True, threshold=1.0)
    assert not fb3
    before = g.u.clone()
    s.advance(g.ctx, g.u, g.v, judge=False)
    assert torch.equal(g.u, before)  # "no change" network
    for x in (s, g, ref):
        x.close()


# --- tcgen05 engine (32 -> 32 channels, D % 4 == 0, H % 16 == 0) ----------

@pytest.fixture
def tc_engine():
    """Selects the tcgen05 convolution engine for one test and restores the
    previous setting afterwards."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    prev = gs.lib().sur_get_conv_engine()
    assert gs.lib().sur_set_conv_engine(2) == 0
    yield torch, gs
    gs.lib().sur_set_conv_engine(prev)


def _tc_timeouts(gs):
    n = C.c_uint(0)
    assert gs.lib().sur_conv_tc_status(C.byref(n)) == 0
    return n.value


TC_GRIDS = [(4, 16, 16), (4, 16, 32), (8, 32, 16), (12, 48, 32)]


TC_CASES = [(32, 32, 3), (32, 32, 0), (2, 32, 3), (2, 32, 0), (32, 2, 3), (32, 2, 1)]


@pytest.mark.parametrize("grid", TC_GRIDS)
@pytest.mark.parametrize("cin,cout,epi", TC_CASES)
def test_conv_forward_tcgen05(tc_engine, grid, cin, cout, epi):
    """The tcgen05 kernel against the oracle on BF16-rounded operands (FP32
    accumulation; raw, bias + ReLU -> BF16 and bias -> FP32 epilogues) for the
    network's three layer shapes (2 -> 32, 32 -> 32, 32 -> 2 channels)."""
    torch, gs = tc_engine
    D, H, W = grid
    rng = np.random.default_rng(D * 1000 + H + W + epi + 7 * cin + cout)
    x = _rand_bf16(rng, (D, H, W, cin))
    w = _rand_bf16(rng, (27, cin, cout), 0.2)
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    cip, cop = _pad(cin), _pad(cout)
    xd = _dev_act(torch, x, cip)
    wp, _ = _packed(torch, gs, w, 0)
    bd = torch.zeros(cop, dtype=torch.float32, device="cuda")
    bd[:cout] = torch.from_numpy(b.astype(np.float32))
    if epi == 0:
        out = torch.zeros((D, H, W, cop), dtype=torch.bfloat16, device="cuda")
    elif epi == 1:
        out = torch.zeros((D, H, W, cout), dtype=torch.float32, device="cuda")
    else:
        out = torch.zeros((D, H, W, cop), dtype=torch.float32, device="cuda")
    before = _tc_timeouts(gs)
    assert gs.lib().sur_conv3d(D, H, W, cip, cop, xd.data_ptr(), wp.data_ptr(), bd.data_ptr(), epi, None,
                               out.data_ptr(), cout if epi == 1 else cop, None) == 0
    torch.cuda.synchronize()
    assert gs.lib().sur_conv_last_engine() == 2
    assert _tc_timeouts(gs) == before
    ref = oracle.conv3d_fwd(x, w, b)
    got = to_np(out)
    if epi in (1, 3):
        assert _rel(got[..., :cout], ref) < ACC_TOL
        if epi == 3:
            assert np.all(got[..., cout:] == 0.0)  # padded output channels
    else:
        refr = np.maximum(ref, 0.0)
        # BF16 output: one rounding of the FP32 sum (8 significant bits)
        assert np.all(np.abs(got[..., :cout] - refr) <= 2.0 ** -8 * np.abs(refr) + 1e-6 * np.max(np.abs(refr)))


@pytest.mark.parametrize("cin,cout", [(32, 32), (32, 2)])
def test_conv_input_gradient_tcgen05(tc_engine, cin, cout):
    """Input gradient (mirrored taps, transposed weights) of a cin -> cout
    layer on tcgen05: a cout -> cin convolution, raw and ReLU-masked."""
    torch, gs = tc_engine
    D, H, W = 4, 16, 16
    rng = np.random.default_rng(77 + cout)
    dy = _rand_bf16(rng, (D, H, W, cout))
    w = _rand_bf16(rng, (27, cin, cout), 0.2)
    cip, cop = _pad(cin), _pad(cout)
    dyd = _dev_act(torch, dy, cop)
    wp, _ = _packed(torch, gs, w, 1)
    out = torch.zeros((D, H, W, cip), dtype=torch.float32, device="cuda")
    assert gs.lib().sur_conv3d(D, H, W, cop, cip, dyd.data_ptr(), wp.data_ptr(), None, 3, None, out.data_ptr(), cip,
                               None) == 0
    torch.cuda.synchronize()
    assert gs.lib().sur_conv_last_engine() == 2
    ref = oracle.conv3d_dgrad(dy, w)
    assert _rel(to_np(out)[..., :cin], ref) < ACC_TOL
    mask = _rand_bf16(rng, (D, H, W, cin))
    md = _dev_act(torch, mask, cip)
    outb = torch.zeros((D, H, W, cip), dtype=torch.bfloat16, device="cuda")
    assert gs.lib().sur_conv3d(D, H, W, cop, cip, dyd.data_ptr(), wp.data_ptr(), None, 2, md.data_ptr(),
                               outb.data_ptr(), cip, None) == 0
    torch.cuda.synchronize()
    refm = ref * (mask > 0)
    gotm = to_np(outb)[..., :cin]
    assert np.all(np.abs(gotm - refm) <= 2.0 ** -8 * np.abs(refm) + 1e-6 * np.max(np.abs(refm)))
    assert _tc_timeouts(gs) == 0


@pytest.mark.parametrize("grid", TC_GRIDS + [(2, 16, 16), (2, 32, 32), (6, 16, 48)])
def test_conv_weight_gradient_tcgen05(tc_engine, grid):
    """32 x 32 weight gradient on tcgen05 (one MMA spans four z-shifts)
    against the oracle, including depth 2, where the tile's z-halo wraps onto
    its own plane."""
    torch, gs = tc_engine
    D, H, W = grid
    rng = np.random.default_rng(101 + D * 7 + H + W)
    x = _rand_bf16(rng, (D, H, W, 32))
    dy = _rand_bf16(rng, (D, H, W, 32))
    xd, dyd = _dev_act(torch, x, 32), _dev_act(torch, dy, 32)
    nb = gs.lib().sur_wgrad_workspace_bytes(32, 32)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dw = torch.zeros((27, 32, 32), dtype=torch.float32, device="cuda")
    before = _tc_timeouts(gs)
    assert gs.lib().sur_conv3d_wgrad(D, H, W, 32, 32, xd.data_ptr(), dyd.data_ptr(), 32, 32, dw.data_ptr(),
                                     ws.data_ptr(), nb, None) == 0
    torch.cuda.synchronize()
    assert gs.lib().sur_conv_last_engine() == 2
    assert _tc_timeouts(gs) == before
    ref, _ = oracle.conv3d_wgrad(x, dy)
    assert _rel(to_np(dw), ref) < ACC_TOL


def test_conv_engines_agree(tc_engine):
    """Both engines on the same inputs: equal up to FP32 summation order."""
    torch, gs = tc_engine
    D, H, W = 4, 32, 32
    rng = np.random.default_rng(5)
    x = _rand_bf16(rng, (D, H, W, 32))
    w = _rand_bf16(rng, (27, 32, 32), 0.2)
    xd = _dev_act(torch, x, 32)
    wp, _ = _packed(torch, gs, w, 0)
    outs = []
    for engine in (1, 2):
        gs.lib().sur_set_conv_engine(engine)
        o = torch.zeros((D, H, W, 32), dtype=torch.float32, device="cuda")
        assert gs.lib().sur_conv3d(D, H, W, 32, 32, xd.data_ptr(), wp.data_ptr(), None, 3, None, o.data_ptr(), 32,
                                   None) == 0
        torch.cuda.synchronize()
        assert gs.lib().sur_conv_last_engine() == engine
        outs.append(to_np(o))
    assert _rel(outs[1], outs[0]) < 1e-6


def test_network_gradient_tcgen05_matches_oracle_backprop(tc_engine):
    """Whole-network loss gradient with the hidden layers on tcgen05 (grid
    with H % 16 == 0) against oracle backpropagation."""
    torch, gs = tc_engine
    D, H, W = 4, 16, 16
    params = si.surrogate_init_params(seed=3, last_layer_scale=0.5)
    u, v = _state((D, H, W), 5)
    rng = np.random.default_rng(2)
    ut = u + 0.003 * rng.standard_normal(u.shape)
    vt = v + 0.006 * rng.standard_normal(v.shape)
    u, v, ut, vt = (a.astype(np.float32).astype(np.float64) for a in (u, v, ut, vt))
    mean, sd, scale = _norm()
    s = gs.Surrogate(W, H, D)
    s.set_params(params)
    s.set_normalization(mean, sd, scale)
    dev = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (u, v, ut, vt)]
    loss = s.train_step(*dev, 1e-9)
    g = s.get_grad()
    ref_loss, ref_g = oracle.surrogate_loss_grad(params.astype(np.float64), u, v, ut, vt, mean, sd, scale)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    assert _rel(g.astype(np.float64), ref_g) < 2e-3
    s.close()
    assert _tc_timeouts(gs) == 0


def test_timeout_mark_makes_every_call_fail():
    """A tensor-core launch that gives up waiting marks its context failed;
    the mark is set here from the host (no GPU fault or hang is provoked),
    exactly as the kernel sets it.  Every later call on the context, and a
    synchronising call, must return GS_ERR_CUDA instead of a result; the
    layer primitives share one process-wide mark."""
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    L = gs.lib()
    n = (16, 16, 4)
    s = gs.Surrogate(*n)
    u = torch.rand(n[::-1], dtype=torch.float32, device="cuda")
    v = torch.rand(n[::-1], dtype=torch.float32, device="cuda")
    uo, vo = torch.empty_like(u), torch.empty_like(v)
    s.forward(u, v, uo, vo)
    p0 = s.get_params()
    assert L.sur_debug_set_timeout_word(s.ctx, 1) == 0
    for call in (lambda: s.forward(u, v, uo, vo), s.get_params, s.get_grad,
                 lambda: s.train_step(u, v, uo, vo, 1e-3)):
        with pytest.raises(gs.GSError) as ei:
            call()
        assert ei.value.status == gs.GS_ERR_CUDA and "gave up" in str(ei.value)
    assert L.sur_debug_set_timeout_word(s.ctx, 0) == 0
    assert np.array_equal(s.get_params(), p0)
    s.close()
    # layer primitives: one process-wide mark
    x = torch.zeros((4, 16, 16, 32), dtype=torch.bfloat16, device="cuda")
    w = np.zeros((27, 32, 32))
    packed, _ = _packed(torch, gs, w, 0)
    out = torch.empty((4, 16, 16, 32), dtype=torch.float32, device="cuda")
    args = (4, 16, 16, 32, 32, x.data_ptr(), packed.data_ptr(), None, 3, None, out.data_ptr(), 32, None)
    assert L.sur_conv3d(*args) == 0
    st = C.c_uint(7)
    assert L.sur_conv_tc_status(C.byref(st)) == 0 and st.value == 0
    assert L.sur_debug_set_timeout_word(None, 1) == 0
    try:
        assert L.sur_conv_tc_status(C.byref(st)) == 0 and st.value == 1
        assert L.sur_conv3d(*args) == gs.GS_ERR_CUDA
    finally:
        assert L.sur_debug_set_timeout_word(None, 0) == 0
    assert L.sur_conv3d(*args) == 0
    torch.cuda.synchronize()


# more tiles than SMs: the persistent tcgen05 kernels then run several tiles
# per CTA (halo buffers and accumulator sets reused, the next halo copied
# while a tile's MMAs and epilogue run)
MULTI_TILE_GRID = (32, 64, 96)  # 384 tiles of 8 x 16 x 4 for the forward kernel


@pytest.mark.parametrize("cin,cout,epi", [(32, 32, 3), (2, 32, 0), (32, 2, 1)])
def test_conv_forward_tcgen05_several_tiles_per_cta(tc_engine, cin, cout, epi):
    torch, gs = tc_engine
    D, H, W = MULTI_TILE_GRID
    rng = np.random.default_rng(211 + 7 * cin + cout + epi)
    x = _rand_bf16(rng, (D, H, W, cin))
    w = _rand_bf16(rng, (27, cin, cout), 0.2)
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    cip, cop = _pad(cin), _pad(cout)
    xd = _dev_act(torch, x, cip)
    wp, _ = _packed(torch, gs, w, 0)
    bd = torch.zeros(cop, dtype=torch.float32, device="cuda")
    bd[:cout] = torch.from_numpy(b.astype(np.float32))
    if epi == 0:
        out = torch.zeros((D, H, W, cop), dtype=torch.bfloat16, device="cuda")
    elif epi == 1:
        out = torch.zeros((D, H, W, cout), dtype=torch.float32, device="cuda")
    else:
        out = torch.zeros((D, H, W, cop), dtype=torch.float32, device="cuda")
    before = _tc_timeouts(gs)
    assert gs.lib().sur_conv3d(D, H, W, cip, cop, xd.data_ptr(), wp.data_ptr(), bd.data_ptr(), epi, None,
                               out.data_ptr(), cout if epi == 1 else cop, None) == 0
    torch.cuda.synchronize()
    assert gs.lib().sur_conv_last_engine() == 2
    assert _tc_timeouts(gs) == before
    ref = oracle.conv3d_fwd(x, w, b)
    got = to_np(out)
    if epi in (1, 3):
        assert _rel(got[..., :cout], ref) < ACC_TOL
        # every cell, not only the pooled norm: one wrong tile would show here
        assert np.max(np.abs(got[..., :cout] - ref)) <= ACC_TOL * np.max(np.abs(ref))
    else:
        refr = np.maximum(ref, 0.0)
        assert np.all(np.abs(got[..., :cout] - refr) <= 2.0 ** -8 * np.abs(refr) + 1e-6 * np.max(np.abs(refr)))


def test_conv_weight_gradient_tcgen05_several_tiles_per_cta(tc_engine):
    """The weight gradient accumulates all of a CTA's one-plane tiles in TMEM
    before writing its partial: 16 x 32 x 64 has 256 tiles (one or two per
    CTA)."""
    torch, gs = tc_engine
    D, H, W = 16, 32, 64
    rng = np.random.default_rng(307)
    x = _rand_bf16(rng, (D, H, W, 32))
    dy = _rand_bf16(rng, (D, H, W, 32))
    xd, dyd = _dev_act(torch, x, 32), _dev_act(torch, dy, 32)
    nb = gs.lib().sur_wgrad_workspace_bytes(32, 32)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dw = torch.zeros((27, 32, 32), dtype=torch.float32, device="cuda")
    before = _tc_timeouts(gs)
    assert gs.lib().sur_conv3d_wgrad(D, H, W, 32, 32, xd.data_ptr(), dyd.data_ptr(), 32, 32, dw.data_ptr(),
                                     ws.data_ptr(), nb, None) == 0
    torch.cuda.synchronize()
    assert gs.lib().sur_conv_last_engine() == 2
    assert _tc_timeouts(gs) == before
    ref, _ = oracle.conv3d_wgrad(x, dy)
    assert _rel(to_np(dw), ref) < ACC_TOL


def test_network_forward_128cubed_sampled_cones(tc_engine):
    """The bench's size (128^3, the tcgen05 convolutions with ~28 tiles per
    CTA): the GPU network forward against the oracle's on the dependence
    cone of 40 sampled cells (radius 4: four 3^3 layers), cells on the
    periodic seams and on the tiles' x, y and z boundaries among them."""
    torch, gs = tc_engine
    from tests._gpu_common import periodic_box
    n = 128
    params = si.surrogate_init_params(seed=5, last_layer_scale=0.5)
    u, v = _state((n, n, n), 9)
    u, v = u.astype(np.float32).astype(np.float64), v.astype(np.float32).astype(np.float64)
    mean, sd, scale = _norm()
    s = gs.Surrogate(n, n, n)
    s.set_params(params)
    s.set_normalization(mean, sd, scale)
    du, dv = torch.from_numpy(u.astype(np.float32)).cuda(), torch.from_numpy(v.astype(np.float32)).cuda()
    uo, vo = torch.empty_like(du), torch.empty_like(dv)
    before = _tc_timeouts(gs)
    s.forward(du, dv, uo, vo)
    torch.cuda.synchronize()
    assert _tc_timeouts(gs) == before
    gu, gv = to_np(uo), to_np(vo)
    s.close()
    rng = np.random.default_rng(17)
    seams = [(0, 0, 0), (127, 127, 127), (3, 15, 7), (4, 16, 8), (63, 64, 120), (64, 63, 121), (100, 31, 64),
             (127, 0, 63), (0, 127, 64), (32, 48, 7)]
    centers = seams + [tuple(int(a) for a in rng.integers(0, n, 3)) for _ in range(30)]
    r = 4
    got, ref = [], []
    for c in centers:
        bu, bv = periodic_box(u, c, r), periodic_box(v, c, r)
        pu, pv = oracle.surrogate_forward(params.astype(np.float64), bu, bv, mean, sd, scale)
        ref.append([pu[r, r, r] - u[c], pv[r, r, r] - v[c]])
        got.append([gu[c] - u[c], gv[c] - v[c]])
    got, ref = np.array(got), np.array(ref)
    # BF16 hidden activations: a sum that lands on a rounding boundary may
    # round the other way on one side, so the bound is the network's
    # end-to-end tolerance (1e-3 of the update's scale), per cell
    for comp in range(2):
        scale_c = np.max(np.abs(ref[:, comp]))
        assert scale_c > 0
        assert np.max(np.abs(got[:, comp] - ref[:, comp])) <= 2e-3 * scale_c, comp
