"""Python binding of libgs_b300 (C ABI in include/gs.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device arrays are PyTorch CUDA tensors (contiguous, 16-byte
aligned); streams default to PyTorch's current stream.  There is no CPU
fallback: if the shared library is missing or no CUDA device is present the
calls raise.

The functions keep the C names (gs_create, gs_step, gs_integrate_adaptive,
ode_axpy_stage, ...); ``GrayScott`` is a small owner of one gs_ctx.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs_b300.so")

GS_OK, GS_ERR_INVALID, GS_ERR_CUDA, GS_ERR_NOMEM = 0, 1, 2, 3
GS_ERR_STEP_UNDERFLOW, GS_ERR_MAX_STEPS, GS_ERR_NONFINITE = 4, 5, 6
GS_FP64, GS_FP32 = 0, 1
GS_RK4, GS_DOPRI5, GS_AB4, GS_EULER, GS_CK54, GS_RKF78, GS_MIDPOINT = 0, 1, 2, 3, 4, 5, 6
ODE_EXP_DECAY, ODE_LOGISTIC = 0, 1

STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID", 2: "GS_ERR_CUDA", 3: "GS_ERR_NOMEM",
                4: "GS_ERR_STEP_UNDERFLOW", 5: "GS_ERR_MAX_STEPS", 6: "GS_ERR_NONFINITE"}


class GSError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)} {msg}".strip())


class gs_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("Du", C.c_double), ("Dv", C.c_double), ("F", C.c_double), ("k", C.c_double),
                ("prec", C.c_int)]


class gsb_instance(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("F", C.c_double), ("k", C.c_double)]


_lib = None
_vp, _dp, _lp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_long)
# int (*gs_observer)(double t, void* u, void* v, void* user)
GS_OBSERVER = C.CFUNCTYPE(C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p)

_SIGNATURES = {
    "gs_create": ([C.POINTER(gs_params), _vp, C.POINTER(_vp)], C.c_int),
    "gs_destroy": ([_vp], C.c_int),
    "gs_bind_state": ([_vp, _vp, _vp], C.c_int),
    "gs_upload_state": ([_vp, _vp, _vp], C.c_int),
    "gs_download_state": ([_vp, _vp, _vp], C.c_int),
    "gs_rhs": ([_vp, C.c_double, _vp, _vp, _vp, _vp], C.c_int),
    "gs_step": ([_vp, C.c_int, _dp, C.c_double, C.c_long], C.c_int),
    "gs_integrate_adaptive": ([_vp, C.c_double, C.c_double, _dp, C.c_double, _dp, C.c_long, _lp, _lp], C.c_int),
    "gs_integrate_adaptive_pair": ([_vp, C.c_int, C.c_double, C.c_double, _dp, C.c_double, _dp, C.c_long, _lp,
                                    _lp], C.c_int),
    "gs_set_step_log": ([_vp, C.c_long], C.c_int),
    "gs_get_step_log": ([_vp, _dp, C.c_long, _lp], C.c_int),
    "gs_set_tile": ([_vp, C.c_int, C.c_int], C.c_int),
    "gs_set_kernel_variant": ([_vp, C.c_int], C.c_int),
    "gs_get_kernel_variant": ([_vp, C.POINTER(C.c_int)], C.c_int),
    "gs_get_stage_configs": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "gs_set_stage_depth": ([_vp, C.c_int], C.c_int),
    "gs_set_dopri5_split": ([_vp, C.c_int], C.c_int),
    "gs_set_small_grid_path": ([_vp, C.c_int, C.c_int], C.c_int),
    "gs_get_small_grid_path": ([_vp], C.c_int),
    "gs_get_dopri5_split": ([_vp], C.c_int),
    "gs_set_dopri5_fusion": ([_vp, C.c_int], C.c_int),
    "gs_get_dopri5_fusion": ([_vp], C.c_int),
    "gs_get_rk4_fusion": ([_vp], C.c_int),
    "gs_set_pair_config": ([_vp, C.c_int, C.c_int, C.c_int], C.c_int),
    "gs_get_pair_configs": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "gs_time_pairs": ([_vp, C.c_int, _dp], C.c_int),
    "gs_set_laplacian": ([_vp, C.c_int, C.c_double], C.c_int),
    "gs_get_dcpse_stencil": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp, C.c_int], C.c_int),
    "gs_set_dcpse_tile": ([_vp, C.c_int], C.c_int),
    "gs_set_observer": ([_vp, GS_OBSERVER, _vp], C.c_int),
    "gs_get_pair_depths_in_use": ([_vp, C.POINTER(C.c_int)], C.c_int),
    "gs_get_stage_depths": ([_vp, C.POINTER(C.c_int)], C.c_int),
    "gs_get_tile": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "gs_autotune": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp], C.c_int),
    "gs_time_stages": ([_vp, C.c_int, _dp], C.c_int),
    "gs_last_error": ([_vp], C.c_char_p),
    "gs_last_global_error": ([], C.c_char_p),
    "ode_axpy_stage": ([C.c_long, C.c_int, C.c_int, _dp, C.POINTER(_vp), _vp, _vp], C.c_int),
    "ode_workspace_size": ([C.c_long], C.c_size_t),
    "ode_integrate_adaptive": ([C.c_int, C.c_long, _vp, _dp, C.c_double, _dp, C.c_double, C.c_double,
                                C.c_long, _lp, _lp, _vp, C.c_size_t, _vp, C.c_long, _vp], C.c_int),
    "ode_integrate_adaptive_noalloc": ([C.c_int, C.c_long, _vp, _dp, C.c_double, _dp, C.c_double, C.c_double,
                                        C.c_long, _lp, _lp, _vp], C.c_int),
    "ode_integrate_ab4": ([C.c_int, C.c_long, _vp, C.c_double, C.c_double, C.c_long, _vp], C.c_int),
    "ode_integrate_const": ([C.c_int, C.c_int, C.c_long, _vp, C.c_double, C.c_double, C.c_long, _vp], C.c_int),
    "ode_integrate_tableau": ([C.c_int, C.c_int, C.c_long, _vp, _vp, C.c_double, C.c_double, C.c_long, _vp],
                              C.c_int),
    "ode_integrate_ab_steps": ([C.c_int, C.c_int, C.c_long, _vp, _vp, C.c_double, C.c_double, C.c_long, _vp],
                               C.c_int),
    "ode_integrate_abm_steps": ([C.c_int, C.c_int, C.c_long, _vp, _vp, C.c_double, C.c_double, C.c_long, _vp],
                                C.c_int),
    "ode_am_weights": ([C.c_int, _dp], C.c_int),
    "ode_integrate_adaptive_each": ([C.c_int, C.c_int, C.c_long, _vp, _vp, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_long, C.c_long, _vp, _vp, _vp, _vp, _vp, _vp],
                                    C.c_int),
    "gs_measure_fp64_peak": ([_dp, _vp], C.c_int),
    "gsb_create": ([C.c_int, C.POINTER(gsb_instance), C.c_double, C.c_double, C.c_double, C.c_int, _vp,
                    C.POINTER(_vp)], C.c_int),
    "gsb_destroy": ([_vp], C.c_int),
    "gsb_layout": ([_vp, C.POINTER(C.c_longlong)], C.c_int),
    "gsb_bind_state": ([_vp, _vp, _vp], C.c_int),
    "gsb_integrate_adaptive": ([_vp, C.c_double, C.c_double, _dp, C.c_double, _dp, C.c_long, _lp, _lp,
                                C.POINTER(C.c_int)], C.c_int),
    "gsb_set_tile": ([_vp, C.c_int, C.c_int], C.c_int),
    "gsb_set_grouping": ([_vp, C.c_longlong], C.c_int),
    "gsb_set_pairs": ([_vp, C.c_int, C.c_int, C.c_int], C.c_int),
    "gsb_get_pairs": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "gsb_set_pair_lanes": ([_vp, C.c_int, C.c_int], C.c_int),
    "gsb_get_pair_lanes": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "gsb_set_stage_depth": ([_vp, C.c_int], C.c_int),
    "gsb_get_grouping": ([_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int)], C.c_int),
    "gsb_autotune": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp], C.c_int),
    "gsb_autotune_run": ([_vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int),
                          C.POINTER(C.c_int), _dp], C.c_int),
    "gsb_last_error": ([_vp], C.c_char_p),
    "gsb_set_step_log": ([_vp, C.c_long], C.c_int),
    "gsb_get_step_log": ([_vp, _dp, C.c_long, _lp], C.c_int),
    "sur_param_count": ([], C.c_long),
    "sur_create": ([C.c_int, C.c_int, C.c_int, _vp, C.POINTER(_vp)], C.c_int),
    "sur_destroy": ([_vp], C.c_int),
    "sur_set_params": ([_vp, C.POINTER(C.c_float)], C.c_int),
    "sur_get_params": ([_vp, C.POINTER(C.c_float)], C.c_int),
    "sur_get_grad": ([_vp, C.POINTER(C.c_float)], C.c_int),
    "sur_set_normalization": ([_vp, _dp, _dp, _dp], C.c_int),
    "sur_forward": ([_vp, _vp, _vp, _vp, _vp], C.c_int),
    "sur_train_step": ([_vp, _vp, _vp, _vp, _vp, C.c_double, _dp], C.c_int),
    "sur_advance": ([_vp, _vp, _vp, _vp, C.c_int, C.c_double, _dp, C.POINTER(C.c_int)], C.c_int),
    "sur_last_error": ([_vp], C.c_char_p),
    "sur_packed_bytes": ([C.c_int, C.c_int], C.c_size_t),
    "sur_pack_weights": ([C.c_int, C.c_int, _vp, C.c_int, _vp, _vp], C.c_int),
    "sur_set_conv_engine": ([C.c_int], C.c_int),
    "sur_get_conv_engine": ([], C.c_int),
    "sur_conv_last_engine": ([], C.c_int),
    "sur_conv_tc_status": ([C.POINTER(C.c_uint)], C.c_int),
    "sur_debug_set_timeout_word": ([_vp, C.c_uint], C.c_int),
    "sur_conv3d": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, C.c_int, _vp, _vp, C.c_int, _vp],
                   C.c_int),
    "sur_wgrad_workspace_bytes": ([C.c_int, C.c_int], C.c_size_t),
    "sur_conv3d_wgrad": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp,
                          C.c_size_t, _vp], C.c_int),
    "sur_moments": ([C.c_long, _vp, _vp, _vp], C.c_int),
}


def lib():
    """Loads libgs_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2309_05331_b300.build`")
    import torch  # noqa: F401  -- load PyTorch's CUDA runtime first so both share it
    L = C.CDLL(LIB_PATH)
    for name, (args, res) in _SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_names():
    """Names the binding expects the library to export."""
    return list(_SIGNATURES)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _check(st, ctx=None):
    if st != GS_OK:
        L = lib()
        msg = (L.gs_last_error(ctx) if ctx else L.gs_last_global_error()) or b""
        raise GSError(st, msg.decode())


# --------------------------------------------------------------------------
# Same-named thin wrappers of the C ABI
# --------------------------------------------------------------------------
def gs_create(nx, ny, nz, L=2.5, Du=2e-5, Dv=1e-5, F=0.053, k=0.014, prec=GS_FP64, Ly=None, Lz=None,
              stream=None):
    p = gs_params(nx, ny, nz, L, L if Ly is None else Ly, L if Lz is None else Lz, Du, Dv, F, k, prec)
    ctx = _vp()
    _check(lib().gs_create(C.byref(p), _stream(stream), C.byref(ctx)))
    return ctx


def gs_destroy(ctx):
    return lib().gs_destroy(ctx)


def gs_bind_state(ctx, u, v):
    _check(lib().gs_bind_state(ctx, _ptr(u), _ptr(v)), ctx)


def gs_upload_state(ctx, u_host, v_host):
    _check(lib().gs_upload_state(ctx, u_host.data_ptr(), v_host.data_ptr()), ctx)


def gs_download_state(ctx, u_host, v_host):
    _check(lib().gs_download_state(ctx, u_host.data_ptr(), v_host.data_ptr()), ctx)


def gs_rhs(ctx, t, u, v, fu, fv):
    _check(lib().gs_rhs(ctx, t, _ptr(u), _ptr(v), _ptr(fu), _ptr(fv)), ctx)


def gs_step(ctx, method, t, dt, nsteps):
    tt = C.c_double(t)
    _check(lib().gs_step(ctx, method, C.byref(tt), dt, nsteps), ctx)
    return tt.value


def gs_integrate_adaptive(ctx, atol, rtol, t, t_end, dt, max_accepted=-1, check=True):
    tt, dd = C.c_double(t), C.c_double(dt)
    na, nr = C.c_long(0), C.c_long(0)
    st = lib().gs_integrate_adaptive(ctx, atol, rtol, C.byref(tt), t_end, C.byref(dd), max_accepted,
                                     C.byref(na), C.byref(nr))
    if check:
        _check(st, ctx)
    return {"status": st, "t": tt.value, "dt": dd.value, "n_acc": na.value, "n_rej": nr.value}


def gs_integrate_adaptive_pair(ctx, pair, atol, rtol, t, t_end, dt, max_accepted=-1, check=True):
    tt, dd = C.c_double(t), C.c_double(dt)
    na, nr = C.c_long(0), C.c_long(0)
    st = lib().gs_integrate_adaptive_pair(ctx, pair, atol, rtol, C.byref(tt), t_end, C.byref(dd), max_accepted,
                                          C.byref(na), C.byref(nr))
    if check:
        _check(st, ctx)
    return {"status": st, "t": tt.value, "dt": dd.value, "n_acc": na.value, "n_rej": nr.value}


def gs_set_step_log(ctx, capacity):
    _check(lib().gs_set_step_log(ctx, capacity), ctx)


def gs_get_step_log(ctx, capacity):
    import numpy as np
    buf = np.zeros(max(capacity, 1))
    cnt = C.c_long(0)
    _check(lib().gs_get_step_log(ctx, buf.ctypes.data_as(_dp), capacity, C.byref(cnt)), ctx)
    return buf[: min(cnt.value, capacity)].copy(), cnt.value


def gs_set_tile(ctx, ty, zc):
    _check(lib().gs_set_tile(ctx, ty, zc), ctx)


def gs_set_kernel_variant(ctx, variant):
    _check(lib().gs_set_kernel_variant(ctx, variant), ctx)


def gs_get_kernel_variant(ctx):
    v = C.c_int(0)
    _check(lib().gs_get_kernel_variant(ctx, C.byref(v)), ctx)
    return v.value


def gs_get_stage_configs(ctx):
    """[(form, ty, zc)] of the Dormand-Prince kernels k1, stage 2..7."""
    f, t, z = (C.c_int * 7)(), (C.c_int * 7)(), (C.c_int * 7)()
    _check(lib().gs_get_stage_configs(ctx, f, t, z), ctx)
    return [(f[i], t[i], z[i]) for i in range(7)]


def gs_set_small_grid_path(ctx, mode, ctas=0):
    _check(lib().gs_set_small_grid_path(ctx, mode, ctas), ctx)


def gs_get_small_grid_path(ctx):
    return lib().gs_get_small_grid_path(ctx)


def gs_set_dopri5_split(ctx, mode):
    _check(lib().gs_set_dopri5_split(ctx, mode), ctx)


def gs_get_dopri5_split(ctx):
    return lib().gs_get_dopri5_split(ctx)


def gs_set_dopri5_fusion(ctx, mode):
    _check(lib().gs_set_dopri5_fusion(ctx, mode), ctx)


def gs_get_dopri5_fusion(ctx):
    return lib().gs_get_dopri5_fusion(ctx)


def gs_set_pair_config(ctx, pair, ty, depth):
    _check(lib().gs_set_pair_config(ctx, pair, ty, depth), ctx)


def gs_get_rk4_fusion(ctx):
    return lib().gs_get_rk4_fusion(ctx)


def gs_get_pair_configs(ctx):
    """(tile height, ring depth) of the pair kernels: Dormand-Prince stages
    2+3, 4+5, 6+7, RK4 stages 1+2, 3+4."""
    t = (C.c_int * 5)()
    d = (C.c_int * 5)()
    _check(lib().gs_get_pair_configs(ctx, t, d), ctx)
    return [(t[i], d[i]) for i in range(5)]


def gs_get_pair_depths_in_use(ctx):
    """Ring depth each pair kernel launches with (configured depth cut to what shared memory holds)."""
    d = (C.c_int * 5)()
    _check(lib().gs_get_pair_depths_in_use(ctx, d), ctx)
    return list(d)


GS_LAP_7POINT, GS_LAP_DCPSE = 0, 1


def gs_set_laplacian(ctx, kind, rc_over_h=3.1):
    _check(lib().gs_set_laplacian(ctx, kind, rc_over_h), ctx)


def gs_set_observer(ctx, fn):
    """Installs fn(t, u_ptr, v_ptr) -> bool (True stops) as ctx's observer, or
    removes it (fn None).  Returns the ctypes callback, which the caller must
    keep alive while it is installed."""
    if fn is None:
        _check(lib().gs_set_observer(ctx, C.cast(None, GS_OBSERVER), None), ctx)
        return None
    cb = GS_OBSERVER(lambda t, u, v, user: 1 if fn(t, u, v) else 0)
    _check(lib().gs_set_observer(ctx, cb, None), ctx)
    return cb


def gs_set_dcpse_tile(ctx, tz):
    _check(lib().gs_set_dcpse_tile(ctx, tz), ctx)


def gs_get_dcpse_stencil(ctx):
    """(offsets [m, 3] in spacings, weights [m]) of the DC-PSE stencil in use."""
    import numpy as np
    m = C.c_int(0)
    _check(lib().gs_get_dcpse_stencil(ctx, C.byref(m), None, None, 0), ctx)
    off = (C.c_int * (3 * m.value))()
    w = np.zeros(m.value)
    _check(lib().gs_get_dcpse_stencil(ctx, C.byref(m), off, w.ctypes.data_as(_dp), m.value), ctx)
    return np.array(off[:], dtype=np.int64).reshape(-1, 3), w


def gs_time_pairs(ctx, reps=5):
    """Average durations (ms) of the k1 kernel and the three Dormand-Prince pair kernels."""
    ms = (C.c_double * 4)()
    _check(lib().gs_time_pairs(ctx, reps, ms), ctx)
    return list(ms)


def gs_set_stage_depth(ctx, depth):
    _check(lib().gs_set_stage_depth(ctx, depth), ctx)


def gs_get_stage_depths(ctx):
    """Ring depth of the staged form for k1 and stages 2..7."""
    d = (C.c_int * 7)()
    _check(lib().gs_get_stage_depths(ctx, d), ctx)
    return list(d)


def gs_get_tile(ctx):
    a, b = C.c_int(0), C.c_int(0)
    _check(lib().gs_get_tile(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def gs_autotune(ctx):
    a, b, ms = C.c_int(0), C.c_int(0), C.c_double(0)
    _check(lib().gs_autotune(ctx, C.byref(a), C.byref(b), C.byref(ms)), ctx)
    return a.value, b.value, ms.value


def gs_time_stages(ctx, reps=5):
    """Average durations (ms) of the k1 kernel and Dormand-Prince stages 2..7."""
    ms = (C.c_double * 7)()
    _check(lib().gs_time_stages(ctx, reps, ms), ctx)
    return list(ms)


def ode_axpy_stage(coef, xs, y, stream=None):
    """y = sum_j coef[j] * xs[j] on the GPU (1..15 operands, same dtype)."""
    import torch
    if y.dtype not in (torch.float32, torch.float64) or any(x.dtype != y.dtype for x in xs):
        raise ValueError("operands must all be float32 or all float64")
    if any(x.numel() != y.numel() for x in xs):
        raise ValueError("operand sizes differ")
    prec = GS_FP64 if y.dtype == torch.float64 else GS_FP32
    c = (C.c_double * len(xs))(*[float(a) for a in coef])
    ptrs = (_vp * len(xs))(*[_ptr(x) for x in xs])
    _check(lib().ode_axpy_stage(y.numel(), prec, len(xs), c, ptrs, _ptr(y), _stream(stream)))


def ode_workspace_size(n):
    return lib().ode_workspace_size(n)


def ode_integrate_adaptive(kind, x, t, t_end, dt, atol, rtol, max_steps=-1, workspace=None, dt_log=None,
                           stream=None, check=True):
    import torch
    n = x.numel()
    if workspace is None:
        workspace = torch.empty(ode_workspace_size(n), dtype=torch.uint8, device=x.device)
    tt, dd = C.c_double(t), C.c_double(dt)
    na, nr = C.c_long(0), C.c_long(0)
    st = lib().ode_integrate_adaptive(kind, n, _ptr(x), C.byref(tt), t_end, C.byref(dd), atol, rtol, max_steps,
                                      C.byref(na), C.byref(nr), _ptr(workspace), workspace.numel(),
                                      _ptr(dt_log), 0 if dt_log is None else dt_log.numel(), _stream(stream))
    if check:
        _check(st)
    return {"status": st, "t": tt.value, "dt": dd.value, "n_acc": na.value, "n_rej": nr.value}


def ode_integrate_adaptive_noalloc(kind, x, t, t_end, dt, atol, rtol, max_steps=-1, stream=None, check=True):
    """ode_integrate_adaptive without a workspace (static scratch, n <= 2^20)."""
    tt, dd = C.c_double(t), C.c_double(dt)
    na, nr = C.c_long(0), C.c_long(0)
    st = lib().ode_integrate_adaptive_noalloc(kind, x.numel(), _ptr(x), C.byref(tt), t_end, C.byref(dd), atol,
                                              rtol, max_steps, C.byref(na), C.byref(nr), _stream(stream))
    if check:
        _check(st)
    return {"status": st, "t": tt.value, "dt": dd.value, "n_acc": na.value, "n_rej": nr.value}


def ode_integrate_ab4(kind, x, t0, dt, nsteps, stream=None):
    _check(lib().ode_integrate_ab4(kind, x.numel(), _ptr(x), t0, dt, nsteps, _stream(stream)))


def ode_integrate_const(kind, method, x, t0, dt, nsteps, stream=None):
    _check(lib().ode_integrate_const(kind, method, x.numel(), _ptr(x), t0, dt, nsteps, _stream(stream)))


ODE_PAPER_EXP, ODE_PAPER_SIGMOID = 2, 3
ODE_TAB_EULER, ODE_TAB_RK4, ODE_TAB_DOPRI5, ODE_TAB_CK54, ODE_TAB_RKF78, ODE_TAB_MIDPOINT = 0, 1, 2, 3, 4, 5


def ode_integrate_tableau(kind, method, x, t0, dt, nsteps, coef=None, stream=None):
    """Fixed steps of a Table 1 tableau on x (FP64 CUDA tensor), in place."""
    _check(lib().ode_integrate_tableau(kind, method, x.numel(), _ptr(x), _ptr(coef), t0, dt, nsteps,
                                       _stream(stream)))


def ode_integrate_ab_steps(kind, steps, x, t0, dt, nsteps, coef=None, stream=None):
    """Adams-Bashforth with `steps` (1..8) steps on x, in place."""
    _check(lib().ode_integrate_ab_steps(kind, steps, x.numel(), _ptr(x), _ptr(coef), t0, dt, nsteps,
                                        _stream(stream)))


def ode_integrate_abm_steps(kind, steps, x, t0, dt, nsteps, coef=None, stream=None):
    _check(lib().ode_integrate_abm_steps(kind, steps, x.numel(), _ptr(x), _ptr(coef), t0, dt, nsteps,
                                         _stream(stream)))


def ode_am_weights(steps):
    import numpy as np
    w = np.zeros(max(steps, 1))
    _check(lib().ode_am_weights(steps, w.ctypes.data_as(_dp)))
    return w[:steps]


def ode_integrate_adaptive_each(kind, method, x, t0, t_end, dt0, atol, rtol, max_acc=-1, max_rej=500, coef=None,
                                outputs=True, stream=None):
    """Every element its own step size; returns per-element t, dt, counts, status (CUDA tensors)."""
    import torch
    n = x.numel()
    out = {}
    if outputs:
        out = {"t": torch.empty(n, dtype=torch.float64, device=x.device),
               "dt": torch.empty(n, dtype=torch.float64, device=x.device),
               "n_acc": torch.empty(n, dtype=torch.int64, device=x.device),
               "n_rej": torch.empty(n, dtype=torch.int64, device=x.device),
               "status": torch.empty(n, dtype=torch.int32, device=x.device)}
    _check(lib().ode_integrate_adaptive_each(kind, method, n, _ptr(x), _ptr(coef), t0, t_end, dt0, atol, rtol,
                                             max_acc, max_rej, _ptr(out.get("t")), _ptr(out.get("dt")),
                                             _ptr(out.get("n_acc")), _ptr(out.get("n_rej")),
                                             _ptr(out.get("status")), _stream(stream)))
    return out


def gs_measure_fp64_peak(stream=None):
    v = C.c_double(0)
    _check(lib().gs_measure_fp64_peak(C.byref(v), _stream(stream)))
    return v.value


# --------------------------------------------------------------------------
# Owner of one Gray-Scott context and its state tensors
# --------------------------------------------------------------------------
class GrayScott:
    """One periodic Gray-Scott problem (Eq. 2) with state tensors u, v on the GPU.

    u, v: torch tensors shaped (nz, ny, nx), float64 or float32 (prec)."""

    def __init__(self, nx, ny, nz, L=2.5, Du=2e-5, Dv=1e-5, F=0.053, k=0.014, prec=GS_FP64, u=None, v=None,
                 Ly=None, Lz=None, stream=None, device="cuda"):
        import torch
        self.shape = (nz, ny, nx)
        self.prec = prec
        self.dtype = torch.float64 if prec == GS_FP64 else torch.float32
        self.ctx = gs_create(nx, ny, nz, L, Du, Dv, F, k, prec, Ly, Lz, stream)
        self.u = torch.empty(self.shape, dtype=self.dtype, device=device) if u is None else u
        self.v = torch.empty(self.shape, dtype=self.dtype, device=device) if v is None else v
        gs_bind_state(self.ctx, self.u, self.v)

    def set_state(self, u, v):
        self.u.copy_(u.to(self.u.device, self.dtype).reshape(self.shape))
        self.v.copy_(v.to(self.v.device, self.dtype).reshape(self.shape))

    def rhs(self, t=0.0):
        import torch
        fu, fv = torch.empty_like(self.u), torch.empty_like(self.v)
        gs_rhs(self.ctx, t, self.u, self.v, fu, fv)
        return fu, fv

    def step(self, method, t, dt, nsteps):
        return gs_step(self.ctx, method, t, dt, nsteps)

    def integrate_adaptive(self, atol, rtol, t, t_end, dt, max_accepted=-1, check=True, pair=None):
        if pair is not None:
            return gs_integrate_adaptive_pair(self.ctx, pair, atol, rtol, t, t_end, dt, max_accepted, check)
        return gs_integrate_adaptive(self.ctx, atol, rtol, t, t_end, dt, max_accepted, check)

    def set_observer(self, fn):
        """fn(t, u, v) -> bool, called by step / integrate_adaptive before each
        step and after the last (u, v: this problem's state tensors, read
        only); True stops the integration.  None removes the observer."""
        self._obs = gs_set_observer(self.ctx, None if fn is None else (lambda t, pu, pv: fn(t, self.u, self.v)))

    def close(self):
        if self.ctx:
            gs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# Batched ensembles of uneven Gray-Scott problems
# --------------------------------------------------------------------------
def _bcheck(st, ctx):
    if st != GS_OK:
        msg = lib().gsb_last_error(ctx) or b""
        raise GSError(st, msg.decode())


class GrayScottBatch:
    """Ensemble of independent Gray-Scott problems (gsb_* C ABI).

    instances: list of dicts {nx, ny, nz, F, k}.  u, v: concatenated state
    tensors of the ensemble precision; ``view(i)`` gives instance i's
    (nz, ny, nx) views."""

    def __init__(self, instances, L=2.5, Du=2e-5, Dv=1e-5, prec=GS_FP32, stream=None, device="cuda"):
        import torch
        n = len(instances)
        arr = (gsb_instance * n)(*[gsb_instance(d["nx"], d["ny"], d["nz"], d["F"], d["k"]) for d in instances])
        self.ctx = _vp()
        _check(lib().gsb_create(n, arr, L, Du, Dv, prec, _stream(stream), C.byref(self.ctx)))
        self.instances = [dict(d) for d in instances]
        offs = (C.c_longlong * (n + 1))()
        _bcheck(lib().gsb_layout(self.ctx, offs), self.ctx)
        self.offsets = [int(o) for o in offs]
        self.dtype = torch.float64 if prec == GS_FP64 else torch.float32
        self.u = torch.zeros(self.offsets[-1], dtype=self.dtype, device=device)
        self.v = torch.zeros(self.offsets[-1], dtype=self.dtype, device=device)
        _bcheck(lib().gsb_bind_state(self.ctx, _ptr(self.u), _ptr(self.v)), self.ctx)

    def view(self, i):
        d = self.instances[i]
        o, n = self.offsets[i], d["nx"] * d["ny"] * d["nz"]
        shape = (d["nz"], d["ny"], d["nx"])
        return self.u[o:o + n].view(shape), self.v[o:o + n].view(shape)

    def set_instance(self, i, u, v):
        uu, vv = self.view(i)
        uu.copy_(u.to(uu.device, self.dtype).reshape(uu.shape))
        vv.copy_(v.to(vv.device, self.dtype).reshape(vv.shape))

    def integrate_adaptive(self, atol, rtol, t, t_end, dt, max_accepted=-1, check=True):
        import numpy as np
        n = len(self.instances)
        tt = np.ascontiguousarray(np.broadcast_to(np.asarray(t, dtype=np.float64), (n,)).copy())
        dd = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)).copy())
        na = np.zeros(n, dtype=np.int64)
        nr = np.zeros(n, dtype=np.int64)
        stv = np.zeros(n, dtype=np.int32)
        st = lib().gsb_integrate_adaptive(self.ctx, atol, rtol, tt.ctypes.data_as(_dp), t_end, dd.ctypes.data_as(_dp),
                                          max_accepted, na.ctypes.data_as(_lp), nr.ctypes.data_as(_lp),
                                          stv.ctypes.data_as(C.POINTER(C.c_int)))
        if check:
            _bcheck(st, self.ctx)
        return {"status": st, "t": tt, "dt": dd, "n_acc": na, "n_rej": nr, "statuses": stv}

    def set_step_log(self, capacity):
        _bcheck(lib().gsb_set_step_log(self.ctx, capacity), self.ctx)
        self._log_cap = capacity

    def step_log(self):
        """Per instance: the accepted step sizes of the last integration."""
        import numpy as np
        cap = getattr(self, "_log_cap", 0)
        buf = np.zeros((len(self.instances), max(cap, 1)))
        cnt = np.zeros(len(self.instances), dtype=np.int64)
        _bcheck(lib().gsb_get_step_log(self.ctx, buf.ctypes.data_as(_dp), cap, cnt.ctypes.data_as(_lp)), self.ctx)
        return [buf[i, :min(int(cnt[i]), cap)].copy() for i in range(len(self.instances))]

    def set_tile(self, ty, zc):
        _bcheck(lib().gsb_set_tile(self.ctx, ty, zc), self.ctx)

    def autotune(self):
        a, b, ms = C.c_int(0), C.c_int(0), C.c_double(0)
        _bcheck(lib().gsb_autotune(self.ctx, C.byref(a), C.byref(b), C.byref(ms)), self.ctx)
        return a.value, b.value, ms.value

    def autotune_run(self, atol, rtol, t0, t_end, dt0):
        """Tile choice by timing this integration itself (state restored)."""
        a, b, ms = C.c_int(0), C.c_int(0), C.c_double(0)
        _bcheck(lib().gsb_autotune_run(self.ctx, atol, rtol, t0, t_end, dt0, C.byref(a), C.byref(b), C.byref(ms)),
                self.ctx)
        return a.value, b.value, ms.value

    def set_stage_depth(self, depth):
        """Staged-form ring depth of the stage kernels (0: vectorised form)."""
        _bcheck(lib().gsb_set_stage_depth(self.ctx, depth), self.ctx)

    def set_pairs(self, on, ty=7, depth=2):
        _bcheck(lib().gsb_set_pairs(self.ctx, int(on), ty, depth), self.ctx)

    def pairs(self):
        on, ty, depth = C.c_int(0), C.c_int(0), C.c_int(0)
        _bcheck(lib().gsb_get_pairs(self.ctx, C.byref(on), C.byref(ty), C.byref(depth)), self.ctx)
        return on.value, ty.value, depth.value

    def set_pair_lanes(self, mode, ty_wide=7):
        """1: 2 or 4 cells per lane where an instance's rows allow; 0: one."""
        _bcheck(lib().gsb_set_pair_lanes(self.ctx, int(mode), ty_wide), self.ctx)

    def pair_lanes(self):
        """(mode, ty_wide, [instances with 1, 2, 4 cells per lane])."""
        mode, tyw, counts = C.c_int(0), C.c_int(0), (C.c_int * 3)()
        _bcheck(lib().gsb_get_pair_lanes(self.ctx, C.byref(mode), C.byref(tyw), counts), self.ctx)
        return mode.value, tyw.value, list(counts)

    def set_grouping(self, cells_per_group):
        """Instance-group budget in cells (-1 automatic, 0 one group)."""
        _bcheck(lib().gsb_set_grouping(self.ctx, cells_per_group), self.ctx)

    def grouping(self):
        """(budget in cells, number of groups) in use."""
        c, n = C.c_longlong(0), C.c_int(0)
        _bcheck(lib().gsb_get_grouping(self.ctx, C.byref(c), C.byref(n)), self.ctx)
        return c.value, n.value

    def close(self):
        if self.ctx:
            lib().gsb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# Learned surrogate
# --------------------------------------------------------------------------
def _scheck(st, ctx):
    if st != GS_OK:
        msg = lib().sur_last_error(ctx) if ctx else lib().gs_last_global_error()
        raise GSError(st, (msg or b"").decode())


class Surrogate:
    """BF16 3D-conv surrogate of 16 RK4 steps (sur_* C ABI) on an (nz, ny, nx) grid."""

    def __init__(self, nx, ny, nz, stream=None):
        self.shape = (nz, ny, nx)
        self.ctx = _vp()
        _check(lib().sur_create(nx, ny, nz, _stream(stream), C.byref(self.ctx)))
        self.nparams = int(lib().sur_param_count())

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.nparams
        _scheck(lib().sur_set_params(self.ctx, p.ctypes.data_as(C.POINTER(C.c_float))), self.ctx)

    def get_params(self):
        import numpy as np
        p = np.zeros(self.nparams, dtype=np.float32)
        _scheck(lib().sur_get_params(self.ctx, p.ctypes.data_as(C.POINTER(C.c_float))), self.ctx)
        return p

    def get_grad(self):
        import numpy as np
        p = np.zeros(self.nparams, dtype=np.float32)
        _scheck(lib().sur_get_grad(self.ctx, p.ctypes.data_as(C.POINTER(C.c_float))), self.ctx)
        return p

    def set_normalization(self, mean, sd, scale):
        a = [(C.c_double * 2)(*map(float, x)) for x in (mean, sd, scale)]
        _scheck(lib().sur_set_normalization(self.ctx, *a), self.ctx)

    def forward(self, u, v, uo, vo):
        _scheck(lib().sur_forward(self.ctx, _ptr(u), _ptr(v), _ptr(uo), _ptr(vo)), self.ctx)

    def train_step(self, u, v, ut, vt, lr):
        loss = C.c_double(0)
        _scheck(lib().sur_train_step(self.ctx, _ptr(u), _ptr(v), _ptr(ut), _ptr(vt), lr, C.byref(loss)), self.ctx)
        return loss.value

    def advance(self, integ_ctx, u, v, judge=False, threshold=1e-3):
        rel, fb = C.c_double(0), C.c_int(0)
        _scheck(lib().sur_advance(self.ctx, integ_ctx, _ptr(u), _ptr(v), int(judge), threshold, C.byref(rel),
                                  C.byref(fb)), self.ctx)
        return rel.value, bool(fb.value)

    def close(self):
        if self.ctx:
            lib().sur_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
