"""The allocation-free adaptive ODE entry point against the regular one.

ode_integrate_adaptive_noalloc serves callers that may not allocate GPU
memory while they integrate (host applications that own all device memory
through their own pool, real-time loops that cannot take cudaMalloc's implicit
synchronisation, plugins restricted to memory they are handed).  Its scratch
is a static device array inside the library, so its results must equal those
of ode_integrate_adaptive with a caller workspace, call after call, even
though each call reuses the array left behind by the previous one.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synthetic_inputs as si
from tests._gpu_common import cuda_or_skip, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative L2, the FP64 parity tolerance of the other tests


def _noalloc_c(gs, kind, x, t, t_end, dt, tol):
    """Direct C-ABI call of the allocation-free entry point."""
    tt, dd = C.c_double(t), C.c_double(dt)
    na, nr = C.c_long(0), C.c_long(0)
    st = gs.lib().ode_integrate_adaptive_noalloc(kind, x.numel(), x.data_ptr(), C.byref(tt), t_end,
                                                 C.byref(dd), tol, tol, -1, C.byref(na), C.byref(nr), None)
    return st, tt.value, dd.value, na.value, nr.value


def _rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc_matches_workspace_entry_point_two_calls_in_a_row(kind):
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    for call, (n, seed, t0, t1) in enumerate([(100003, 1, 0.0, 10.0), (1 << 20, 5, 2.0, 7.5)]):
        x0 = si.ode_initial_values(n, seed=seed)
        x_ref = torch.from_numpy(x0.copy()).cuda()
        ref = gs.ode_integrate_adaptive(kind, x_ref, t0, t1, 1e-3, 1e-8, 1e-8)
        x_new = torch.from_numpy(x0.copy()).cuda()
        st, t, dt, na, nr = _noalloc_c(gs, kind, x_new, t0, t1, 1e-3, 1e-8)
        assert st == gs.GS_OK, (call, st)
        assert t == ref["t"] == t1
        assert (na, nr) == (ref["n_acc"], ref["n_rej"]), call
        assert dt == pytest.approx(ref["dt"], rel=1e-12)
        assert _rel_l2(to_np(x_new), to_np(x_ref)) <= TOL, call


def test_noalloc_rejects_sizes_beyond_its_capacity():
    torch = cuda_or_skip()
    import paper_2309_05331_b300 as gs
    x = torch.zeros((1 << 20) + 1, dtype=torch.float64, device="cuda")
    st, *_ = _noalloc_c(gs, 0, x, 0.0, 1.0, 1e-3, 1e-8)
    assert st == gs.GS_ERR_INVALID
    assert b"capacity" in gs.lib().gs_last_global_error()
