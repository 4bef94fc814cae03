"""The C-ABI library loads on a CPU-only host and exports every entry point
declared in include/gs.h (the method's interface) and in the internal header
of tuning, timing and test hooks (no compute calls: there is no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


INTERNAL = os.path.join(ROOT, "paper_2309_05331_b300", "csrc", "gs_internal.h")


def _declared(paths=None):
    names = set()
    if paths is None:
        paths = [os.path.join(ROOT, "include", fn) for fn in sorted(os.listdir(os.path.join(ROOT, "include")))
                 if fn.endswith(".h")]
    for path in paths:
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        # function declarations (a typedef of a function-pointer type declares no symbol)
        for m in re.finditer(r"^\s*(?!typedef\b)(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                             src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2309_05331_b300 import build
    return build.build()


def test_header_declares_the_named_boundary():
    d = _declared()
    for name in ("gs_create", "gs_step", "gs_integrate_adaptive", "ode_axpy_stage"):
        assert name in d


def test_public_header_holds_no_tuning_knobs():
    pub, internal = _declared(), _declared([INTERNAL])
    assert not (pub & internal)
    for name in ("gs_set_tile", "gs_set_kernel_variant", "gs_set_pair_config", "gs_time_stages", "gs_time_pairs",
                 "gsb_set_tile", "sur_set_conv_engine", "gs_measure_fp64_peak", "sur_debug_set_timeout_word"):
        assert name in internal and name not in pub


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = (_declared() | _declared([INTERNAL])) - exported
    assert not missing, missing


def test_library_loads_through_the_binding(libpath):
    import paper_2309_05331_b300 as gs
    L = gs.lib()
    for name in gs.exported_names():
        assert hasattr(L, name)
    assert set(gs.exported_names()) == _declared() | _declared([INTERNAL])
    # a pure host query works without a GPU
    assert gs.ode_workspace_size(1000) >= 256 + 8000


def test_invalid_arguments_are_rejected_without_a_gpu(libpath):
    import ctypes as C
    import paper_2309_05331_b300 as gs
    L = gs.lib()
    assert L.gs_create(None, None, None) == gs.GS_ERR_INVALID
    p = gs.gs_params(0, 4, 4, 2.5, 2.5, 2.5, 2e-5, 1e-5, 0.053, 0.014, gs.GS_FP64)
    ctx = C.c_void_p()
    assert L.gs_create(C.byref(p), None, C.byref(ctx)) == gs.GS_ERR_INVALID
    assert L.ode_axpy_stage(10, gs.GS_FP64, 16, None, None, None, None) == gs.GS_ERR_INVALID
    assert L.gs_step(None, 0, None, 0.1, 1) == gs.GS_ERR_INVALID
