"""Times one surrogate convolution call (sur_conv3d, or with --wgrad the
weight gradient sur_conv3d_wgrad) on a cubic grid.

    python -m paper_2309_05331_b300.conv_timing --grid 128 --engine 2 --epi 0 --cin 32 --cout 32
    python -m paper_2309_05331_b300.conv_timing --grid 128 --engine 2 --wgrad

Random BF16 activations and weights; prints one JSON line with the CUDA-event
time per call (after warm-up), the FLOP rate and the engine that ran.
"""
from __future__ import annotations

import argparse
import json

from . import lib


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--engine", type=int, default=0, help="0 automatic, 1 mma.sync, 2 tcgen05")
    ap.add_argument("--epi", type=int, default=0)
    ap.add_argument("--cin", type=int, default=32, help="padded input channels (8 or 32)")
    ap.add_argument("--cout", type=int, default=32, help="padded output channels (8 or 32)")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--wgrad", action="store_true", help="time the weight gradient instead")
    a = ap.parse_args(argv)
    n, ci, co = a.grid, a.cin, a.cout
    x = torch.randn((n, n, n, ci), device="cuda").to(torch.bfloat16)
    w = (0.2 * torch.randn((27, ci, co), device="cuda")).float()
    wp = torch.zeros(lib().sur_packed_bytes(ci, co), dtype=torch.uint8, device="cuda")
    assert lib().sur_pack_weights(ci, co, w.data_ptr(), 0, wp.data_ptr(), None) == 0
    b = torch.zeros(co, device="cuda")
    odt = torch.bfloat16 if a.epi in (0, 2) else torch.float32
    out = torch.empty((n, n, n, co), dtype=odt, device="cuda")
    mask = torch.randn((n, n, n, co), device="cuda").to(torch.bfloat16)
    assert lib().sur_set_conv_engine(a.engine) == 0
    if a.wgrad:
        dy = torch.randn((n, n, n, co), device="cuda").to(torch.bfloat16)
        nb = lib().sur_wgrad_workspace_bytes(ci, co)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        dw = torch.empty((27, ci, co), dtype=torch.float32, device="cuda")
        fn, args = lib().sur_conv3d_wgrad, (n, n, n, ci, co, x.data_ptr(), dy.data_ptr(), ci, co, dw.data_ptr(),
                                            ws.data_ptr(), nb, None)
    else:
        fn, args = lib().sur_conv3d, (n, n, n, ci, co, x.data_ptr(), wp.data_ptr(), b.data_ptr(), a.epi,
                                      mask.data_ptr() if a.epi == 2 else None, out.data_ptr(), co, None)
    for _ in range(3):
        assert fn(*args) == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        fn(*args)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flops = 2.0 * n ** 3 * 27 * ci * co
    print(json.dumps({"grid": n, "cin": ci, "cout": co, "op": "wgrad" if a.wgrad else f"conv epi {a.epi}",
                      "engine": lib().sur_conv_last_engine(),
                      "us": ms * 1e3, "tflops": flops / ms / 1e9}))


if __name__ == "__main__":
    main()
