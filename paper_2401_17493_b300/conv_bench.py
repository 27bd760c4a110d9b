"""Microbenchmark of the U-Net convolution kernels through the C ABI.

    python -m paper_2401_17493_b300.conv_bench [layer]

For each layer shape of the U-Net at training batch 4 (random BF16
activations and weights) it times `claire_conv3d_forward` (bias + ReLU) and
`claire_conv3d_wgrad` with CUDA events (3 warm-ups, 20 timed launches) and
prints one JSON line per layer: microseconds, TFLOP/s (2 V Cout 27 Cin per
launch) and the minimum-traffic rate (each activation read once, each output
written once).  With a layer name only that layer runs (the command profiled
by ncu for the convolution captures).

    python -m paper_2401_17493_b300.conv_bench steps [n]

times n (default 8) whole training steps of the U-Net (forward, loss,
backward, Adam) at batch 4 on random 64^3 inputs and targets, after one
untimed epoch of 4 steps (the command profiled for the training launch list).
"""

import ctypes
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

LAYERS = [("e0b", 64, 16, 16), ("d0a", 64, 48, 16), ("e1b", 32, 32, 32), ("d1a", 32, 96, 32),
          ("e2b", 16, 64, 64), ("d2a", 16, 192, 64), ("bb", 8, 128, 128)]
BATCH = 4


def train_steps(n):
    import time
    import torch
    from paper_2401_17493_b300 import unet as U
    gen = torch.Generator(device="cuda").manual_seed(0)
    inputs = [torch.rand((2, 64, 64, 64), device="cuda", generator=gen) for _ in range(16)]
    targets = [0.01 * torch.randn((3, 64, 64, 64), device="cuda", generator=gen)
               for _ in range(16)]
    model = U.UNet3D(seed=0)
    U.train(model, inputs, targets, 1, batch=BATCH)         # 4 untimed steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U.train(model, inputs, targets, max(1, n // 4), batch=BATCH)
    torch.cuda.synchronize()
    steps = 4 * max(1, n // 4)
    print(json.dumps({"training_steps": steps, "batch": BATCH,
                      "ms_per_step": (time.perf_counter() - t0) / steps * 1e3}), flush=True)


def main():
    import torch
    from paper_2401_17493_b300 import build, claire as C
    build.build()
    L = C.load_library()
    only = sys.argv[1] if len(sys.argv) > 1 else None
    if only == "steps":
        train_steps(int(sys.argv[2]) if len(sys.argv) > 2 else 8)
        return
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    gen = torch.Generator(device="cuda").manual_seed(0)
    for name, n, cin, cout in LAYERS:
        if only and name != only:
            continue
        B = BATCH
        V = B * n ** 3
        x = (torch.randn(V, cin, device="cuda", generator=gen) * 0.5).to(torch.bfloat16)
        w = (torch.randn(cout, 27, cin, device="cuda", generator=gen) * 0.05).to(torch.bfloat16)
        b = torch.zeros(cout, device="cuda")
        y = torch.empty(V, cout, device="cuda", dtype=torch.bfloat16)
        dy = (torch.randn(V, cout, device="cuda", generator=gen) * 0.1).to(torch.bfloat16)
        nsplit = max(1, min(160, V // 128))             # >= one weight-gradient CTA per SM
        part = torch.empty(nsplit * cout * 27 * cin, device="cuda")
        dw = torch.empty(cout * 27 * cin, device="cuda")

        def fwd():
            if L.claire_conv3d_forward(p(x), B, n, n, n, cin, p(w), p(b), cout, 1, p(y), None,
                                       st) != C.OK:
                raise RuntimeError("claire_conv3d_forward failed")

        def wgrad():
            if L.claire_conv3d_wgrad(p(x), B, n, n, n, cin, p(dy), cout, p(part), nsplit, p(dw),
                                     st) != C.OK:
                raise RuntimeError("claire_conv3d_wgrad failed")

        out = {"layer": name, "V": V, "cin": cin, "cout": cout}
        for tag, fn in (("fwd", fwd), ("wgrad", wgrad)):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 20
            out[tag + "_us"] = round(ms * 1e3, 1)
            out[tag + "_tflops"] = round(2.0 * V * cout * 27 * cin / (ms * 1e-3) / 1e12, 1)
            out[tag + "_gbs_min"] = round(V * (cin + cout) * 2 / (ms * 1e-3) / 1e9, 1)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
