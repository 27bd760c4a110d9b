"""Per-kernel microbenchmark through the C ABI (one kernel per entry point).

    python -m paper_2401_17493_b300.kernel_bench [--size 256] [--reps 20] [--only sl]

Each entry point below launches exactly one of the library's kernels on a
256^3 grid (fields of 64 MiB, larger than L2), timed with CUDA events on the
launching stream after warm-up.  GB/s use the algorithmic bytes of the launch
(each input field read once, each output written once).  Also the command
profiled by ncu for the per-kernel captures.
"""

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--only", default=None)
    ap.add_argument("--precision", type=int, default=0, help="0 FP32, 1 FP16 field storage")
    ap.add_argument("--sl-gather", type=int, default=None, choices=[0, 1, 2],
                    help="SL gather variant (0 64 shared loads per node from a TMA-staged "
                         "brick, 1 register window, 2 64 loads from a cp.async-staged brick)")
    ap.add_argument("--sl-t1", type=int, default=None, choices=[4, 8, 16],
                    help="SL brick depth along x1")
    ap.add_argument("--march-t1", type=int, default=None, choices=[8, 16, 32, 64],
                    help="planes per CTA of the FD8 history kernels")
    args = ap.parse_args()
    import torch
    from paper_2401_17493_b300 import build, claire, synth
    build.build()
    n = args.size
    shape = (n, n, n)
    N = n ** 3
    gen = torch.Generator(device="cuda").manual_seed(0)
    u = torch.rand(shape, device="cuda", generator=gen)
    v = torch.from_numpy(synth.bandlimited_velocity(shape, 8, 4.0, 3).astype(np.float32)).cuda()
    ctx = claire.Context(shape, nt=4, precision=args.precision)
    if args.sl_gather is not None or args.sl_t1 is not None or args.march_t1 is not None:
        w0, t0, m0 = ctx.tuning()
        ctx.set_tuning(w0 if args.sl_gather is None else args.sl_gather,
                       t0 if args.sl_t1 is None else args.sl_t1,
                       m0 if args.march_t1 is None else args.march_t1)
    ctx.set_images(u, u)
    d, _ = ctx.trace(v)
    out1 = torch.empty(shape, device="cuda")
    w = torch.empty((3,) + shape, device="cuda")
    w2 = torch.empty((3,) + shape, device="cuda")
    vt = torch.from_numpy(synth.bandlimited_velocity(shape, 8, 1.0, 5).astype(np.float32)).cuda()
    ctx.objective_gradient(0.5 * v, want_gradient=False)     # state history for the matvec
    cases = {
        "sl": (lambda: ctx.lib.claire_interp(ctx.h, claire._ptr(u), claire._ptr(d),
                                             claire._ptr(out1)), 20 * N),
        "trace": (lambda: ctx.lib.claire_trace(ctx.h, claire._ptr(v), claire._ptr(w), None),
                  24 * N),
        # both directions (forward and backward departure points) in one launch
        "trace2": (lambda: ctx.lib.claire_trace(ctx.h, claire._ptr(v), claire._ptr(w),
                                                claire._ptr(w2)), 36 * N),
        "grad8": (lambda: ctx.lib.claire_grad8(ctx.h, claire._ptr(u), claire._ptr(w)), 16 * N),
        "div8": (lambda: ctx.lib.claire_div8(ctx.h, claire._ptr(v), claire._ptr(out1)), 16 * N),
        # one Gauss-Newton matvec: sdot_hist, 8 SL steps, accum_hist, spectral, cufft
        "matvec": (lambda: ctx.lib.claire_hessian_matvec(ctx.h, claire._ptr(vt), claire._ptr(w)),
                   None),
        # one application of the preconditioner (two-level where every n_i % 4 == 0):
        # fine FFTs, split, the nested CG on the n/2 grid, merge
        "precond": (lambda: ctx.lib.claire_precondition(ctx.h, claire._ptr(vt), claire._ptr(w),
                                                        None), None),
    }
    kind = {"sl": "sl_step", "trace": "trace", "trace2": "trace", "grad8": "grad8", "div8": "div8",
            "matvec": None, "precond": None}
    res = {}
    for name, (fn, nbytes) in cases.items():
        if args.only and name != args.only:
            continue
        for _ in range(args.warmup):
            assert fn() == 0
        torch.cuda.synchronize()
        # per-launch CUDA events on the launching stream (the library's profiler)
        ctx.profile_reset(timing=True)
        for _ in range(args.reps):
            assert fn() == 0
        prof = ctx.profile_read()
        if kind[name] is None:          # report every kernel class the call launched
            for k, p in prof.items():
                if p["timed"]:
                    ms = p["ms"] / p["timed"]
                    res[f"{name}/{k}"] = {"ms_per_launch": ms,
                                          "launches_per_call": p["launches"] / args.reps,
                                          "GB/s": p["bytes"] / p["launches"] / (ms * 1e-3) / 1e9}
            continue
        p = prof[kind[name]]
        ms = p["ms"] / p["timed"]
        res[name] = {"ms": ms, "GB/s": p["bytes"] / p["launches"] / (ms * 1e-3) / 1e9,
                     "bytes_per_launch": p["bytes"] / p["launches"]}
    print(json.dumps({"size": n, "precision": args.precision, "tuning": ctx.tuning(),
                      "kernels": res}))
    ctx.close()


if __name__ == "__main__":
    main()
