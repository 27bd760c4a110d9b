"""Batched solves of uneven-grid pairs through the C ABI: the command profiled
for the grouped-launch list.

    python -m paper_2401_17493_b300.batch_bench [--pairs 8] [--mode grouped] [--reps 1]
                                                [--wait-us -1] [--graphs 1]

Builds `pairs` seeded blob pairs on grids cycling through 64^3, 96 x 112 x 80,
128^3 and 160 x 192 x 144 (nt 4, beta_v 5e-3, rel-grad 5e-2, two-level
preconditioner where every n_i % 4 == 0), solves them once untimed, then
`reps` times timed with `mode` = sequential (one solve after another),
batched (claire_solve_batch: one host thread and stream per pair, graphs) or
grouped (claire_solve_batch_grouped: one persistent launch per SL / trace /
FD8 march phase for the pairs that posted one; the first post of a round waits
up to `wait_us` microseconds for the others, < 0: until all have posted).
`--graphs 0` runs the PCG parts launch by launch (the profiled command: ncu
lists no kernels of graphs with conditional nodes).  Prints one JSON line.
"""

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

GRIDS = [(64, 64, 64), (96, 112, 80), (128, 128, 128), (160, 192, 144)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=8)
    ap.add_argument("--mode", default="grouped", choices=["sequential", "batched", "grouped"])
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--wait-us", type=int, default=-1)
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1])
    args = ap.parse_args()
    import numpy as np
    import torch
    from paper_2401_17493_b300 import build, claire, synth
    build.build()
    claire.load_library()
    ctxs, vs = [], []
    for i in range(args.pairs):
        shape = GRIDS[i % len(GRIDS)]
        m0, m1, _ = synth.blob_pair(shape, seed=500 + i, kmax=3, max_disp_voxels=2.0)
        ctx = claire.Context(shape, nt=4, beta_v=5e-3, eps_opt=5e-2, graphs=args.graphs)
        ctx.set_images(torch.from_numpy(m0.astype(np.float32)).cuda(),
                       torch.from_numpy(m1.astype(np.float32)).cuda())
        ctxs.append(ctx)
        vs.append(torch.zeros((3,) + shape, device="cuda"))

    def run():
        for v in vs:
            v.zero_()
        if args.mode == "sequential":
            return [ctx.solve(v)[1] for ctx, v in zip(ctxs, vs)], None
        if args.mode == "batched":
            return claire.solve_batch(ctxs, vs)[1], None
        _, st, launches = claire.solve_batch(ctxs, vs, grouped=True, wait_us=args.wait_us)
        return st, launches

    run()                                               # plans, graphs, caches
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.reps):
        stats, launches = run()
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / args.reps
    out = {"mode": args.mode, "pairs": args.pairs, "seconds": sec, "wait_us": args.wait_us,
           "graphs": args.graphs,
           "matvecs": int(sum(s.matvecs for s in stats)),
           "pde_solves": int(sum(s.pde_solves for s in stats)),
           "all_converged": all(s.grad_rel <= 5e-2 for s in stats)}
    if launches is not None:
        out["grouped_launches"], out["per_pair_launches_replaced"] = launches
    print(json.dumps(out), flush=True)
    for c in ctxs:
        c.close()


if __name__ == "__main__":
    main()
