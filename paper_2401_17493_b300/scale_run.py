"""Large single registration on one GPU: the 768^3 phantom pair in the
mixed-precision form (FP16 state / adjoint / incremental histories, FP32
arithmetic and coordinates, FP64 reductions), nt = 4, beta_v = 1e-3.

Reports the HBM high-water mark (library workspace and the process's peak
device use), the solve time, Hessian matvecs/s, and the per-kernel-class
event timings with the SL gather's fraction of the measured HBM peak.

    python -m paper_2401_17493_b300.scale_run [--n 768] [--precision 1] [--out res.json]
"""

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))


def run(n=768, precision=1, beta=1e-3, matvecs=10, precond=1, solves=1):
    """One registration of the n^3 phantom pair (seed 3) on the current device;
    returns the record printed by main().  With solves > 1 the first solve is an
    untimed warm-up (plans, first-use allocations) and the others are timed."""
    import torch
    from paper_2401_17493_b300 import claire, synth
    shape = (n, n, n)
    t0 = time.perf_counter()
    m0, m1 = synth.ellipsoid_pair_torch(shape, seed=3, max_disp_voxels=4.0 * n / 256)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    ctx = claire.Context(shape, nt=4, beta_v=beta, precision=precision, eps_opt=5e-2,
                         max_pcg=200, precond=precond, max_inner=10)
    ctx.set_images(m0, m1)
    del m0, m1
    torch.cuda.empty_cache()
    v = torch.zeros((3,) + shape, device="cuda")
    times = []
    for k in range(max(1, solves)):
        v.zero_()
        if k == max(1, solves) - 1:
            ctx.profile_reset(timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = ctx.solve(v)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t_solve = times[-1] if solves <= 1 else sum(times[1:]) / (len(times) - 1)
    prof = ctx.profile_read()
    ctx.profile_reset(timing=False)
    vt = torch.randn_like(v) * 1e-2
    out = torch.empty_like(v)
    ctx.hessian_matvec(vt, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(matvecs):
        ctx.hessian_matvec(vt, out)
    torch.cuda.synchronize()
    mv_s = matvecs / (time.perf_counter() - t0)
    free, total = torch.cuda.mem_get_info()
    try:
        peak = json.load(open(os.path.join(os.path.dirname(HERE), "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        peak = 6400.0
    kern = {k: {"launches": p["launches"], "ms": p["ms"],
                "gbs": p["timed_bytes"] / (p["ms"] * 1e-3) / 1e9 if p["ms"] > 0 else None}
            for k, p in prof.items() if p["launches"]}
    sl = kern.get("sl_step", {})
    res = {
        "grid": shape, "voxels": n ** 3, "precision": "fp16 fields" if precision else "fp32",
        "precond": "two-level" if precond else "spectral",
        "beta_v": beta, "generate_s": t_gen, "solve_s": t_solve, "timed_solves": len(times) - (solves > 1),
        "newton_iters": st.newton_iters, "matvecs": st.matvecs, "inner_iters": st.inner_iters,
        "grad_rel": st.grad_rel,
        "mismatch_rel": st.mismatch_rel, "status": st.status,
        "matvecs_per_s": mv_s,
        "workspace_gb": ctx.workspace_bytes / 1e9,
        "device_used_gb": (total - free) / 1e9,
        "torch_peak_gb": torch.cuda.max_memory_allocated() / 1e9,
        "sl_step_gbs": sl.get("gbs"), "sl_step_hbm_frac": (sl.get("gbs") or 0) / peak,
        "kernels": kern,
    }
    ctx.close()
    del v, vt, out
    torch.cuda.empty_cache()
    return res


def main():
    from paper_2401_17493_b300 import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=768)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--beta", type=float, default=1e-3)
    ap.add_argument("--matvecs", type=int, default=10)
    ap.add_argument("--precond", type=int, default=1, help="0 spectral, 1 two-level")
    ap.add_argument("--solves", type=int, default=1, help="> 1: untimed warm-up solve first")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    build.build()
    res = run(args.n, args.precision, args.beta, args.matvecs, args.precond, args.solves)
    print(json.dumps(res), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
