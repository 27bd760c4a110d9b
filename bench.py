#!/usr/bin/env python
"""Benchmark of the 256^3 registration hot path on one B300 (or N replicas).

One step = one complete registration of the 256^3 brain-like phantom pair:
beta_v continuation 1e-1 -> 1e-2 -> 1e-3 -> 1e-4 (Sec. 2.6), each level solved
by inexact Gauss-Newton-Krylov to a relative gradient of 5e-2, nt = 4,
H1-seminorm regularisation, FP32, PCG preconditioned with the two-level
zero-velocity Hessian (the paper's default, Sec. 2.6; nested CG capped at 10
iterations).  The same solve with the spectral preconditioner is reported beside it.  Inputs (m0, m1, v = 0) are resident in HBM
when the timed region starts; the working set (~4 GB) is far larger than L2.

Printed (rank 0, one JSON line): solve seconds per registration (value), plus
Hessian matvecs/s at 256^3, the interpolation + FD8 share of HBM peak, the
roofline of the dominant kernel (event-timed inside the timed solves), the
end-to-end number through the host-buffer C entry point, clocks sampled
during the timed region, per-level counts of the continuation and the solve
under the other reading of its stopping denominator, the plain FP32 solver
against the mixed + warm-started + batched form on held-out 128^3 pairs (with
a U-Net trained in this run), the 768^3 registration, and the FP64 CPU oracle
timed at 256^3 on the host cores.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
With N > 1 (torchrun) every rank registers its own pair: replicas only, no
collective on the data path (weak scaling).
"""

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "256³ solve s to rel-grad 5e-2; Hessian matvecs/s; interp+FD % of HBM peak"
BETAS = [1e-1, 1e-2, 1e-3, 1e-4]
NT = 4
EPS_OPT = 5e-2
MAX_PCG = 200
SEED = 2
PRECOND = 1                # two-level zero-velocity preconditioner (Sec. 2.5.6, 2.6)
MAX_INNER = 10             # nested CG cap per preconditioner application
INTERP_FD = ("trace", "sl_step", "adjoint_factor", "grad8", "div8", "sdot_hist", "accum_hist")
# DRAM traffic per voxel and launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum over the matvec's SL steps at 256^3, 24 algorithmic
# B/voxel), with the SHA-256 of the kernel's source (sl_source_sha) at the time
# of the capture: when the source differs, the figure is stale and
# roofline.traffic is reported as null.
NCU_TRAFFIC_PER_VOXEL = {
    "sl_step": (23.27, "457bed694d4d863d84c9e3be41eedd6ee1e49b8f44b6984a8ace9529d0fff7b1")}
# 64-tap gathers of a field per 256^3 registration of the headline solve (trace
# components x directions + SL steps + adjoint factors), counted by the
# library's launch profile in this bench's own arm ("field_gathers_per_registration"):
# the reference arm scales its per-gather time by it.
GATHERS_PER_REGISTRATION = 161
# Grouped batch: how long the first post of a round waits for the other pairs
# (microseconds); 10 measured best among 0, 10, 40, 200 and waiting for all.
GROUP_WAIT_US = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="claire", choices=["claire", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--matvecs", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-pair batched workload")
    ap.add_argument("--batch-pairs", type=int, default=32)
    ap.add_argument("--no-combined", action="store_true",
                    help="skip the plain vs mixed + warm start + batched comparison")
    ap.add_argument("--combined-train", type=int, default=2000,
                    help="solver-generated 128^3 training pairs of the bench's U-Net")
    ap.add_argument("--combined-epochs", type=int, default=40)
    ap.add_argument("--combined-eval", type=int, default=200, help="held-out pairs")
    ap.add_argument("--no-scale", action="store_true", help="skip the 768^3 registration")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="replay the PCG parts of the 256^3 solves as CUDA graphs (default); 0 "
                         "launches every kernel (profilers list the kernels inside graphs that "
                         "hold a conditional node only this way)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x):
    """Max of a float over the ranks of the initialised process group (the timed
    region of the slowest replica); the value itself in a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_registration(t_max, steps, world):
    """Whole-job time per registration: `world` replicas each registered `steps`
    pairs within the slowest replica's time t_max (any unit)."""
    return t_max / (steps * world)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"claire_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(n):
    """The headline pair and the velocity that generated m1 (float32)."""
    from paper_2401_17493_b300 import synth
    return synth.ellipsoid_pair((n, n, n), seed=SEED)


BATCH_GRIDS = [(64, 64, 64), (96, 112, 80), (128, 128, 128), (160, 192, 144), (192, 192, 192)]
BATCH_BETA = 5e-3


def _batch_pair(seed):
    import numpy as np
    from paper_2401_17493_b300 import synth
    rng = np.random.default_rng(seed)
    shape = BATCH_GRIDS[int(rng.integers(0, len(BATCH_GRIDS)))]
    m0, m1, _ = synth.ellipsoid_pair(shape, seed=seed)
    return shape, m0, m1


def batch_workload(npairs):
    """Seeded pairs 1000.. on grids drawn uniformly from BATCH_GRIDS (generated in
    spawned worker processes: no fork after CUDA initialisation)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_pair, range(1000, 1000 + npairs)))


def run_batch(args, pairs):
    """Uneven-grid batch: sequential per-pair solves vs claire_solve_batch
    (concurrent streams, CUDA-graph PCG iterations) vs
    claire_solve_batch_grouped (one persistent launch per SL / trace / FD8 march
    phase for all pairs, launch by launch otherwise), beta_v 5e-3, nt 4."""
    import numpy as np
    import torch
    from paper_2401_17493_b300 import claire
    ctxs, vs = [], []
    for shape, m0, m1 in pairs:
        ctx = claire.Context(shape, nt=NT, beta_v=BATCH_BETA, eps_opt=EPS_OPT, max_pcg=MAX_PCG,
                             graphs=1, precond=PRECOND, max_inner=MAX_INNER)
        ctx.set_images(torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda())
        ctxs.append(ctx)
        vs.append(torch.zeros((3,) + shape, device="cuda"))
    for ctx, v in zip(ctxs, vs):                       # warm-up: plans, graphs, caches
        v.zero_()
        ctx.solve(v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_stats = []
    for ctx, v in zip(ctxs, vs):
        v.zero_()
        seq_stats.append(ctx.solve(v)[1])
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    v_seq = [v.clone() for v in vs]
    for v in vs:
        v.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, bstats = claire.solve_batch(ctxs, vs)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    same = all(torch.equal(a, b) for a, b in zip(v_seq, vs))
    grouped = {}
    for name, wait_us in (("grouped", GROUP_WAIT_US), ("grouped_lockstep", -1)):
        for v in vs:                                   # warm-up, then timed
            v.zero_()
        claire.solve_batch(ctxs, vs, grouped=True, wait_us=wait_us)
        for v in vs:
            v.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, gstats, glaunches = claire.solve_batch(ctxs, vs, grouped=True, wait_us=wait_us)
        torch.cuda.synchronize()
        tg = time.perf_counter() - t0
        grouped[name] = {"seconds": tg, "wait_us": wait_us, "speedup": None,
                         "vs_batched": None, "grouped_launches": int(glaunches[0]),
                         "per_pair_launches_replaced": int(glaunches[1]),
                         "all_converged": all(st.grad_rel <= EPS_OPT for st in gstats),
                         "equals_sequential": all(torch.equal(a, b) for a, b in zip(v_seq, vs))}
    voxels = sum(int(np.prod(c.shape)) for c in ctxs)
    # PDE solves x voxels: the transport work of the batch, comparable across grid sizes
    vox_pde = sum(int(np.prod(c.shape)) * st.pde_solves for c, st in zip(ctxs, bstats))
    for c in ctxs:
        c.close()
    for g in grouped.values():
        g["speedup"] = t_seq / g["seconds"]
        g["vs_batched"] = t_batch / g["seconds"]
    return {"pairs": len(ctxs), "grids": sorted(set(str(c) for c, _, _ in pairs)),
            "voxels": voxels, "sequential_s": t_seq, "batched_s": t_batch,
            "speedup": t_seq / t_batch, "pairs_per_s": len(ctxs) / t_batch,
            "matvecs": int(sum(st.matvecs for st in bstats)),
            "all_converged": all(st.grad_rel <= EPS_OPT for st in bstats),
            "batched_equals_sequential": bool(same),
            **grouped,
            "voxel_pde_solves": vox_pde,
            "voxel_pde_solves_per_s": {"batched": vox_pde / t_batch, "sequential": vox_pde / t_seq,
                                       "grouped": vox_pde / grouped["grouped"]["seconds"]},
            "workload": "ellipsoid phantom pairs seeds 1000.., grids from {64^3, 96x112x80, "
                        "128^3, 160x192x144, 192^3}, beta_v 5e-3, nt 4, rel-grad 5e-2, "
                        "two-level preconditioner"}


def sl_source_sha():
    """SHA-256 of the SL step's source: in kernels.cu its tile function and
    kernel (from the section comment to the next section), sl_tma.cuh (the TMA
    brick staging), sl_brick.cuh, common.cuh and tc_sm100.cuh."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2401_17493_b300", "csrc")
    try:
        k = open(os.path.join(csrc, "kernels.cu")).read()
        m = re.search(r"// MODE 0: out = .*?(?=// -+ grouped launches\n)", k, flags=re.S)
        if m is None:
            return None
        h = hashlib.sha256(m.group(0).encode())
        for f in ("sl_tma.cuh", "sl_brick.cuh", "common.cuh", "tc_sm100.cuh"):
            h.update(open(os.path.join(csrc, f), "rb").read())
        return h.hexdigest()
    except OSError:
        return None


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def set_oracle_threads(t):
    from oracle import fd8, interp, spectral
    interp.set_threads(t)
    fd8.set_threads(t)
    spectral.WORKERS = t


def pick_oracle_threads():
    """All usable host CPUs, or half of them when that gathers a 96^3 field
    faster (the gathers are memory-bound; on some hosts fewer threads win)."""
    import numpy as np
    from oracle import interp
    full = host_threads()
    rng = np.random.default_rng(0)
    n = 96
    u = rng.standard_normal((n,) * 3)
    q = np.stack(np.meshgrid(*[np.arange(n, dtype=float)] * 3, indexing="ij"))
    q = q + rng.uniform(-2.0, 2.0, size=(3, n, n, n))
    best = None
    for t in sorted({full, max(1, full // 2)}, reverse=True):
        interp.set_threads(t)
        t0 = time.perf_counter()
        interp.interp(u, q)
        dt = time.perf_counter() - t0
        if best is None or dt < best[1]:
            best = (t, dt)
    interp.set_threads(1)
    return best[0]


def cpu_oracle_units(m0, m1, v, vt, beta):
    """The FP64 oracle at the full grid on the host cores: one transport m(1)
    (trace + nt SL steps), one objective + gradient evaluation (state, adjoint,
    gradient), one Gauss-Newton Hessian matvec.  Returns seconds of each, the
    threads used and the threads kept busy (process CPU time / wall time)."""
    import numpy as np
    from oracle import reduced, transport
    threads = pick_oracle_threads()
    set_oracle_threads(threads)
    a, b = m0.astype(np.float64), m1.astype(np.float64)
    v, vt = v.astype(np.float64), vt.astype(np.float64)
    c0, t0 = time.process_time(), time.perf_counter()
    transport.state_solve(a, v, NT)
    t1 = time.perf_counter()
    prob = reduced.Problem(a, b, nt=NT, beta_v=beta)
    ev = reduced.evaluate(prob, v)
    t2 = time.perf_counter()
    reduced.hessian_matvec(prob, ev, vt)
    t3 = time.perf_counter()
    busy = (time.process_time() - c0) / (t3 - t0)
    set_oracle_threads(1)
    return {"transport_s": t1 - t0, "gradient_s": t2 - t1, "matvec_s": t3 - t2,
            "threads": threads, "busy": busy}


def oracle_registration_estimate(u, st, levels):
    """Seconds of the oracle's own registration with the GPU solve's counts: one
    evaluation at v = 0 and one per level start, per Newton step the gradient
    completion (an evaluation minus its state solve) and the Armijo trial state
    solves, plus the matvecs.  The nested coarse-grid CG of the two-level
    preconditioner is not counted."""
    n_gn = st["newton_iters"]
    trials = n_gn + st.get("linesearch_halvings", 0)
    return ((1 + levels) * u["gradient_s"] + n_gn * (u["gradient_s"] - u["transport_s"]) +
            trials * u["transport_s"] + st["matvecs"] * u["matvec_s"])


def run_reference(args, world, rank):
    """The oracle arm: each step is one FP64 SL step of the headline workload at
    its full grid (the 64-tap gather of m0 at the RK2 departure points of the
    velocity that generated m1), on the host cores.  value / ms_per_step are the
    time that step took; the registration estimate is a separate key."""
    if rank != 0:
        return
    import numpy as np
    from oracle import interp, transport
    n = args.size
    m0, m1, v = workload(n)
    threads = pick_oracle_threads()
    set_oracle_threads(threads)
    m0 = m0.astype(np.float64)
    y = transport.departure_points(v.astype(np.float64), NT, +1)     # untimed, once
    for _ in range(args.warmup):
        interp.interp(m0, y)
    times, busy = [], []
    for _ in range(args.steps):
        c0, t0 = time.process_time(), time.perf_counter()
        interp.interp(m0, y)
        dt = time.perf_counter() - t0
        times.append(dt)
        busy.append((time.process_time() - c0) / dt)
    value = float(np.mean(times))
    cores = int(round(max(busy)))
    sample = (f"one FP64 oracle SL step (64-tap gather of the {n}^3 template at the RK2 "
              f"departure points of the workload's velocity) per step, {threads} threads of "
              f"{host_threads()} host CPUs, {cores} kept busy")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{n}^3 ellipsoid phantom pair (seed {SEED}), nt 4",
                   "sample": "one SL step per step (not a registration)"},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if GATHERS_PER_REGISTRATION > 0:
        line["registration_estimate"] = {
            "value": value * GATHERS_PER_REGISTRATION, "unit": "s",
            "basis": f"per-gather time x {GATHERS_PER_REGISTRATION} field gathers of one GPU "
                     "registration of this workload (an extrapolation, not a measurement)"}
    print(json.dumps(line), flush=True)


def continuation_levels(ctx, betas, reps):
    """Per-level counts of the continuation, and the solve under the other
    reading of its stopping rule.

    reading C-10 (the headline): every level stops at eps_opt ||g(v = 0)||_inf;
    own-start reading: each level stops at eps_opt ||g(v_start)||_inf, v_start
    the level's warm start (its gradient evaluated with the level's beta_v).
    Both run level by level (claire_solve per level); the other reading is also
    timed (reps solves after one warm-up, CUDA events, the per-level gradient
    evaluations included) and its final gradient is also given relative to
    ||g(v = 0)||_inf."""
    import torch
    shape = ctx.shape
    stream = torch.cuda.current_stream()
    v = torch.zeros((3,) + shape, device="cuda")
    ctx.set_beta(betas[0])
    _, g = ctx.objective_gradient(v)
    g0 = float(g.abs().max())
    levels = []
    for b in betas:
        ctx.set_beta(b)
        ctx.set_options(gnorm0=g0)
        _, st = ctx.solve(v)
        levels.append({"beta_v": b, "newton_iters": st.newton_iters, "matvecs": st.matvecs,
                       "grad_rel": st.grad_rel, "mismatch_rel": st.mismatch_rel})

    def own_start():
        v.zero_()
        out = []
        for b in betas:
            ctx.set_beta(b)
            ctx.set_options(gnorm0=0.0)
            _, gs = ctx.objective_gradient(v)
            ctx.set_options(gnorm0=float(gs.abs().max()))
            _, st = ctx.solve(v)
            out.append(st)
        return out

    own_start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sts = own_start()
    e1.record(stream)
    torch.cuda.synchronize()
    _, gf = ctx.objective_gradient(v)
    ctx.set_options(gnorm0=0.0)
    ctx.set_beta(betas[0])
    return {
        "denominator_g0": {"levels": levels},
        "denominator_own_start": {
            "seconds": e0.elapsed_time(e1) / 1e3 / reps, "reps": reps,
            "levels": [{"beta_v": b, "newton_iters": st.newton_iters, "matvecs": st.matvecs,
                        "grad_rel_own": st.grad_rel, "mismatch_rel": st.mismatch_rel}
                       for b, st in zip(betas, sts)],
            "newton_iters": sum(st.newton_iters for st in sts),
            "matvecs": sum(st.matvecs for st in sts),
            "mismatch_rel": sts[-1].mismatch_rel,
            "grad_rel_vs_g0": float(gf.abs().max()) / g0},
    }


def run_combined(args):
    """The plain FP32 solver (zero initial guess, pairs one after another)
    against mixed precision + U-Net warm start + batched solves on held-out
    128^3 pairs (unet.evaluate_combined), with a U-Net trained here on
    solver-generated pairs: seeds 10000.. for training, 20000.. held out,
    beta_v 1e-2, rel-grad 5e-2 with the same denominator for both arms.  The
    default recipe (2000 pairs, 40 epochs, 200 held out) is the learned warm
    start's own; smaller ones train faster and gain less."""
    import torch
    from paper_2401_17493_b300 import unet
    n, beta = 128, 1e-2
    t0 = time.perf_counter()
    inputs, targets = [], []
    seeds = list(range(10000, 10000 + args.combined_train))
    for i in range(0, len(seeds), 64):
        pairs = unet.make_pairs(seeds[i:i + 64], n)
        vs = unet.solve_targets(pairs, n, beta)
        for (m0, m1), v in zip(pairs, vs):
            inputs.append(unet.resample(torch.stack([m0, m1]).contiguous(), (n,) * 3,
                                        (64,) * 3, 2))
            targets.append(unet.resample(v.contiguous(), (n,) * 3, (64,) * 3, 3))
        del pairs, vs
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    model = unet.UNet3D(seed=0)
    t0 = time.perf_counter()
    hist = unet.train(model, inputs, targets, args.combined_epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del inputs, targets
    held = unet.make_pairs(list(range(20000, 20000 + args.combined_eval)), n)
    res = unet.evaluate_combined(model, held, n, beta, batch=min(64, args.combined_eval))
    del held
    res.update({"grid": n, "beta_v": beta, "train_pairs": args.combined_train,
                "epochs": args.combined_epochs, "train_s": t_train, "targets_s": t_data,
                "final_loss": hist[-1] if hist else None,
                "target_2x_met": bool(res["speedup"] >= 2.0)})
    torch.cuda.empty_cache()
    return res


def run_claire(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2401_17493_b300 import build, claire

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    n = args.size
    shape = (n, n, n)
    m0, m1, v_gen = workload(n)
    pairs = None
    if not args.no_batch and rank == 0 and world == 1:
        pairs = batch_workload(args.batch_pairs)     # before any CUDA call of this process
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    m0d, m1d = dev(m0), dev(m1)
    ctx = claire.Context(shape, nt=NT, beta_v=BETAS[0], eps_opt=EPS_OPT, max_newton=50,
                         max_pcg=MAX_PCG, precond=PRECOND, max_inner=MAX_INNER,
                         graphs=args.graphs)
    ctx.set_images(m0d, m1d)
    stream = torch.cuda.current_stream()
    v = torch.zeros((3,) + shape, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        v.zero_()
        ctx.solve_continuation(BETAS, v)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    ctx.profile_reset(timing=True)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        v.zero_()
        _, st = ctx.solve_continuation(BETAS, v)
        stats.append(st.as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    t_max = reduce_max(ms_total)
    s_per_solve = per_registration(t_max / 1e3, args.steps, world)
    launches_per_step = sum(p["launches"] for k, p in prof.items() if k != "cufft") / args.steps

    # the same solve with the spectral preconditioner (beta_v L)^-1
    v_fp32 = v.clone()
    ctx.set_options(precond=0)
    vs_ = torch.zeros_like(v)
    for _ in range(args.warmup):
        vs_.zero_()
        ctx.solve_continuation(BETAS, vs_)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    sstats = []
    for _ in range(args.steps):
        vs_.zero_()
        _, sts = ctx.solve_continuation(BETAS, vs_)
        sstats.append(sts.as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    spec_s = e0.elapsed_time(e1) / 1e3 / args.steps
    spectral_pc = {"value": spec_s, "unit": "s", "matvecs": sstats[-1]["matvecs"],
                   "newton_iters": sstats[-1]["newton_iters"],
                   "grad_rel": sstats[-1]["grad_rel"], "mismatch_rel": sstats[-1]["mismatch_rel"],
                   "status": sstats[-1]["status"],
                   "two_level_speedup": spec_s / (t_max / 1e3 / args.steps)}
    ctx.set_options(precond=PRECOND)

    # mixed-precision form (FP16 field storage): same protocol, same accuracy criteria
    ctx.set_options(precision=1)
    vm = torch.zeros_like(v)
    for _ in range(args.warmup):
        vm.zero_()
        ctx.solve_continuation(BETAS, vm)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    mstats = []
    for _ in range(args.steps):
        vm.zero_()
        _, stm = ctx.solve_continuation(BETAS, vm)
        mstats.append(stm.as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    mixed_s = e0.elapsed_time(e1) / 1e3 / args.steps
    mixed = {"value": mixed_s, "unit": "s", "speedup_vs_fp32": (t_max / 1e3 / args.steps) / mixed_s,
             "grad_rel": mstats[-1]["grad_rel"], "mismatch_rel": mstats[-1]["mismatch_rel"],
             "matvecs": mstats[-1]["matvecs"], "status": mstats[-1]["status"],
             "v_rel_diff_vs_fp32": float(torch.linalg.vector_norm(vm - v_fp32) /
                                         torch.linalg.vector_norm(v_fp32)),
             "storage": "fp16 fields, fp32 math/coordinates/PCG vectors, fp64 reductions"}
    ctx.set_options(precision=0)

    # Hessian matvecs/s at the converged point (50 back-to-back GN matvecs)
    J, _ = ctx.objective_gradient(v, want_gradient=False)
    vt = torch.randn((3,) + shape, device="cuda") * 1e-2
    out = torch.empty_like(vt)
    for _ in range(5):
        ctx.hessian_matvec(vt, out)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.matvecs):
        ctx.hessian_matvec(vt, out)
    e1.record(stream)
    torch.cuda.synchronize()
    matvecs_per_s = args.matvecs / (e0.elapsed_time(e1) / 1e3)
    # per-class rates of the matvec kernels (every launch event-timed; a separate pass,
    # the matvecs/s above ran without the per-launch events)
    ctx.profile_reset(timing=True)
    for _ in range(10):
        ctx.hessian_matvec(vt, out)
    torch.cuda.synchronize()
    mprof = ctx.profile_read()
    ctx.profile_reset(timing=False)
    m_bytes = sum(mprof[k]["timed_bytes"] for k in INTERP_FD if k in mprof)
    m_ms = sum(mprof[k]["ms"] for k in INTERP_FD if k in mprof)
    matvec_interp_gbs = m_bytes / (m_ms * 1e-3) / 1e9 if m_ms > 0 else None

    # per-level counts (reading C-10) and the solve under the own-start reading
    levels = continuation_levels(ctx, BETAS, max(1, min(args.steps, 5)))
    levels["headline_levels_match"] = (
        sum(lv["newton_iters"] for lv in levels["denominator_g0"]["levels"]) ==
        stats[-1]["newton_iters"] and
        sum(lv["matvecs"] for lv in levels["denominator_g0"]["levels"]) == stats[-1]["matvecs"])

    # end to end through the host-buffer entry point: H2D m0, m1, v; solve; D2H v
    m0h = torch.from_numpy(m0).pin_memory()
    m1h = torch.from_numpy(m1).pin_memory()
    vh = torch.zeros((3,) + shape).pin_memory()
    e2e_times = []
    for _ in range(max(1, args.steps)):
        vh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve_host(m0h, m1h, vh, BETAS)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = per_registration(reduce_max(sum(e2e_times)), len(e2e_times), world)

    peak, peak_src = peaks()
    mine = {k: p for k, p in prof.items() if k != "cufft" and p["timed"] > 0}
    dom = max(mine, key=lambda k: mine[k]["ms"])
    d = mine[dom]
    # launches replayed inside captured graphs are counted, not timed: the rate is
    # the timed launches' algorithmic bytes over their event-timed duration
    achieved = d["timed_bytes"] / (d["ms"] * 1e-3) / 1e9
    traffic = None
    if dom in NCU_TRAFFIC_PER_VOXEL and NCU_TRAFFIC_PER_VOXEL[dom][1] == sl_source_sha():
        traffic = NCU_TRAFFIC_PER_VOXEL[dom][0]
    # 64-tap field gathers per registration: 3 per trace direction (a trace launch
    # moves 12 + 12 x directions bytes per voxel), one per SL step / adjoint factor
    tr = prof.get("trace", {"bytes": 0.0, "launches": 0})
    gathers = ((tr["bytes"] / n ** 3 - 12 * tr["launches"]) / 4 +
               prof.get("sl_step", {"launches": 0})["launches"] +
               prof.get("adjoint_factor", {"launches": 0})["launches"]) / args.steps
    interp_bytes = sum(mine[k]["timed_bytes"] for k in INTERP_FD if k in mine)
    interp_ms = sum(mine[k]["ms"] for k in INTERP_FD if k in mine)
    interp_gbs = interp_bytes / (interp_ms * 1e-3) / 1e9
    total_kernel_ms = sum(p["ms"] for p in prof.values())

    v_final = v_fp32.cpu().numpy()
    vt_host = vt.cpu().numpy()
    st0 = stats[-1]
    workspace_gb = ctx.workspace_bytes / 1e9
    ctx.close()
    del m0d, m1d, v, vs_, vm, vt, out, v_fp32
    torch.cuda.empty_cache()

    batch = run_batch(args, pairs) if pairs is not None else None
    if batch is not None:           # the same rate of one 256^3 registration, for comparison
        batch["voxel_pde_solves_per_s"]["single_large_solve"] = st0["pde_solves"] * n ** 3 / s_per_solve
    combined = None
    if rank == 0 and world == 1 and not args.no_combined:
        combined = run_combined(args)
    scale = None
    if rank == 0 and world == 1 and not args.no_scale and n == 256:
        from paper_2401_17493_b300 import scale_run
        scale = scale_run.run(768, precision=1, beta=1e-3, matvecs=10, precond=PRECOND, solves=2)
        scale.pop("kernels", None)
        scale["workload"] = ("768^3 ellipsoid phantom pair (seed 3), FP16 histories, nt 4, "
                             "beta_v 1e-3, rel-grad 5e-2, two-level preconditioner; one "
                             "untimed warm-up solve, one timed")
        f32 = scale_run.run(768, precision=0, beta=1e-3, matvecs=10, precond=PRECOND, solves=2)
        scale["fp32_storage"] = {k: f32[k] for k in ("solve_s", "newton_iters", "matvecs",
                                                     "grad_rel", "mismatch_rel", "matvecs_per_s",
                                                     "workspace_gb", "device_used_gb")}
        scale["mixed_vs_fp32"] = {"time": f32["solve_s"] / scale["solve_s"],
                                  "workspace": scale["workspace_gb"] / f32["workspace_gb"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        units = cpu_oracle_units(m0, m1, v_final, vt_host, BETAS[-1])
        est = oracle_registration_estimate(units, st0, len(BETAS))
        cpu = {"value": est, "unit": "s", "cores": int(round(units["busy"])), "kind": "oracle",
               "sample": (f"FP64 oracle at {n}^3 on {units['threads']} threads of "
                          f"{host_threads()} host CPUs ({units['busy']:.1f} kept busy): one "
                          f"transport {units['transport_s']:.1f} s, one objective+gradient "
                          f"{units['gradient_s']:.1f} s, one GN matvec {units['matvec_s']:.1f} s "
                          "(measured, at the converged velocity); value = those unit costs x "
                          "the timed GPU solve's counts (evaluations, Armijo trials, matvecs)"),
               "units": units}

    line = {
        "metric": METRIC, "value": s_per_solve, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{n}^3 ellipsoid phantom pair (seed {SEED}), beta_v continuation "
                               "1e-1..1e-4, rel-grad 5e-2 per level, nt 4, H1 seminorm, FP32, "
                               "two-level zero-velocity preconditioner" +
                               (", PCG parts replayed as CUDA graphs" if args.graphs else ""),
                   "l2": "working set ~%.1f GB > 126 MB L2" % workspace_gb,
                   "parallelism": "replicas" if world > 1 else "single"},
        "matvecs_per_s": matvecs_per_s,
        "spectral_preconditioner": spectral_pc,
        "mixed": mixed,
        "batch": batch,
        "continuation": levels,
        "combined": combined,
        "scale_768": scale,
        "field_gathers_per_registration": gathers,
        "interp_fd_hbm_frac": interp_gbs / peak,
        "interp_fd_gbs": interp_gbs,
        "matvec_interp_fd_hbm_frac": None if matvec_interp_gbs is None else matvec_interp_gbs / peak,
        "matvec_kernels": {k: {"launches_per_matvec": p["launches"] / 10,
                               "gbs": p["timed_bytes"] / (p["ms"] * 1e-3) / 1e9}
                           for k, p in mprof.items() if p["ms"] > 0},
        "solve": {"newton_iters": st0["newton_iters"], "pcg_iters": st0["pcg_iters"],
                  "matvecs": st0["matvecs"], "pde_solves": st0["pde_solves"],
                  "grad_rel": st0["grad_rel"], "mismatch_rel": st0["mismatch_rel"],
                  "inner_iters": st0["inner_iters"], "status": st0["status"]},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None if traffic is None else traffic * n ** 3,
                     "traffic_source": "ncu dram bytes of this kernel source" if traffic
                     else "null: the kernel source changed since the ncu capture",
                     "peak_source": peak_src,
                     "share_of_timed_kernel_time": d["ms"] / total_kernel_ms},
        "kernels": {k: {"launches": p["launches"], "timed": p["timed"], "ms": round(p["ms"], 3),
                        "gbs": (p["timed_bytes"] / (p["ms"] * 1e-3) / 1e9) if p["ms"] > 0
                        else None}
                    for k, p in prof.items() if p["launches"] > 0},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(4 * n ** 3 * 5),
                "d2h_bytes_per_step": int(4 * n ** 3 * 3)},
        "gpu_launches": int(round(launches_per_step)),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_claire(args, world, rank, local)


if __name__ == "__main__":
    main()
