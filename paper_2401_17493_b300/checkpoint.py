"""Checkpointed continuation: resume a registration after an interruption.

Runs the beta_v continuation (Sec. 2.6) one level per library call and writes,
after each level, the velocity (``level_<i>.npy``, [3][n1][n2][n3] FP32) and a
JSON record (``levels.json``: the betas, the relative-gradient denominator
||g(v = 0)||_inf of level 0 and every finished level's stats) into a
directory.  A later call with the same directory skips the levels already
written and starts from the last saved velocity with the same denominator, so
a resumed run takes the same stopping decisions and returns bitwise the result
of an uninterrupted checkpointed run.  Files are replaced atomically, so an
interruption leaves either the old or the new record of a level.

Against one claire_solve_continuation call, every level after the first
re-evaluates J and g at its starting velocity (two PDE solves) instead of
reusing the previous level's evaluation.
"""

import json
import os

import numpy as np


def _save_npy(path, arr):
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.save(f, arr)
    os.replace(tmp, path)


def _save_json(path, obj):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(obj, f, indent=1)
    os.replace(tmp, path)


def solve_checkpointed(ctx, betas, directory, v=None):
    """Continuation over betas on Context ctx (images already set), checkpointed
    in directory.  Returns (v, record) with record the content of levels.json."""
    import torch
    betas = [float(b) for b in betas]
    os.makedirs(directory, exist_ok=True)
    meta_path = os.path.join(directory, "levels.json")
    if os.path.exists(meta_path):
        with open(meta_path) as f:
            meta = json.load(f)
        if meta["betas"] != betas or tuple(meta["shape"]) != tuple(ctx.shape):
            raise ValueError(f"{directory} holds a run with other betas or another grid")
    else:
        meta = {"betas": betas, "shape": list(ctx.shape), "gnorm0": None, "levels": []}
    device = getattr(ctx, "device", "cuda")
    done = len(meta["levels"])
    if done:
        v = torch.from_numpy(np.load(os.path.join(directory, f"level_{done - 1}.npy"))).to(device)
    elif v is None:
        v = torch.zeros(ctx.vshape, dtype=torch.float32, device=device)
    saved_gnorm0 = ctx.opts.gnorm0
    try:
        for i in range(done, len(betas)):
            if meta["gnorm0"] is not None:
                ctx.set_options(gnorm0=meta["gnorm0"])
            v, st = ctx.solve_continuation([betas[i]], v)
            if meta["gnorm0"] is None:
                meta["gnorm0"] = float(st.gnorm0)
            _save_npy(os.path.join(directory, f"level_{i}.npy"), v.detach().cpu().numpy())
            rec = {"level": i, "beta_v": betas[i]}
            rec.update({k: (float(x) if isinstance(x, float) else x)
                        for k, x in st.as_dict().items()})
            meta["levels"].append(rec)
            _save_json(meta_path, meta)
    finally:
        ctx.set_options(gnorm0=saved_gnorm0)
    return v, meta
