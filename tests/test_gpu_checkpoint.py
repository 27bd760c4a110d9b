"""Checkpointed continuation on the GPU (paper_2401_17493_b300.checkpoint).

* A run interrupted after level 1 (its last level file and record removed) and
  resumed in a fresh context returns bitwise the velocity and the same per-level
  counters as the uninterrupted checkpointed run.
* The checkpointed run meets the tolerance on every level and stays within 1e-3
  (relative L2) of one claire_solve_continuation call, which reuses each
  level's evaluation instead of re-evaluating at the level's start.
"""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2401_17493_b300 import synth

SHAPE = (32, 32, 32)
BETAS = [1e-1, 1e-2, 1e-3]


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


def _ctx(claire, m0, m1):
    ctx = claire.Context(SHAPE, nt=4, beta_v=BETAS[0])
    ctx.set_images(torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda())
    return ctx


def test_resumed_run_equals_uninterrupted_run(claire, tmp_path):
    from paper_2401_17493_b300 import checkpoint
    m0, m1, _ = synth.blob_pair(SHAPE, seed=9, kmax=3, max_disp_voxels=2.0)
    with _ctx(claire, m0, m1) as ctx:
        va, meta_a = checkpoint.solve_checkpointed(ctx, BETAS, str(tmp_path / "a"))
        vs, st = ctx.solve_continuation(BETAS)
    assert all(r["grad_rel"] <= 5e-2 and r["status"] == claire.OK for r in meta_a["levels"])
    rel = float(torch.linalg.norm(va - vs) / torch.linalg.norm(vs))
    assert rel < 1e-3

    # interrupted after level 1: the files of level 2 never got written
    b = tmp_path / "b"
    with _ctx(claire, m0, m1) as ctx:
        checkpoint.solve_checkpointed(ctx, BETAS[:2] + [BETAS[2]], str(b))
    os.remove(b / "level_2.npy")
    meta = json.loads((b / "levels.json").read_text())
    meta["levels"] = meta["levels"][:2]
    (b / "levels.json").write_text(json.dumps(meta))
    with _ctx(claire, m0, m1) as ctx:
        vb, meta_b = checkpoint.solve_checkpointed(ctx, BETAS, str(b))
    assert torch.equal(vb, va)
    keys = ("newton_iters", "matvecs", "pde_solves", "status")
    assert [[r[k] for k in keys] for r in meta_b["levels"]] == \
        [[r[k] for k in keys] for r in meta_a["levels"]]
    assert np.array_equal(np.load(b / "level_2.npy"), va.cpu().numpy())
