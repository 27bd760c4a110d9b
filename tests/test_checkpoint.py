"""Host logic of the checkpointed continuation (paper_2401_17493_b300.checkpoint),
on a fake context: levels written one by one, the level-0 denominator reused by
later levels, resume after an interruption from the last saved level with the
same result, the caller's options restored, and a directory of another run
refused.  The GPU path is covered in tests/test_gpu_checkpoint.py."""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2401_17493_b300 import checkpoint
from paper_2401_17493_b300.claire import Stats

BETAS = [1e-1, 1e-2, 1e-3]
SHAPE = (4, 6, 8)


class FakeContext:
    """Each level adds beta to v; fails on purpose at the level fail_at."""
    device = "cpu"

    def __init__(self, fail_at=None):
        self.shape = SHAPE
        self.vshape = (3,) + SHAPE
        self.opts = Stats()          # any struct with a gnorm0 field
        self.opts.gnorm0 = -1.0
        self.calls = []
        self.fail_at = fail_at

    def set_options(self, **kw):
        for k, x in kw.items():
            setattr(self.opts, k, x)

    def solve_continuation(self, betas, v):
        assert len(betas) == 1
        level = len(self.calls)
        if self.fail_at is not None and level == self.fail_at:
            raise RuntimeError("interrupted")
        self.calls.append((betas[0], self.opts.gnorm0, v.clone()))
        st = Stats()
        st.gnorm0 = 7.5 if self.opts.gnorm0 <= 0 else self.opts.gnorm0
        st.newton_iters = level + 1
        return v + betas[0], st


def _after(v0, n):
    v = v0.clone()
    for b in BETAS[:n]:
        v = v + b
    return v


def test_levels_are_written_and_the_denominator_is_kept(tmp_path):
    ctx = FakeContext()
    v0 = torch.full((3,) + SHAPE, 0.25)
    v, meta = checkpoint.solve_checkpointed(ctx, BETAS, str(tmp_path), v0)
    assert torch.equal(v, _after(v0, 3))
    assert [c[0] for c in ctx.calls] == BETAS
    assert [c[1] for c in ctx.calls] == [-1.0, 7.5, 7.5]
    assert ctx.opts.gnorm0 == -1.0                       # the caller's option is restored
    assert meta["gnorm0"] == 7.5 and [r["level"] for r in meta["levels"]] == [0, 1, 2]
    for i in range(3):
        saved = np.load(os.path.join(tmp_path, f"level_{i}.npy"))
        assert np.array_equal(saved, _after(v0, i + 1).numpy())
    with open(os.path.join(tmp_path, "levels.json")) as f:
        assert json.load(f) == meta
    assert not [p for p in os.listdir(tmp_path) if p.endswith(".tmp")]


def test_resume_after_an_interruption_gives_the_same_result(tmp_path):
    v0 = torch.zeros((3,) + SHAPE)
    ref, _ = checkpoint.solve_checkpointed(FakeContext(), BETAS, str(tmp_path / "a"), v0)
    broken = FakeContext(fail_at=2)
    with pytest.raises(RuntimeError):
        checkpoint.solve_checkpointed(broken, BETAS, str(tmp_path / "b"), v0)
    assert broken.opts.gnorm0 == -1.0
    assert sorted(os.listdir(tmp_path / "b")) == ["level_0.npy", "level_1.npy", "levels.json"]
    again = FakeContext()
    v, meta = checkpoint.solve_checkpointed(again, BETAS, str(tmp_path / "b"))
    assert len(again.calls) == 1                          # only the missing level runs
    beta, g0, start = again.calls[0]
    assert beta == BETAS[2] and g0 == 7.5
    assert torch.equal(start, _after(v0, 2))              # from the last saved velocity
    assert torch.equal(v, ref)
    assert [r["level"] for r in meta["levels"]] == [0, 1, 2]
    # a finished directory runs nothing more
    done = FakeContext()
    v2, _ = checkpoint.solve_checkpointed(done, BETAS, str(tmp_path / "b"))
    assert done.calls == [] and torch.equal(v2, ref)


def test_directory_of_another_run_is_refused(tmp_path):
    checkpoint.solve_checkpointed(FakeContext(), BETAS, str(tmp_path))
    with pytest.raises(ValueError):
        checkpoint.solve_checkpointed(FakeContext(), BETAS[:2], str(tmp_path))
