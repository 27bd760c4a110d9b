"""Batched solves over uneven grids, CUDA-graph PCG iterations and the
autotuner: each must give the same registrations as the plain sequential
per-pair solve (the kernels are deterministic; graph replay runs the same
launches; tile shapes change only the block partition of the FP64 sums)."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2401_17493_b300 import synth

SHAPES = [(32, 32, 32), (48, 40, 34), (64, 64, 64), (40, 48, 56)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


def _contexts(C, **opts):
    ctxs = []
    for i, shape in enumerate(SHAPES):
        m0, m1, _ = synth.blob_pair(shape, seed=100 + i, kmax=3, max_disp_voxels=2.0)
        ctx = C.Context(shape, nt=4, beta_v=5e-3, **opts)
        ctx.set_images(dev(m0), dev(m1))
        ctxs.append(ctx)
    return ctxs


def test_batched_solve_equals_sequential_solves(claire):
    seq = []
    for ctx in _contexts(claire):
        v, st = ctx.solve()
        seq.append((v.cpu().numpy(), st.matvecs, st.status))
        ctx.close()
    ctxs = _contexts(claire)
    vs, stats = claire.solve_batch(ctxs)
    for (vref, mv, status), v, st in zip(seq, vs, stats):
        assert st.status == status and st.matvecs == mv
        assert np.array_equal(v.cpu().numpy(), vref)
    for c in ctxs:
        c.close()


def test_batched_continuation(claire):
    betas = [5e-2, 5e-3]
    ctxs = _contexts(claire)
    vs, stats = claire.solve_batch(ctxs, betas=betas, max_threads=2)
    for ctx, v, st in zip(ctxs, vs, stats):
        assert st.grad_rel <= 5e-2 and st.J < st.J0
        v2, st2 = ctx.solve_continuation(betas)
        assert np.array_equal(v.cpu().numpy(), v2.cpu().numpy())
        ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replayed_pcg_equals_launch_by_launch(claire, precision):
    shape = SHAPES[1]
    m0, m1, _ = synth.blob_pair(shape, seed=7, kmax=3, max_disp_voxels=2.0)
    out = []
    for graphs in (0, 1):
        with claire.Context(shape, nt=4, beta_v=1e-2, graphs=graphs, precision=precision) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            v, st = ctx.solve_continuation([1e-1, 1e-2])
            torch.cuda.synchronize()
            out.append((v.cpu().numpy(), st.matvecs, st.pcg_iters))
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("precision,inner", [(0, {}), (1, {}), (0, dict(max_inner=3)),
                                              (0, dict(inner_rtol=1e-4, max_inner=40))])
def test_graph_nested_cg_equals_host_loop(claire, precision, inner):
    """With the two-level preconditioner a captured PCG part B holds the nested CG
    as a conditional while node driven on the device: same iterates (bitwise), same
    outer and nested iteration counts as the host-driven loop, also when the
    iteration cap or a fixed tolerance ends the nested solves."""
    shape = (48, 32, 40)
    m0, m1, _ = synth.blob_pair(shape, seed=9, kmax=3, max_disp_voxels=2.5)
    out = []
    for graphs in (0, 1):
        with claire.Context(shape, nt=4, beta_v=1e-3, graphs=graphs, precision=precision,
                            precond=1, **inner) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            v, st = ctx.solve_continuation([1e-1, 1e-2, 1e-3])
            torch.cuda.synchronize()
            out.append((v.cpu().numpy(), st.matvecs, st.pcg_iters, st.inner_iters))
    assert out[0][3] > 0 and out[0][2] > 1
    assert out[0][1:] == out[1][1:]
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("opts", [dict(distance=1), dict(hessian=1), dict(beta_w=1e-3),
                                  dict(precision=1, precond=0)])
def test_graph_replay_equals_launch_by_launch_in_every_mode(claire, opts):
    """Graph replay is bitwise launch-by-launch execution also with the NCC distance,
    full Newton, the near-incompressible term and mixed precision with the spectral
    preconditioner."""
    shape = (32, 32, 32)
    m0, m1, _ = synth.blob_pair(shape, seed=27, kmax=3, max_disp_voxels=2.0)
    out = []
    for graphs in (0, 1):
        with claire.Context(shape, nt=4, beta_v=1e-3, graphs=graphs, **opts) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            v, st = ctx.solve_continuation([1e-2, 1e-3])
            torch.cuda.synchronize()
            out.append((v.cpu().numpy(), st.matvecs, st.pcg_iters, st.inner_iters, st.status))
    assert out[0][1:] == out[1][1:]
    assert np.array_equal(out[0][0], out[1][0])


def test_graph_replays_are_counted_like_launches(claire):
    """The launch accounting of a solve is the same with and without graphs: captured
    parts count their kernels per replay, the nested CG's while-node body per device
    iteration (read back with the PCG scalars).  The preconditioner class differs by
    design: the device loop adds its begin and control kernels and updates the
    direction after the last iteration too."""
    shape = (32, 32, 32)
    m0, m1, _ = synth.blob_pair(shape, seed=23, kmax=3, max_disp_voxels=2.0)
    counts = []
    for graphs in (0, 1):
        with claire.Context(shape, nt=4, beta_v=1e-3, graphs=graphs, precond=1) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            ctx.solve()                                # captures the graphs
            ctx.profile_reset(timing=False)
            _, st = ctx.solve()
            prof = ctx.profile_read()
        counts.append({k: (p["launches"], round(p["bytes"])) for k, p in prof.items()})
        assert st.inner_iters > 0
    host, graph = counts
    assert graph["precond"][0] > host["precond"][0] > 0
    del host["precond"], graph["precond"]
    assert host == graph


@pytest.mark.parametrize("precision", [0, 1])
def test_reused_context_equals_fresh_context(claire, precision):
    """A context reused for another pair (set_images, a new gnorm0, the captured graphs
    kept) gives bitwise the registration of a fresh context."""
    shape = (32, 32, 32)
    pairs = [synth.blob_pair(shape, seed=s, kmax=3, max_disp_voxels=2.0)[:2] for s in (21, 22)]
    opts = dict(nt=4, beta_v=1e-2, graphs=1, precision=precision, precond=1)
    with claire.Context(shape, **opts) as ctx:
        ctx.set_images(dev(pairs[0][0]), dev(pairs[0][1]))
        ctx.solve()
        ctx.set_images(dev(pairs[1][0]), dev(pairs[1][1]))
        ctx.set_options(gnorm0=0.5)
        v_reused, st_reused = ctx.solve()
    with claire.Context(shape, gnorm0=0.5, **opts) as ctx:
        ctx.set_images(dev(pairs[1][0]), dev(pairs[1][1]))
        v_fresh, st_fresh = ctx.solve()
    assert st_reused.matvecs == st_fresh.matvecs and st_reused.inner_iters == st_fresh.inner_iters
    assert torch.equal(v_reused, v_fresh)


def test_autotuner_picks_valid_shapes_and_keeps_results(claire):
    shape = SHAPES[2]
    m0, m1, _ = synth.blob_pair(shape, seed=8, kmax=3, max_disp_voxels=2.0)
    with claire.Context(shape, nt=4, beta_v=1e-2, max_newton=2, max_pcg=8,
                        fixed_iters=1, precond=0) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v0, _ = ctx.solve()
        sl_t1, march_t1 = ctx.autotune()
        assert sl_t1 in (4, 8, 16) and march_t1 in (8, 16, 32, 64)
        v1, _ = ctx.solve()
    a, b = v1.cpu().numpy(), v0.cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5


GROUP_SHAPES = SHAPES + [(40, 36, 136)]        # the last one with TMA-staged interior bricks


def _group_contexts(C, precisions, **opts):
    ctxs = []
    for i, (shape, prec) in enumerate(zip(GROUP_SHAPES, precisions)):
        m0, m1, _ = synth.blob_pair(shape, seed=300 + i, kmax=3, max_disp_voxels=2.0)
        ctx = C.Context(shape, nt=4, beta_v=5e-3, precision=prec, **opts)
        ctx.set_images(dev(m0), dev(m1))
        ctxs.append(ctx)
    return ctxs


@pytest.mark.parametrize("precisions", [(0, 0, 0, 0, 0), (0, 1, 0, 1, 0)])
def test_grouped_batch_equals_sequential_solves(claire, precisions):
    """One persistent launch per SL / trace / FD8 march phase for all pairs of the
    batch gives every pair bitwise its sequential registration; mixed-precision
    pairs keep their FP16 kernels on their own streams, beside the grouped FP32
    ones.  Graph capture is set on the contexts and suspended for the batch."""
    seq = []
    for ctx in _group_contexts(claire, precisions, graphs=1):
        v, st = ctx.solve()
        seq.append((v.cpu().numpy(), st.matvecs, st.status, st.newton_iters))
        ctx.close()
    ctxs = _group_contexts(claire, precisions, graphs=1)
    vs, stats, launches = claire.solve_batch(ctxs, grouped=True)
    for (vref, mv, status, nit), v, st in zip(seq, vs, stats):
        assert st.status == status and st.matvecs == mv and st.newton_iters == nit
        assert np.array_equal(v.cpu().numpy(), vref)
    # each grouped launch stands for the launches of several pairs
    grouped_launches, replaced = launches
    assert 0 < grouped_launches < replaced
    for c in ctxs:
        o = claire.Options()
        assert c.lib.claire_get_options(c.h, ctypes.byref(o)) == claire.OK
        assert o.graphs == 1                        # restored after the batch
        c.close()
    assert claire.wait_status() == 0


def test_grouped_batch_continuation_and_reuse(claire):
    """Continuation levels through the grouped batch equal the per-context
    continuation, and the contexts stay usable for ungrouped solves afterwards."""
    betas = [5e-2, 5e-3]
    ctxs = _group_contexts(claire, (0, 0, 0, 0, 0))
    vs, stats, _ = claire.solve_batch(ctxs, betas=betas, grouped=True)
    for ctx, v, st in zip(ctxs, vs, stats):
        assert st.grad_rel <= 5e-2 and st.J < st.J0
        v2, st2 = ctx.solve_continuation(betas)
        assert np.array_equal(v.cpu().numpy(), v2.cpu().numpy())
        ctx.close()


TUNINGS = [(0, 4, 16), (2, 16, 32), (0, 8, 64), (0, 16, 8), (2, 4, 32)]


def test_grouped_batch_with_per_pair_tile_shapes(claire):
    """Pairs with different gather variants, brick depths and march depths share
    grouped launches (the launch's shared memory sized for the deepest brick, one
    TMA box shape per pair): each pair still equals its own sequential solve with
    the same shapes, bitwise."""
    seq = []
    for ctx, tune in zip(_group_contexts(claire, (0,) * 5), TUNINGS):
        ctx.set_tuning(*tune)
        v, st = ctx.solve()
        seq.append((v.cpu().numpy(), st.matvecs))
        ctx.close()
    ctxs = _group_contexts(claire, (0,) * 5)
    for ctx, tune in zip(ctxs, TUNINGS):
        ctx.set_tuning(*tune)
    for wait_us in (-1, 10):
        vs, stats, _ = claire.solve_batch(ctxs, grouped=True, wait_us=wait_us)
        for (vref, mv), v, st in zip(seq, vs, stats):
            assert st.matvecs == mv
            assert np.array_equal(v.cpu().numpy(), vref)
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("wait_us", [-1, 10])
def test_grouped_batch_survives_a_failing_pair(claire, wait_us):
    """A pair whose objective is not finite (NaN in its reference image) fails
    after it has posted grouped launches; its thread leaves the group, the other
    pairs finish with their sequential results and the call reports ENONFINITE."""
    seq = []
    for ctx in _group_contexts(claire, (0,) * 5):
        v, _ = ctx.solve()
        seq.append(v.cpu().numpy())
        ctx.close()
    ctxs = _group_contexts(claire, (0,) * 5)
    bad = 2
    shape = GROUP_SHAPES[bad]
    m0, m1, _ = synth.blob_pair(shape, seed=300 + bad, kmax=3, max_disp_voxels=2.0)
    m1 = m1.copy()
    m1[1, 2, 3] = np.nan
    ctxs[bad].set_images(dev(m0), dev(m1))
    vs = [torch.zeros(c.vshape, device="cuda") for c in ctxs]
    with pytest.raises(claire.ClaireError) as e:
        claire.solve_batch(ctxs, vs, grouped=True, wait_us=wait_us)
    assert e.value.status == claire.ENONFINITE
    for i, (v, vref) in enumerate(zip(vs, seq)):
        if i != bad:
            assert np.array_equal(v.cpu().numpy(), vref)
    for c in ctxs:
        c.close()
