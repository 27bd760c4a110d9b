"""The three SL gather variants give bitwise the same values.

The register-window gather (each lane keeps four x1 tap planes in registers
and contracts the nodes that share its reference floor; the others go through
a deferred queue) and the 64-shared-load brick gather, from a brick staged by
TMA tiled loads or by the threads' cp.async copies, evaluate every node with
the same taps in the same FP32 order, so every SL step, trace, adjoint factor
and every quantity built from them must agree bit for bit, for every brick
depth, on ragged grids (partial tiles along every axis), on a grid whose x3
extent is not a multiple of 4 (scalar staging path), on grids with interior
x3 tiles (TMA-staged bricks beside cp.async-staged edge bricks; with n3 % 8 ==
0 also for the FP16 fields of the mixed form), and for
displacements from sub-voxel to many periods (global-memory gathers).  The
oracle parity of the default variant is covered by the other GPU tests (the
256^3 sampled cases stage most bricks by TMA).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2401_17493_b300 import synth

SHAPES = [(22, 18, 40), (18, 20, 34), (64, 64, 64), (20, 22, 100), (40, 36, 136)]
VARIANTS = [(0, 8), (1, 4), (1, 8), (1, 16), (0, 4), (2, 8), (2, 16), (0, 16)]


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _displacements(shape, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "smooth":                    # band-limited, under a voxel per step
        v = synth.bandlimited_velocity(shape, 3, 0.9, seed)
        return (v / (2 * np.pi / np.array(shape, dtype=float))[:, None, None, None]).astype(
            np.float32)
    if kind == "uniform":                   # every floor of the staged halo and beyond
        return rng.uniform(-3.7, 3.7, size=(3,) + shape).astype(np.float32)
    d = rng.uniform(-1.2, 1.2, size=(3,) + shape)
    far = rng.random(shape) < 0.05          # a few departure points many periods away
    d[:, far] = rng.uniform(-90, 90, size=(3, int(far.sum())))
    return d.astype(np.float32)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["smooth", "uniform", "wrap"])
def test_interpolation_variants_are_bitwise_equal(claire, shape, kind):
    rng = np.random.default_rng(7)
    u = dev(rng.standard_normal(shape))
    d = dev(_displacements(shape, kind, 3))
    outs = []
    with claire.Context(shape) as ctx:
        for w, t1 in VARIANTS:
            ctx.set_tuning(w, t1, 32)
            assert ctx.tuning() == (w, t1, 32)
            outs.append(ctx.interp(u, d).clone())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    assert claire.wait_status() == 0             # no bounded brick wait ran out


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("scale", [0.3, 1.0, 6.0])
def test_trace_variants_are_bitwise_equal(claire, shape, scale):
    v = dev(scale * synth.bandlimited_velocity(shape, 3, 2.0, 11))
    res = []
    with claire.Context(shape, nt=4) as ctx:
        for w, t1 in VARIANTS:
            ctx.set_tuning(w, t1, 32)
            df, db = ctx.trace(v)
            res.append((df.clone(), db.clone()))
    for df, db in res[1:]:
        assert torch.equal(df, res[0][0]) and torch.equal(db, res[0][1])


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", [0, 1])
def test_gradient_and_matvec_variants_are_bitwise_equal(claire, shape, precision):
    m0, m1, v = synth.blob_pair(shape, seed=2, kmax=3, max_disp_voxels=2.5)
    vt = dev(synth.bandlimited_velocity(shape, 3, 1.0, 12))
    res = []
    with claire.Context(shape, nt=4, beta_v=1e-2, precision=precision) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        for w, t1 in VARIANTS:
            ctx.set_tuning(w, t1, 32)
            J, g = ctx.objective_gradient(dev(0.7 * v))
            Hv = ctx.hessian_matvec(vt)
            m = ctx.transport(dev(0.7 * v))
            res.append((J, g.clone(), Hv.clone(), m.clone()))
    for J, g, Hv, m in res[1:]:
        assert J == res[0][0]
        assert torch.equal(g, res[0][1]) and torch.equal(Hv, res[0][2])
        assert torch.equal(m, res[0][3])


def test_solve_variants_are_bitwise_equal(claire):
    shape = (32, 32, 32)
    m0, m1, _ = synth.blob_pair(shape, seed=4, kmax=3, max_disp_voxels=2.0)
    vs = []
    for w in (0, 1, 2):
        with claire.Context(shape, nt=4, beta_v=1e-2, precond=1, max_inner=10) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            ctx.set_tuning(w, 8, 32)
            v, st = ctx.solve()
            vs.append((v.clone(), st.matvecs, st.newton_iters))
    for other in vs[1:]:
        assert torch.equal(vs[0][0], other[0]) and vs[0][1:] == other[1:]


def test_tuning_rejects_unknown_shapes(claire):
    with claire.Context((16, 16, 16)) as ctx:
        for bad in [(3, 8, 32), (-1, 8, 32), (1, 12, 32), (1, 8, 24)]:
            with pytest.raises(claire.ClaireError):
                ctx.set_tuning(*bad)
        assert ctx.tuning() == (0, 8, 32)


def test_tuning_change_after_graph_capture_gives_the_same_solve(claire):
    """Captured PCG graphs bake the launch shapes: set_tuning drops them, and the
    next solve (re-captured with the new shapes) is bitwise the first one."""
    shape = (32, 32, 32)
    m0, m1, _ = synth.blob_pair(shape, seed=6, kmax=3, max_disp_voxels=2.0)
    with claire.Context(shape, nt=4, beta_v=1e-2, precond=1, max_inner=10, graphs=1) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v1, s1 = ctx.solve()
        v1 = v1.clone()
        ctx.set_tuning(1, 4, 16)
        v2, s2 = ctx.solve()
        ctx.set_tuning(0, 16, 64)
        v3, s3 = ctx.solve()
        ctx.set_tuning(2, 8, 32)
        v4, s4 = ctx.solve()
    assert torch.equal(v1, v2) and torch.equal(v1, v3) and torch.equal(v1, v4)
    assert s1.matvecs == s2.matvecs == s3.matvecs == s4.matvecs
