"""options.warm_check: the initial-guess test of a learned warm start inside the solver.

* A guess that raises the objective (J(v0) > J(0), the distance of the template)
  is rejected: the solve restarts from v = 0 and returns bitwise the zero-initialised
  solve, with stats.warm_fallback = 1, in claire_solve and in claire_solve_batch.
* An accepted guess gives bitwise the solve without the check from the same guess,
  with the same PDE-solve count (its evaluation is the solver's first one).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2401_17493_b300 import synth

SHAPE = (32, 32, 32)


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


@pytest.fixture(scope="module")
def pair(claire):
    """(m0, m1, a guess below J(0), a guess above J(0)).  The good guess is 0.9 times
    the iterate after one Gauss-Newton step (Armijo lowered J below J(0)); the bad
    one is -3 times the generating velocity."""
    m0, m1, v = synth.blob_pair(SHAPE, seed=11, kmax=3, max_disp_voxels=2.0)
    m0, m1 = dev(m0), dev(m1)
    with claire.Context(SHAPE, nt=4, beta_v=1e-2, max_newton=1) as ctx:
        ctx.set_images(m0, m1)
        v1, st = ctx.solve()
    assert st.newton_iters == 1
    return m0, m1, 0.9 * v1, dev(-3.0 * v)


def _ctx(claire, m0, m1, precision, **kw):
    ctx = claire.Context(SHAPE, nt=4, beta_v=1e-2, precision=precision, **kw)
    ctx.set_images(m0, m1)
    return ctx


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("given_gnorm0", [True, False])
def test_rejected_guess_gives_the_zero_initialised_solve(claire, pair, precision,
                                                         given_gnorm0):
    m0, m1, _, v_bad = pair
    with _ctx(claire, m0, m1, precision) as ctx:
        J0, g0 = ctx.objective_gradient(torch.zeros_like(v_bad))
        Jb, _ = ctx.objective_gradient(v_bad, want_gradient=False)
        assert Jb > J0
        gn = float(g0.abs().max()) if given_gnorm0 else 0.0
        ctx.set_options(gnorm0=gn)
        vz, sz = ctx.solve(torch.zeros_like(v_bad))
        ctx.set_options(warm_check=1)
        vw, sw = ctx.solve(v_bad.clone())
    assert sz.warm_fallback == 0 and sw.warm_fallback == 1
    assert sw.status == claire.OK and sw.matvecs == sz.matvecs
    assert torch.equal(vw, vz)


@pytest.mark.parametrize("precision", [0, 1])
def test_accepted_guess_changes_nothing(claire, pair, precision):
    m0, m1, v_good, _ = pair
    with _ctx(claire, m0, m1, precision) as ctx:
        J0, g0 = ctx.objective_gradient(torch.zeros_like(v_good))
        Jg, _ = ctx.objective_gradient(v_good, want_gradient=False)
        assert Jg < J0
        ctx.set_options(gnorm0=float(g0.abs().max()))
        v1, s1 = ctx.solve(v_good.clone())
        ctx.set_options(warm_check=1)
        v2, s2 = ctx.solve(v_good.clone())
    assert s2.warm_fallback == 0
    assert (s2.matvecs, s2.newton_iters, s2.pde_solves) == (s1.matvecs, s1.newton_iters,
                                                            s1.pde_solves)
    assert torch.equal(v2, v1)


def test_batch_applies_the_check_per_pair(claire, pair):
    m0, m1, v_good, v_bad = pair
    ref = []
    for v0 in (v_good, torch.zeros_like(v_good)):
        with _ctx(claire, m0, m1, 0) as ctx:
            ref.append(ctx.solve(v0.clone())[0])
    ctxs = [_ctx(claire, m0, m1, 0, warm_check=1, graphs=1) for _ in range(2)]
    try:
        vs, stats = claire.solve_batch(ctxs, [v_good.clone(), v_bad.clone()])
    finally:
        for c in ctxs:
            c.close()
    assert [s.warm_fallback for s in stats] == [0, 1]
    assert torch.equal(vs[0], ref[0]) and torch.equal(vs[1], ref[1])
