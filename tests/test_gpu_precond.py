"""GPU parity of the two-level zero-velocity preconditioner (Sec. 2.5.6).

The CUDA path (options.precond = 1) against oracle.precond on seeded blob
images, at a 32^3 grid (coarse 16^3) and a non-cubic 48 x 32 x 40 grid.
Tolerances (relative L2, FP32 GPU with nested CG to 1e-6 vs FP64 oracle with
nested CG to 1e-11): preconditioned residual 1e-4; with a constant image or a
purely high-frequency residual the result must equal the spectral
preconditioner to 1e-5; v after 2 GN x 4 PCG 1e-3.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import precond as OP, reduced as OR, solver as OSV, spectral as OS
from paper_2401_17493_b300 import synth

SHAPES = [(32, 32, 32), (48, 32, 40)]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


def _setup(shape, seed=1):
    m0, m1, v = synth.blob_pair(shape, seed=seed, kmax=3, max_disp_voxels=2.0)
    vt = 0.5 * v                                   # evaluate away from v = 0: m(1) != m0
    r = synth.bandlimited_velocity(shape, 6, 1.0, seed + 100)
    return m0, m1, vt, r


@pytest.mark.parametrize("shape", SHAPES)
def test_two_level_preconditioner_matches_oracle(claire, shape):
    m0, m1, vt, r = _setup(shape)
    beta = 1e-3
    with claire.Context(shape, nt=4, beta_v=beta, precond=1, inner_rtol=1e-6,
                        max_inner=300) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        ctx.objective_gradient(dev(vt), want_gradient=False)
        z, its = ctx.precondition(dev(r))
    prob = OR.Problem(_f64(m0), _f64(m1), 4, beta)
    ev = OR.evaluate_objective(prob, _f64(vt))
    z_ref, its_ref = OP.two_level_inverse(_f64(r), ev.m[4], beta, 1.0, 1e-11, 1000)
    assert its > 0 and its_ref > 0
    assert rel(host(z), z_ref) < 1e-4
    # it is not the spectral preconditioner: the coarse data term acts
    assert rel(OS.apply_reg_inverse(_f64(r), beta, 1.0), z_ref) > 1e-2


def test_constant_image_gives_the_spectral_preconditioner(claire):
    shape = (32, 32, 32)
    _, _, vt, r = _setup(shape)
    m = np.full(shape, 0.3, dtype=np.float32)
    with claire.Context(shape, nt=4, beta_v=1e-2, precond=1, inner_rtol=1e-6) as ctx:
        ctx.set_images(dev(m), dev(m))
        ctx.objective_gradient(dev(vt), want_gradient=False)
        z, its = ctx.precondition(dev(r))
        ref = ctx.spectral(claire.OP_REG_INV, dev(r))
    assert its <= 1
    assert rel(host(z), host(ref)) < 1e-5
    assert rel(host(z), OS.apply_reg_inverse(_f64(r), 1e-2, 1.0)) < 1e-5


def test_high_frequency_residual_skips_the_coarse_solve(claire):
    shape = (32, 32, 32)
    m0, m1, vt, _ = _setup(shape, seed=2)
    r = synth.bandlimited_velocity(shape, 12, 1.0, 77)          # modes up to |k| = 12 > n/4
    r = r - OP.prolong3(OP.restrict3(r, OP.coarse_shape(shape)), shape)
    assert np.max(np.abs(r)) > 1e-2
    with claire.Context(shape, nt=4, beta_v=1e-3, precond=1, inner_rtol=1e-6) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        ctx.objective_gradient(dev(vt), want_gradient=False)
        z, _ = ctx.precondition(dev(r))
    assert rel(host(z), OS.apply_reg_inverse(r, 1e-3, 1.0)) < 1e-5


def test_two_gauss_newton_by_four_pcg_match_oracle(claire):
    shape = (32, 32, 32)
    m0, m1, _ = synth.blob_pair(shape, seed=3, kmax=3, max_disp_voxels=2.0)
    beta = 1e-3
    with claire.Context(shape, nt=4, beta_v=beta, max_newton=2, max_pcg=4, fixed_iters=1,
                        precond=1, inner_rtol=1e-6, max_inner=300) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve()
    prob = OR.Problem(_f64(m0), _f64(m1), 4, beta)

    # the oracle with the same fixed nested tolerance (options.inner_rtol)
    import oracle.solver as S
    orig = S.two_level_inverse
    S.two_level_inverse = lambda r, m, a, g, rtol, it, gm_c=None: orig(r, m, a, g, 1e-11, 1000,
                                                                        gm_c=gm_c)
    try:
        vo, so, _ = OSV.gauss_newton(prob, None, OSV.Options(max_newton=2, max_pcg=4,
                                                              fixed_iters=True,
                                                              precond="two_level"))
    finally:
        S.two_level_inverse = orig
    assert st.newton_iters == 2 and st.matvecs == 8 and st.inner_iters > 0
    assert rel(host(v), vo) < 1e-3
    assert abs(st.J - so.J) / so.J < 1e-4


def test_two_level_solve_converges_with_fewer_matvecs(claire):
    shape = (64, 64, 64)
    m0, m1, _ = synth.blob_pair(shape, seed=5, kmax=4, max_disp_voxels=3.0)
    res = {}
    for pc in (0, 1):
        with claire.Context(shape, nt=4, beta_v=1e-3, precond=pc) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            v, st = ctx.solve()
        assert st.status == claire.OK and st.grad_rel <= 5e-2
        res[pc] = st
    assert res[1].inner_iters > 0 and res[0].inner_iters == 0
    assert res[1].matvecs < res[0].matvecs


def test_two_level_in_mixed_precision_converges(claire):
    shape = (64, 64, 64)
    m0, m1, _ = synth.blob_pair(shape, seed=6, kmax=4, max_disp_voxels=3.0)
    with claire.Context(shape, nt=4, beta_v=1e-3, precond=1, precision=1) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve()
    assert st.status == claire.OK and st.grad_rel <= 5e-2 and st.inner_iters > 0


def test_two_level_errors(claire):
    with claire.Context((36, 32, 32)) as ctx:            # 36 % 4 == 0 is fine
        ctx.set_options(precond=1)
        with pytest.raises(claire.ClaireError) as e:       # no evaluation yet
            ctx.precondition(torch.zeros((3, 36, 32, 32), device="cuda"))
        assert e.value.status == claire.EORDER
    with claire.Context((34, 32, 32)) as ctx:            # 34 / 2 is odd
        with pytest.raises(claire.ClaireError) as e:
            ctx.set_options(precond=1)
        assert e.value.status == claire.EINVAL
        with pytest.raises(claire.ClaireError) as e:
            ctx.set_options(precond=3)
        assert e.value.status == claire.EINVAL
        ctx.set_options(precond=2)                        # automatic: spectral here


def test_automatic_preconditioner_is_the_default(claire):
    """options.precond = 2 (the default) is the two-level preconditioner on grids whose
    sizes are multiples of 4 and the spectral one otherwise."""
    for shape, expect_two_level in (((32, 32, 32), True), ((34, 32, 32), False)):
        m0, m1, vt, r = _setup(shape)
        with claire.Context(shape, nt=4, beta_v=1e-3) as ctx:
            assert ctx.opts.precond == 2
            ctx.set_images(dev(m0), dev(m1))
            ctx.objective_gradient(dev(vt), want_gradient=False)
            z, its = ctx.precondition(dev(r))
            ref = ctx.spectral(claire.OP_REG_INV, dev(r))
        if expect_two_level:
            assert its > 0 and rel(host(z), host(ref)) > 1e-2
        else:
            assert its == 0 and rel(host(z), host(ref)) < 1e-6
