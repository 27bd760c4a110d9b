"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Every row of the hot path is compared element by element on seeded inputs at
sizes the oracle finishes in seconds, on a ragged shape (22 x 18 x 40 does not
divide the 32 x 4 x 2 thread blocks) and on the 64^3 parity workload.
Tolerances (relative L2, FP32 GPU vs FP64 oracle): transport and objective
1e-5, gradient and Hessian matvec 1e-4, v after 2 GN x 10 PCG 1e-3; single
kernels (interpolation, FD8, spectral) 1e-5.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import interp as OI, fd8 as OF, spectral as OS, transport as OT
from oracle import reduced as OR, solver as OSV, defgrad as ODG
from paper_2401_17493_b300 import synth

RAGGED = (22, 18, 40)
CUBE = (64, 64, 64)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


def _pair(shape, seed=1, kmax=4, disp=3.0):
    m0, m1, v = synth.blob_pair(shape, seed=seed, kmax=kmax, max_disp_voxels=disp)
    return m0, m1, v


def _f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("shape", [RAGGED, CUBE])
def test_trace_matches_oracle_departure_points(claire, shape):
    _, _, v = _pair(shape)
    with claire.Context(shape, nt=4) as ctx:
        df, db = ctx.trace(dev(v))
    base = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij"))
    ref_f = OT.departure_points(_f64(v), 4, +1) - base
    ref_b = OT.departure_points(_f64(v), 4, -1) - base
    assert rel(host(df), ref_f) < 1e-5
    assert rel(host(db), ref_b) < 1e-5


@pytest.mark.parametrize("shape", [RAGGED, CUBE])
def test_interpolation_matches_oracle(claire, shape):
    rng = np.random.default_rng(0)
    u = rng.standard_normal(shape).astype(np.float32)
    d = rng.uniform(-3.7, 3.7, size=(3,) + shape).astype(np.float32)
    with claire.Context(shape) as ctx:
        out = ctx.interp(dev(u), dev(d))
    base = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij"))
    ref = OI.interp(_f64(u), base + _f64(d))
    assert rel(host(out), ref) < 1e-5


def test_interpolation_with_zero_displacement_is_bitwise_identity(claire):
    rng = np.random.default_rng(1)
    u = rng.standard_normal(RAGGED).astype(np.float32)
    with claire.Context(RAGGED) as ctx:
        out = ctx.interp(dev(u), torch.zeros((3,) + RAGGED, device="cuda"))
    assert np.array_equal(out.cpu().numpy(), u)


def test_interpolation_wraps_large_displacements(claire):
    rng = np.random.default_rng(2)
    u = rng.standard_normal(RAGGED).astype(np.float32)
    d = rng.uniform(-60.0, 60.0, size=(3,) + RAGGED).astype(np.float32)
    with claire.Context(RAGGED) as ctx:
        out = ctx.interp(dev(u), dev(d))
    base = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in RAGGED], indexing="ij"))
    assert rel(host(out), OI.interp(_f64(u), base + _f64(d))) < 1e-5


def test_far_node_count_matches_the_departure_points(claire):
    """claire_far_nodes counts the nodes whose departure points leave the staged SL
    brick (floor of d outside [-2, 1] on x1 and x2, [-3, 2] on x3): exactly the
    count of the trace's own departure points, zero for small displacements."""
    m0, m1, _ = _pair(RAGGED, seed=3)

    def outside(d):
        p = np.floor(d.cpu().numpy())
        return int(((p[0] < -2) | (p[0] > 1) | (p[1] < -2) | (p[1] > 1) |
                    (p[2] < -3) | (p[2] > 2)).sum())

    for disp in (0.5, 12.0):                  # voxels per unit time; n_t = 4 steps
        v = synth.bandlimited_velocity(RAGGED, 3, disp, 21).astype(np.float32)
        with claire.Context(RAGGED, nt=4) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            with pytest.raises(claire.ClaireError) as e:
                ctx.far_nodes()
            assert e.value.status == claire.EORDER
            ctx.objective_gradient(dev(v))
            fwd, bwd = ctx.far_nodes()
            df, db = ctx.trace(dev(v))
        assert (fwd, bwd) == (outside(df), outside(db))
        if disp < 1.0:
            assert fwd == 0 and bwd == 0
        else:
            assert fwd > 0 and bwd > 0


@pytest.mark.parametrize("shape", [RAGGED, CUBE, (40, 20, 34)])
def test_fd8_gradient_and_divergence_match_oracle(claire, shape):
    # (40, 20, 34): two x1 slabs of the divergence march (the second partial), a
    # partial x2 tile and n3 % 4 != 0 (element-wise plane staging)
    u = synth.smooth_field(shape, 5, 3).astype(np.float32)
    w = synth.bandlimited_velocity(shape, 5, 2.0, 4).astype(np.float32)
    with claire.Context(shape) as ctx:
        gu = ctx.grad8(dev(u))
        dw = ctx.div8(dev(w))
    assert rel(host(gu), OF.grad8(_f64(u))) < 1e-5
    assert rel(host(dw), OF.div8(_f64(w))) < 1e-5


@pytest.mark.parametrize("gamma", [1.0, 2.0])
def test_spectral_operators_match_oracle(claire, gamma):
    shape = RAGGED
    x = synth.bandlimited_velocity(shape, 6, 2.0, 5).astype(np.float32)
    x64 = _f64(x)
    alpha, beta_w = 3e-2, 1e-3
    with claire.Context(shape, beta_v=alpha, gamma=gamma, beta_w=beta_w) as ctx:
        L = ctx.spectral(claire.OP_L, dev(x))
        Minv = ctx.spectral(claire.OP_REG_INV, dev(x))
        P = ctx.spectral(claire.OP_LERAY_PAR, dev(x))
        C = ctx.spectral(claire.OP_NEAR_INC, dev(x))
    assert rel(host(L), OS.apply_L(x64, gamma)) < 1e-5
    assert rel(host(Minv), OS.apply_reg_inverse(x64, alpha, gamma)) < 1e-5
    assert rel(host(P), OS.leray_parallel(x64)) < 1e-5
    assert rel(host(C), OS.near_incompressible_term(x64, alpha, beta_w)) < 1e-5


@pytest.mark.parametrize("shape", [RAGGED, CUBE])
def test_transport_matches_oracle(claire, shape):
    m0, m1, v = _pair(shape)
    with claire.Context(shape, nt=4) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        out = ctx.transport(dev(v))
    ref = OT.state_solve(_f64(m0), _f64(v), 4)[-1]
    assert rel(host(out), ref) < 1e-5


def test_zero_velocity_transport_is_bitwise_identity(claire):
    m0, m1, _ = _pair(RAGGED)
    with claire.Context(RAGGED, nt=4) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        out = ctx.transport(torch.zeros((3,) + RAGGED, device="cuda"))
    assert np.array_equal(out.cpu().numpy(), m0)


@pytest.mark.parametrize("shape,beta_w", [(RAGGED, 0.0), (CUBE, 0.0), (RAGGED, 1e-3)])
def test_objective_gradient_and_matvec_match_oracle(claire, shape, beta_w):
    m0, m1, vtrue = _pair(shape)
    v = 0.4 * vtrue
    vt = synth.bandlimited_velocity(shape, 4, 1.5, 9).astype(np.float32)
    with claire.Context(shape, nt=4, beta_v=1e-2, beta_w=beta_w) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        J, g = ctx.objective_gradient(dev(v))
        Hv = ctx.hessian_matvec(dev(vt))
    prob = OR.Problem(_f64(m0), _f64(m1), 4, 1e-2, 1.0, beta_w)
    ev = OR.evaluate(prob, _f64(v))
    assert abs(J - ev.J) / abs(ev.J) < 1e-5
    assert rel(host(g), ev.g) < 1e-4
    assert rel(host(Hv), OR.hessian_matvec(prob, ev, _f64(vt))) < 1e-4


@pytest.mark.parametrize("nt", [1, 2, 3, 8])
def test_other_time_step_counts_match_oracle(claire, nt):
    """n_t in {1, 2, 8} uses the FD8 march with 2, 3, 9 history fields; n_t = 3 the
    per-node fallback kernels."""
    shape = (24, 20, 16)
    m0, m1, vtrue = _pair(shape, kmax=3, disp=2.0)
    v = 0.4 * vtrue
    vt = synth.bandlimited_velocity(shape, 4, 1.5, 19).astype(np.float32)
    with claire.Context(shape, nt=nt, beta_v=1e-2) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        J, g = ctx.objective_gradient(dev(v))
        Hv = ctx.hessian_matvec(dev(vt))
    prob = OR.Problem(_f64(m0), _f64(m1), nt, 1e-2)
    ev = OR.evaluate(prob, _f64(v))
    assert abs(J - ev.J) / abs(ev.J) < 1e-5
    assert rel(host(g), ev.g) < 1e-4
    assert rel(host(Hv), OR.hessian_matvec(prob, ev, _f64(vt))) < 1e-4


@pytest.mark.parametrize("shape", [RAGGED, (32, 32, 32)])
def test_full_newton_matvec_matches_oracle(claire, shape):
    """options.hessian = 1: eq. (matvec) with the lam terms (full Newton)."""
    m0, m1, v = _pair(shape, kmax=3, disp=2.0)
    vt = synth.bandlimited_velocity(shape, 4, 1.0, 41)
    with claire.Context(shape, nt=4, beta_v=1e-2, hessian=1) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        ctx.objective_gradient(dev(0.5 * v))
        Hv = ctx.hessian_matvec(dev(vt))
        ctx.set_options(hessian=0)
        ctx.objective_gradient(dev(0.5 * v))
        Hgn = ctx.hessian_matvec(dev(vt))
    prob = OR.Problem(_f64(m0), _f64(m1), 4, 1e-2)
    ev = OR.evaluate(prob, _f64(0.5 * v))
    ref = OR.hessian_matvec(prob, ev, _f64(vt), full_newton=True)
    ref_gn = OR.hessian_matvec(prob, ev, _f64(vt))
    assert rel(host(Hv), ref) < 1e-4
    assert rel(host(Hgn), ref_gn) < 1e-4
    assert rel(ref, ref_gn) > 1e-3                   # the extra terms are not negligible


def test_full_newton_solve_matches_oracle(claire):
    shape = (32, 32, 32)
    m0, m1, _ = _pair(shape, seed=7, kmax=3, disp=1.5)
    with claire.Context(shape, nt=4, beta_v=1e-2, max_newton=2, max_pcg=5, fixed_iters=1,
                        hessian=1, precond=0) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve()
    prob = OR.Problem(_f64(m0), _f64(m1), 4, 1e-2)
    vo, so, _ = OSV.gauss_newton(prob, None, OSV.Options(max_newton=2, max_pcg=5,
                                                          fixed_iters=True, full_newton=True))
    assert st.newton_iters == 2 and st.pcg_iters == so.pcg_iters
    assert rel(host(v), vo) < 1e-3
    assert abs(st.J - so.J) / so.J < 1e-4


def test_full_newton_needs_fp32_storage(claire):
    with claire.Context(RAGGED) as ctx:
        with pytest.raises(claire.ClaireError) as e:
            ctx.set_options(hessian=1, precision=1)
        assert e.value.status == claire.EINVAL


def test_matvec_before_gradient_is_an_order_error(claire):
    with claire.Context(RAGGED) as ctx:
        with pytest.raises(claire.ClaireError) as e:
            ctx.hessian_matvec(torch.zeros((3,) + RAGGED, device="cuda"))
        assert e.value.status == claire.EORDER


def test_two_gauss_newton_by_ten_pcg_on_the_64_cube_matches_oracle(claire):
    """The parity workload: 64^3 blobs, nt 4, beta_v 1e-2, 2 GN x 10 PCG."""
    m0, m1, _ = synth.blob_pair(CUBE, seed=1)
    with claire.Context(CUBE, nt=4, beta_v=1e-2, max_newton=2, max_pcg=10,
                        fixed_iters=1, precond=0) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve()
    prob = OR.Problem(_f64(m0), _f64(m1), 4, 1e-2)
    vo, so, _ = OSV.gauss_newton(prob, None, OSV.Options(max_newton=2, max_pcg=10,
                                                          fixed_iters=True))
    assert st.newton_iters == 2 and st.matvecs == 20
    assert rel(host(v), vo) < 1e-3
    assert abs(st.J - so.J) / so.J < 1e-4


def test_solve_to_tolerance_on_a_ragged_grid(claire):
    m0, m1, _ = _pair(RAGGED, seed=2, kmax=2, disp=1.5)
    with claire.Context(RAGGED, nt=4, beta_v=5e-2, eps_opt=5e-2) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve()
    assert st.status == claire.OK
    assert st.grad_rel <= 5e-2
    assert st.J < st.J0
    prob = OR.Problem(_f64(m0), _f64(m1), 4, 5e-2)
    ev = OR.evaluate(prob, host(v))
    gnorm0 = np.max(np.abs(OR.gradient_at_zero(prob)))
    assert np.max(np.abs(ev.g)) / gnorm0 <= 5.5e-2     # the oracle agrees it converged


def test_continuation_matches_sequential_solves(claire):
    m0, m1, _ = _pair(RAGGED, seed=3, kmax=2, disp=1.5)
    betas = [1e-1, 1e-2]
    with claire.Context(RAGGED, nt=4, beta_v=1e-1) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve_continuation(betas)
    prob = OR.Problem(_f64(m0), _f64(m1), 4, 1e-1)
    vo, so, _ = OSV.continuation(prob, betas, OSV.Options())
    assert st.newton_iters == so.newton_iters
    assert rel(host(v), vo) < 1e-3


def test_solve_host_equals_device_solve(claire):
    m0, m1, _ = _pair(RAGGED, seed=4, kmax=2, disp=1.5)
    with claire.Context(RAGGED, nt=4, beta_v=5e-2) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        vd, sd = ctx.solve()
        vh = torch.zeros((3,) + RAGGED).pin_memory()
        vh, sh = ctx.solve_host(torch.from_numpy(m0).pin_memory(),
                                torch.from_numpy(m1).pin_memory(), vh)
    assert np.array_equal(vh.numpy(), vd.cpu().numpy())
    assert sh.matvecs == sd.matvecs


@pytest.mark.parametrize("precision,pinned", [(0, True), (1, True), (0, False)])
def test_solve_host_continuation_equals_device_solve(claire, precision, pinned):
    """claire_solve_host overlaps its host copies with the solve (the FP32 form uploads
    m1 on a side stream, accepted steps are copied to pinned host memory as they come):
    the result is bitwise the device solve's, and the context stays reusable."""
    shape = (32, 32, 32)
    m0, m1, _ = _pair(shape, seed=6, kmax=3, disp=2.0)
    betas = [1e-1, 1e-2, 1e-3]
    host = (lambda a: torch.from_numpy(a).pin_memory()) if pinned else torch.from_numpy
    with claire.Context(shape, nt=4, beta_v=1e-1, precision=precision) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        vd, sd = ctx.solve_continuation(betas)
        vh = host(np.zeros((3,) + shape, dtype=np.float32))
        vh, sh = ctx.solve_host(host(m0), host(m1), vh, betas)
        ctx.set_images(dev(m0), dev(m1))
        vd2, _ = ctx.solve_continuation(betas)
    assert sh.newton_iters == sd.newton_iters and sd.newton_iters > 1
    assert sh.matvecs == sd.matvecs
    assert np.array_equal(vh.numpy(), vd.cpu().numpy())
    assert np.array_equal(vd2.cpu().numpy(), vd.cpu().numpy())


def test_solve_host_from_a_converged_guess_returns_it(claire):
    """No accepted step: the initial guess comes back unchanged (the result copy is
    then taken at the end of the call)."""
    m0, m1, _ = _pair(RAGGED, seed=4, kmax=2, disp=1.5)
    with claire.Context(RAGGED, nt=4, beta_v=5e-2) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        vd, _ = ctx.solve()
        v0 = vd.cpu().pin_memory()
        vh = v0.clone().pin_memory()
        vh, sh = ctx.solve_host(torch.from_numpy(m0).pin_memory(),
                                torch.from_numpy(m1).pin_memory(), vh)
    assert sh.newton_iters == 0
    assert np.array_equal(vh.numpy(), v0.numpy())


@pytest.mark.parametrize("shape", [RAGGED, (32, 32, 32)])
def test_det_deformation_gradient_matches_oracle(claire, shape):
    _, _, v = _pair(shape, kmax=3, disp=2.0)
    with claire.Context(shape, nt=4) as ctx:
        (mn, mx, mean), det = ctx.det_deformation_gradient(dev(v), want_field=True)
    d_ref, (rmn, rmx, rmean) = ODG.det_deformation_gradient(_f64(v), 4)
    assert rel(host(det), d_ref) < 1e-5
    assert abs(mn - rmn) < 1e-5 and abs(mx - rmx) < 1e-5 and abs(mean - rmean) < 1e-6


def test_invalid_shapes_and_options_are_rejected(claire):
    for shape in [(15, 16, 16), (16, 14, 16), (16, 16, 17)]:
        with pytest.raises(claire.ClaireError) as e:
            claire.Context(shape)
        assert e.value.status == claire.EINVAL
    with claire.Context(RAGGED) as ctx:
        with pytest.raises(claire.ClaireError):
            ctx.set_options(max_pcg=0)
        with pytest.raises(TypeError):
            ctx.transport(torch.zeros((3,) + RAGGED))          # host tensor
        with pytest.raises(ValueError):
            ctx.transport(torch.zeros((3, 16, 16, 16), device="cuda"))


def test_non_finite_input_is_reported(claire):
    m0, m1, v = _pair(RAGGED)
    m1 = m1.copy()
    m1[3, 4, 5] = np.nan
    with claire.Context(RAGGED) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        with pytest.raises(claire.ClaireError) as e:
            ctx.objective_gradient(dev(v))
        assert e.value.status == claire.ENONFINITE
