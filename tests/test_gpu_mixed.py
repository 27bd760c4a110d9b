"""Mixed-precision form (FP16 field storage, FP32 math and coordinates, FP64
reductions) against the FP64 oracle.  The error of each output is measured and
bounded; the bounds follow from FP16's 2^-11 relative rounding of stored fields
(about 5e-4 per stored value), amplified by the FD8 stencil (coefficient sum
~2.1) and accumulated over n_t steps."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import reduced as OR, solver as OSV
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


def f64(a):
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


@pytest.mark.parametrize("shape", [RAGGED, CUBE])
def test_mixed_transport_error(claire, shape):
    """m(1) with FP16 storage between the SL steps against the FP64 oracle's m(1):
    n_t roundings of the stored state (2^-11 relative each) plus the FP32 path."""
    from oracle import transport as OT
    m0, m1, vtrue = synth.blob_pair(shape, seed=1)
    v = 0.8 * vtrue
    ref = OT.state_solve(f64(m0), f64(v), 4)[-1]
    with claire.Context(shape, nt=4, beta_v=1e-2, precision=1) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        m_mixed = host(ctx.transport(dev(v)))
        ctx.set_options(precision=0)
        m_fp32 = host(ctx.transport(dev(v)))
    e_mixed, e_fp32 = rel(m_mixed, ref), rel(m_fp32, ref)
    print(f"mixed {shape}: m(1) {e_mixed:.2e} (FP32 storage {e_fp32:.2e})")
    assert e_fp32 < 1e-5
    assert 1e-6 < e_mixed < 1e-3


@pytest.mark.parametrize("shape", [RAGGED, CUBE])
def test_mixed_objective_gradient_and_matvec_errors(claire, shape):
    m0, m1, vtrue = synth.blob_pair(shape, seed=1)
    v = 0.4 * vtrue
    vt = synth.bandlimited_velocity(shape, 4, 1.5, 9).astype(np.float32) * 37.0   # any scale
    prob = OR.Problem(f64(m0), f64(m1), 4, 1e-2)
    ev = OR.evaluate(prob, f64(v))
    H_ref = OR.hessian_matvec(prob, ev, f64(vt))
    with claire.Context(shape, nt=4, beta_v=1e-2, precision=1) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        J, g = ctx.objective_gradient(dev(v))
        Hv = ctx.hessian_matvec(dev(vt))
    eJ, eg, eH = abs(J - ev.J) / ev.J, rel(host(g), ev.g), rel(host(Hv), H_ref)
    print(f"mixed {shape}: J {eJ:.2e}  g {eg:.2e}  Hv {eH:.2e}")
    assert eJ < 2e-3 and eg < 2e-2 and eH < 2e-2


@pytest.mark.parametrize("nt", [2, 8])
def test_mixed_other_time_step_counts(claire, nt):
    shape = (24, 20, 16)
    m0, m1, vtrue = synth.blob_pair(shape, seed=2, kmax=3, max_disp_voxels=2.0)
    v = 0.4 * vtrue
    vt = synth.bandlimited_velocity(shape, 4, 1.5, 29).astype(np.float32)
    prob = OR.Problem(f64(m0), f64(m1), nt, 1e-2)
    ev = OR.evaluate(prob, f64(v))
    with claire.Context(shape, nt=nt, beta_v=1e-2, precision=1) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        J, g = ctx.objective_gradient(dev(v))
        Hv = ctx.hessian_matvec(dev(vt))
    assert abs(J - ev.J) / ev.J < 2e-3
    assert rel(host(g), ev.g) < 2e-2
    assert rel(host(Hv), OR.hessian_matvec(prob, ev, f64(vt))) < 2e-2


def test_mixed_images_far_from_unit_range_are_scaled(claire):
    shape = RAGGED
    m0, m1, vtrue = synth.blob_pair(shape, seed=2)
    v = 0.4 * vtrue
    for s in (3e3, 1e-3):                 # FP16 overflow / underflow without the image scale
        prob = OR.Problem(f64(m0) * s, f64(m1) * s, 4, 1e-2)
        ev = OR.evaluate(prob, f64(v))
        with claire.Context(shape, nt=4, beta_v=1e-2, precision=1) as ctx:
            ctx.set_images(dev(m0 * s), dev(m1 * s))
            J, g = ctx.objective_gradient(dev(v))
        assert abs(J - ev.J) / ev.J < 2e-3
        assert rel(host(g), ev.g) < 2e-2


def test_mixed_two_gauss_newton_by_ten_pcg_against_oracle(claire):
    m0, m1, _ = synth.blob_pair(CUBE, seed=1)
    with claire.Context(CUBE, nt=4, beta_v=1e-2, max_newton=2, max_pcg=10, fixed_iters=1,
                        precision=1, precond=0) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve()
    prob = OR.Problem(f64(m0), f64(m1), 4, 1e-2)
    vo, so, _ = OSV.gauss_newton(prob, None, OSV.Options(max_newton=2, max_pcg=10,
                                                          fixed_iters=True))
    ev_ = rel(host(v), vo)
    print(f"mixed 2x10 solve: v {ev_:.2e}  J {abs(st.J - so.J) / so.J:.2e}")
    assert ev_ < 3e-2
    assert abs(st.J - so.J) / so.J < 5e-3


def test_mixed_solve_reaches_the_same_accuracy_as_fp32(claire):
    m0, m1, _ = synth.blob_pair(CUBE, seed=3, kmax=3, max_disp_voxels=2.5)
    out = {}
    for prec in (0, 1):
        with claire.Context(CUBE, nt=4, beta_v=1e-2, precision=prec) as ctx:
            ctx.set_images(dev(m0), dev(m1))
            v, st = ctx.solve()
            out[prec] = (host(v), st.grad_rel, st.mismatch_rel, st.status)
    assert out[0][3] == claire.OK and out[1][3] == claire.OK
    assert out[1][1] <= 5e-2
    assert abs(out[1][2] - out[0][2]) < 0.05 * out[0][2]
    assert rel(out[1][0], out[0][0]) < 5e-2
