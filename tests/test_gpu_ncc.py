"""GPU parity of the NCC distance (Appendix, options.distance = 1).

J, g and the Gauss-Newton / full-Newton Hessian matvec against the FP64 oracle
with distance = "ncc" (relative L2: J 1e-5, g and H v 1e-4), a fixed
2 GN x 5 PCG solve (v 1e-3), and the invariance of the NCC solve to a scaling
of the reference image (same v up to FP32 rounding).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import reduced as OR, solver as OSV
from paper_2401_17493_b300 import synth

RAGGED = (22, 18, 40)


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


@pytest.mark.parametrize("shape", [RAGGED, (32, 32, 32)])
@pytest.mark.parametrize("hessian", [0, 1])
def test_ncc_objective_gradient_matvec_match_oracle(claire, shape, hessian):
    m0, m1, v = synth.blob_pair(shape, seed=2, kmax=3, max_disp_voxels=2.0)
    vt = synth.bandlimited_velocity(shape, 4, 1.0, 43)
    beta = 1e-4
    with claire.Context(shape, nt=4, beta_v=beta, distance=1, hessian=hessian) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        J, g = ctx.objective_gradient(dev(0.5 * v))
        Hv = ctx.hessian_matvec(dev(vt))
    prob = OR.Problem(_f64(m0), _f64(m1), 4, beta, distance="ncc")
    ev = OR.evaluate(prob, _f64(0.5 * v))
    Hr = OR.hessian_matvec(prob, ev, _f64(vt), full_newton=bool(hessian))
    assert abs(J - ev.J) / ev.J < 1e-5
    assert rel(host(g), ev.g) < 1e-4
    assert rel(host(Hv), Hr) < 1e-4


def test_ncc_solve_matches_oracle(claire):
    shape = (32, 32, 32)
    m0, m1, _ = synth.blob_pair(shape, seed=3, kmax=3, max_disp_voxels=2.0)
    beta = 1e-4
    with claire.Context(shape, nt=4, beta_v=beta, distance=1, max_newton=2, max_pcg=5,
                        fixed_iters=1, precond=0) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve()
    prob = OR.Problem(_f64(m0), _f64(m1), 4, beta, distance="ncc")
    vo, so, _ = OSV.gauss_newton(prob, None, OSV.Options(max_newton=2, max_pcg=5,
                                                          fixed_iters=True))
    assert st.newton_iters == 2 and st.matvecs == so.matvecs
    assert rel(host(v), vo) < 1e-3
    assert abs(st.J - so.J) / so.J < 1e-4
    assert abs(st.mismatch_rel - so.mismatch_rel) < 1e-4


def test_ncc_solve_is_invariant_to_reference_scaling(claire):
    shape = (64, 64, 64)
    m0, m1, _ = synth.blob_pair(shape, seed=4, kmax=4, max_disp_voxels=3.0)
    out = []
    for scale in (1.0, 4.0):
        with claire.Context(shape, nt=4, beta_v=1e-4, distance=1, precond=1) as ctx:
            ctx.set_images(dev(m0), dev(scale * m1))
            v, st = ctx.solve()
        assert st.status == claire.OK and st.grad_rel <= 5e-2 and st.mismatch_rel < 0.5
        out.append((host(v), st))
    assert out[0][1].matvecs == out[1][1].matvecs
    assert rel(out[1][0], out[0][0]) < 1e-4


def test_ncc_needs_fp32_storage(claire):
    with claire.Context(RAGGED) as ctx:
        with pytest.raises(claire.ClaireError) as e:
            ctx.set_options(distance=1, precision=1)
        assert e.value.status == claire.EINVAL
        with pytest.raises(claire.ClaireError) as e:
            ctx.set_options(distance=2)
        assert e.value.status == claire.EINVAL
