"""GPU regularisation-parameter search with det F bounds (Sec. 2.6).

* The trial sequence of `claire_beta_search` follows the rule of
  `oracle.solver.beta_search` applied to the GPU's own det F1 values.
* The returned velocity satisfies eps_d < det F1 < 1/eps_d by the FP64 oracle.
* Where no det F1 value of the oracle's own search lies within 1e-3 of a bound,
  GPU and oracle take the same trials and end on the same beta.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import reduced as OR, solver as OSV, defgrad as ODG
from paper_2401_17493_b300 import synth


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


def test_beta_search_follows_the_rule_and_matches_oracle(claire):
    shape = (16, 16, 16)
    m0, m1, _ = synth.blob_pair(shape, seed=5, kmax=2, max_disp_voxels=2.5)
    eps_d, rtol, nb = 0.5, 0.2, 4
    with claire.Context(shape, nt=4, beta_v=1.0, precond=0) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        beta, v, trials, st = ctx.beta_search(eps_d=eps_d, rtol=rtol, max_bisect=nb)
    assert beta > 0.0 and len(trials) >= 3 and st.newton_iters > 0

    # replay the rule on the GPU's own det values
    def lookup(b):
        k = int(np.argmin([abs(t[0] - b) for t in trials]))
        assert abs(trials[k][0] - b) <= 1e-12 * b
        return trials[k][1], trials[k][2]
    rb, _, rtrials = OSV.beta_search(lambda b, v0: b, lookup, eps_d=eps_d, rtol=rtol,
                                     max_bisect=nb)
    assert [t[0] for t in rtrials] == pytest.approx([t[0] for t in trials], rel=1e-12)
    assert rb == pytest.approx(beta, rel=1e-12)

    # the result satisfies the bound (FP64 det F of the GPU velocity)
    _, (mn, mx, _) = ODG.det_deformation_gradient(v.cpu().numpy().astype(np.float64), 4)
    assert eps_d < mn and mx < 1.0 / eps_d

    # the oracle's own search
    p = OR.Problem(m0.astype(np.float64), m1.astype(np.float64), nt=4, beta_v=1.0)
    gnorm0 = float(np.max(np.abs(OR.gradient_at_zero(p))))

    def solve(b, v0):
        p.beta_v = b
        return OSV.gauss_newton(p, v0, OSV.Options(eps_opt=5e-2), gnorm0=gnorm0)[0]

    def bounds(vv):
        _, (a, b, _) = ODG.det_deformation_gradient(vv, 4)
        return a, b
    ob, _, otrials = OSV.beta_search(solve, bounds, eps_d=eps_d, rtol=rtol, max_bisect=nb)
    margin = min(min(abs(t[2] - eps_d), abs(t[3] - 1.0 / eps_d)) for t in otrials)
    if margin > 1e-3:
        assert [t[0] for t in otrials] == pytest.approx([t[0] for t in trials], rel=1e-12)
        assert ob == pytest.approx(beta, rel=1e-12)


def test_beta_search_rejects_bad_arguments(claire):
    with claire.Context((16, 16, 16)) as ctx:
        for kw in (dict(eps_d=1.5), dict(eps_d=0.0), dict(beta0=-1.0), dict(rtol=0.0)):
            with pytest.raises(claire.ClaireError) as e:
                ctx.beta_search(**kw)
            assert e.value.status == claire.EINVAL
