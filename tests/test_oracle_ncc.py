"""Pins for the NCC distance of the Appendix (oracle.reduced, distance = "ncc").

* dist = 1 - cos^2 of the angle between m(1) and m1: 0 for any multiple of m1,
  symmetric, in [0, 1].
* lam(1) is minus the gradient of dist w.r.t. m(1): central differences.
* lam~(1) is the derivative of lam(1) in the direction m~(1): central
  differences.  The printed q1 fails this check; its negative passes
  (reading C-16).
* J and g, and the GN Hessian, on a small registration: central differences
  of J against <g, w> and of g against H w (Gauss-Newton drops terms, so the
  latter is only checked at a zero-residual point, where GN is exact).
"""

import numpy as np

from oracle import reduced as R
from paper_2401_17493_b300 import synth


def _prob(n=16, seed=5, beta=1e-3):
    m0, m1, v = synth.blob_pair((n, n, n), seed=seed, kmax=2, max_disp_voxels=1.0)
    return R.Problem(m0, m1, nt=4, beta_v=beta, distance="ncc"), v.astype(np.float64)


def test_ncc_distance_is_one_minus_squared_cosine():
    p, _ = _prob()
    m1 = p.m1
    for s in (0.3, 1.0, 2.5, -1.7):
        assert abs(R.distance(p, s * m1)) < 1e-14
    rng = np.random.default_rng(0)
    u = rng.standard_normal(m1.shape)
    d = R.distance(p, u)
    cos = np.sum(u * m1) / np.sqrt(np.sum(u * u) * np.sum(m1 * m1))
    assert abs(d - (1.0 - cos * cos)) < 1e-14 and 0.0 <= d <= 1.0
    q = R.Problem(u, u, distance="ncc")
    q.m1 = m1
    p2 = R.Problem(m1, m1, distance="ncc")
    p2.m1 = u
    assert abs(R.distance(q, u) - R.distance(p2, m1)) < 1e-14          # symmetric


def test_adjoint_final_is_minus_the_distance_gradient():
    p, _ = _prob()
    rng = np.random.default_rng(1)
    m = p.m1 + 0.2 * rng.standard_normal(p.shape)
    w = rng.standard_normal(p.shape)
    lam = R.adjoint_final(p, m)
    eps = 1e-5
    fd = (R.distance(p, m + eps * w) - R.distance(p, m - eps * w)) / (2 * eps)
    assert abs(fd + R.inner(p, lam, w)) <= 1e-7 * abs(fd)


def test_incremental_final_is_the_derivative_of_the_adjoint_final():
    p, _ = _prob()
    rng = np.random.default_rng(2)
    m = p.m1 + 0.2 * rng.standard_normal(p.shape)
    mt = rng.standard_normal(p.shape)
    eps = 1e-5
    fd = (R.adjoint_final(p, m + eps * mt) - R.adjoint_final(p, m - eps * mt)) / (2 * eps)
    ours = R.incremental_adjoint_final(p, m, mt)
    assert np.max(np.abs(ours - fd)) <= 1e-7 * np.max(np.abs(fd))
    # the q1 printed in the paper (opposite sign) is not the derivative
    a, b, c = R.inner(p, p.m1, m), R.inner(p, p.m1, p.m1), R.inner(p, m, m)
    al, ga = R.inner(p, p.m1, mt), R.inner(p, m, mt)
    q1_printed = 2 * a * ga / c ** 2 - al / c
    printed = ours + 2.0 * (q1_printed - (al / c - 2 * a * ga / c ** 2)) * p.m1 / b
    assert np.max(np.abs(printed - fd)) > 1e-2 * np.max(np.abs(fd))


def test_ncc_gradient_matches_central_differences_of_J():
    p, v = _prob()
    v = 0.5 * v
    ev = R.evaluate(p, v)
    w = synth.bandlimited_velocity(p.shape, 3, 1.0, 9).astype(np.float64)
    eps = 1e-3
    Jp = R.evaluate_objective(p, v + eps * w).J
    Jm = R.evaluate_objective(p, v - eps * w).J
    fd = (Jp - Jm) / (2 * eps)
    ip = p.h3 * float(np.sum(ev.g * w))
    assert abs(fd - ip) <= 5e-2 * abs(fd)          # optimize-then-discretize (Sec. 2.3)


def test_ncc_gauss_newton_hessian_at_a_zero_residual_point():
    """m1 = m(1) of the current v: GN is the exact second derivative up to discretisation."""
    p, v = _prob(beta=1e-2)
    v = 0.5 * v
    ev0 = R.evaluate_objective(p, v)
    p.m1 = ev0.m[-1].copy()                         # zero residual (dist = 0)
    ev = R.evaluate(p, v)
    assert ev.mismatch < 1e-12
    w = synth.bandlimited_velocity(p.shape, 3, 1.0, 10).astype(np.float64)
    eps = 1e-3
    gp = R.evaluate(p, v + eps * w).g
    gm = R.evaluate(p, v - eps * w).g
    fd = (gp - gm) / (2 * eps)
    Hw = R.hessian_matvec(p, ev, w)
    assert np.linalg.norm(Hw - fd) <= 5e-2 * np.linalg.norm(fd)
