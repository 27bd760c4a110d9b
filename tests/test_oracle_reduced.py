"""Pins for oracle.reduced: the v = 0 closed forms (Sec. 2.5.6, zero velocity
approximation), finite-difference checks of g and H at 16^3 (P-8), Hessian
symmetry and positivity (P-9, Sec. 2.5.5)."""

import numpy as np
import pytest

from oracle import reduced as R
from oracle import transport as T
from oracle.fd8 import grad8, div8
from oracle.spectral import apply_L


def _x(shape):
    return np.meshgrid(*[np.arange(n) * 2 * np.pi / n for n in shape], indexing="ij")


def _case(shape=(16, 16, 16)):
    x = _x(shape)
    m0 = (np.exp(-2 * (np.sin(x[0] / 2) ** 2 + np.sin(x[1] / 2) ** 2 + np.sin(x[2] / 2) ** 2))
          + 0.3 * np.cos(x[0] + x[1]))
    m1 = (np.exp(-2 * (np.sin((x[0] - 0.3) / 2) ** 2 + np.sin((x[1] + 0.2) / 2) ** 2
                       + np.sin(x[2] / 2) ** 2)) + 0.3 * np.cos(x[0] + x[1] - 0.2))
    v = 0.15 * np.stack([np.sin(x[1]), np.cos(x[0] + x[2]), np.sin(x[0]) * np.cos(x[1])])
    vt = np.stack([np.cos(x[0] + 2 * x[1]), np.sin(x[2]), np.cos(x[1] - x[2])])
    return x, m0, m1, v, vt


def test_zero_velocity_objective_gradient_and_hessians():
    rng = np.random.default_rng(0)
    shape = (16, 16, 16)
    x = _x(shape)
    m0 = np.sin(x[0]) * np.cos(x[1]) + 0.1 * rng.standard_normal(shape)
    m1 = np.cos(x[2]) + 0.1 * rng.standard_normal(shape)
    alpha = 3e-2
    p = R.Problem(m0, m1, nt=4, beta_v=alpha)
    v0 = np.zeros((3,) + shape)
    ev = R.evaluate(p, v0)
    h3 = (2 * np.pi / 16) ** 3
    assert abs(ev.J - 0.5 * h3 * np.sum((m0 - m1) ** 2)) < 1e-12 * ev.J
    lam = m1 - m0
    gm0 = grad8(m0)
    assert np.allclose(ev.g, lam[None] * gm0, atol=1e-12)
    vt = rng.standard_normal((3,) + shape)
    s = np.sum(gm0 * vt, axis=0)
    H_gn = alpha * apply_L(vt, 1.0) + gm0 * s[None]
    assert np.allclose(R.hessian_matvec(p, ev, vt), H_gn, atol=1e-10)
    H_full = H_gn + 0.5 * (div8(lam[None] * vt)[None] * gm0 - lam[None] * grad8(s))
    assert np.allclose(R.hessian_matvec(p, ev, vt, full_newton=True), H_full, atol=1e-10)


def test_gradient_matches_central_differences_of_the_objective():
    x, m0, m1, v, vt = _case()
    p = R.Problem(m0, m1, nt=4, beta_v=1e-2)
    ev = R.evaluate(p, v)
    dd = p.h3 * np.sum(ev.g * vt)
    for eps in (1e-2, 1e-4):
        fd = (R.evaluate_objective(p, v + eps * vt).J - R.evaluate_objective(p, v - eps * vt).J) / (2 * eps)
        assert abs(fd - dd) / abs(dd) < 5e-2


def test_full_newton_hessian_matches_central_differences_of_the_gradient():
    x, m0, m1, v, vt = _case()
    p = R.Problem(m0, m1, nt=4, beta_v=1e-2)
    ev = R.evaluate(p, v)
    eps = 1e-4
    fd = (R.evaluate(p, v + eps * vt).g - R.evaluate(p, v - eps * vt).g) / (2 * eps)
    H = R.hessian_matvec(p, ev, vt, full_newton=True)
    assert np.linalg.norm(fd - H) / np.linalg.norm(fd) < 5e-2


def test_gauss_newton_is_the_hessian_at_a_zero_residual_point():
    x, m0, m1, v, vt = _case()
    p = R.Problem(m0, T.state_solve(m0, v, 4)[-1], nt=4, beta_v=1e-2)
    ev = R.evaluate(p, v)
    assert np.max(np.abs(ev.lam[-1])) == 0.0
    eps = 1e-4
    fd = (R.evaluate(p, v + eps * vt).g - R.evaluate(p, v - eps * vt).g) / (2 * eps)
    H = R.hessian_matvec(p, ev, vt)
    assert np.linalg.norm(fd - H) / np.linalg.norm(fd) < 2e-2


@pytest.mark.parametrize("full", [False, True])
def test_hessian_is_symmetric_and_gauss_newton_is_positive(full):
    x, m0, m1, v, vt = _case()
    w = np.stack([np.sin(x[0]), np.cos(x[1] + x[0]), np.sin(2 * x[2])])
    p = R.Problem(m0, m1, nt=4, beta_v=1e-2)
    ev = R.evaluate(p, v)
    Hv = R.hessian_matvec(p, ev, vt, full)
    Hw = R.hessian_matvec(p, ev, w, full)
    assert abs(np.sum(Hv * w) - np.sum(vt * Hw)) / (np.linalg.norm(Hv) * np.linalg.norm(w)) < 1e-2
    if not full:
        # <v~, H_GN v~> ~= alpha <L v~, v~> + ||m~(1)||^2 (continuum identity, Sec. 2.5.5)
        mt1 = T.incremental_state_solve(ev.m, vt, v, 4)[-1]
        quad = p.h3 * np.sum(vt * Hv)
        model = p.h3 * (1e-2 * np.sum(vt * apply_L(vt, 1.0)) + np.sum(mt1 ** 2))
        assert quad > 0
        assert abs(quad - model) / model < 5e-2


def test_near_incompressible_model_projects_the_data_term():
    x, m0, m1, v, vt = _case()
    p0 = R.Problem(m0, m1, nt=4, beta_v=1e-2)
    pw = R.Problem(m0, m1, nt=4, beta_v=1e-2, beta_w=1e12)
    g0 = R.evaluate(p0, v).g
    gw = R.evaluate(pw, v).g
    from oracle.spectral import leray
    b = g0 - 1e-2 * apply_L(v, 1.0)
    assert np.allclose(gw, 1e-2 * apply_L(v, 1.0) + leray(b), atol=1e-8)
