"""Pins for oracle.defgrad (Appendix, eq. def-grad): identity cases, an exact
shear flow, an ordering-sensitive shear with an analytic solution, and the
first-order relation det F1 ~ 1 + div v."""

import numpy as np
from scipy.integrate import quad

from oracle import defgrad as DG
from oracle.fd8 import d8, div8


def _x(shape):
    return np.meshgrid(*[np.arange(n) * 2 * np.pi / n for n in shape], indexing="ij")


def test_identity_for_zero_and_constant_velocity():
    shape = (16, 16, 16)
    d, (mn, mx, mean) = DG.det_deformation_gradient(np.zeros((3,) + shape), 4)
    assert np.array_equal(d, np.ones(shape))
    v = np.stack([np.full(shape, c) for c in (0.3, -0.2, 0.5)])
    F = DG.deformation_gradient(v, 4)
    assert np.allclose(F, np.eye(3)[:, :, None, None, None], atol=1e-13)


def test_single_shear_gives_identity_plus_velocity_gradient():
    shape = (16, 16, 16)
    x = _x(shape)
    a = 0.4
    v = np.stack([a * np.sin(x[1]), 0 * x[0], 0 * x[0]])
    F = DG.deformation_gradient(v, 4)
    A01 = d8(v[0], 1, 2 * np.pi / 16)
    expect = np.zeros((3, 3) + shape)
    for i in range(3):
        expect[i, i] = 1.0
    expect[0, 1] = A01
    assert np.allclose(F, expect, atol=1e-12)


def test_double_shear_matches_the_analytic_deformation_gradient():
    """v = (a sin x2, b sin x3, 0): F13 = a b cos(x3) int_0^1 cos(x2 - c + c t) t dt,
    c = b sin x3, which distinguishes (grad v) F from F (grad v)."""
    n = 32
    shape = (n, n, n)
    x = _x(shape)
    a, b = 0.5, 0.4
    v = np.stack([a * np.sin(x[1]), b * np.sin(x[2]), 0 * x[0]])
    F = DG.deformation_gradient(v, 16)
    rng = np.random.default_rng(0)
    for _ in range(10):
        i, j = rng.integers(0, n, 2)
        x2, x3 = x[1][0, i, j], x[2][0, i, j]
        c = b * np.sin(x3)
        f13 = a * b * np.cos(x3) * quad(lambda t: np.cos(x2 - c + c * t) * t, 0, 1)[0]
        f12 = a * quad(lambda t: np.cos(x2 - c + c * t), 0, 1)[0]
        f23 = b * np.cos(x3)
        assert abs(F[0, 2, 0, i, j] - f13) < 2e-3 * (abs(a * b) + 1e-3)
        assert abs(F[0, 1, 0, i, j] - f12) < 2e-3
        assert abs(F[1, 2, 0, i, j] - f23) < 1e-5


def test_det_is_one_plus_divergence_to_first_order():
    shape = (16, 16, 16)
    x = _x(shape)
    base = np.stack([np.sin(x[0]), np.cos(x[1] + x[2]), 0.5 * np.sin(x[2])])
    errs = []
    for eps in (1e-2, 5e-3):
        d, _ = DG.det_deformation_gradient(eps * base, 4)
        errs.append(np.max(np.abs(d - 1.0 - div8(eps * base))))
    assert errs[0] < 1e-3
    assert errs[0] / errs[1] > 3.5        # second-order remainder
