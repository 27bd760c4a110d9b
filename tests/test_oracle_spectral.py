"""Pins for oracle.spectral: single modes, inverse rule (C-3), Leray, restrict/prolong."""

import numpy as np
import pytest

from oracle import spectral


def _grid(shape):
    return np.meshgrid(*[np.arange(n) * 2 * np.pi / n for n in shape], indexing="ij")


@pytest.mark.parametrize("gamma", [1.0, 2.0, 0.5])
def test_regulariser_on_single_modes(gamma):
    shape = (16, 12, 20)
    x = _grid(shape)
    for k in [(1, 2, 3), (0, 0, 5), (4, -3, 0), (8, 0, 0)]:   # (8,0,0) is the Nyquist mode
        u = np.cos(k[0] * x[0] + k[1] * x[1] + k[2] * x[2])
        v = np.stack([u, 2 * u, -u])
        Lv = spectral.apply_L(v, gamma)
        assert np.allclose(Lv, (k[0] ** 2 + k[1] ** 2 + k[2] ** 2) ** gamma * v, atol=1e-9)


def test_h1_seminorm_is_minus_laplacian_of_analytic_field():
    shape = (16, 16, 16)
    x = _grid(shape)
    u = np.sin(x[0]) * np.cos(2 * x[1]) + 0.3 * np.sin(3 * x[2] + x[0])
    lap = -(1 + 4) * np.sin(x[0]) * np.cos(2 * x[1]) - 0.3 * (9 + 1) * np.sin(3 * x[2] + x[0])
    Lu = spectral.apply_L(np.stack([u, u, u]), 1.0)
    assert np.allclose(Lu[0], -lap, atol=1e-10)


def test_preconditioner_inverts_regulariser_up_to_the_mean():
    rng = np.random.default_rng(0)
    shape = (12, 16, 10)
    u = rng.standard_normal((3,) + shape)
    alpha = 3e-2
    back = spectral.apply_reg_inverse(spectral.apply_reg(u, alpha, 1.0), alpha, 1.0)
    mean = u.mean(axis=(1, 2, 3), keepdims=True)
    assert np.allclose(back, u - mean, atol=1e-10)
    # zero symbol set to one (C-3): a constant is scaled by 1 / alpha
    c = np.ones((3,) + shape) * 2.0
    assert np.allclose(spectral.apply_reg_inverse(c, alpha, 1.0), 2.0 / alpha)


def test_leray_on_analytic_gradient_and_curl_fields():
    shape = (16, 16, 16)
    x = _grid(shape)
    # gradient of phi = sin(x1) cos(2 x2) sin(x3): P_par keeps it, Leray removes it
    grad_phi = np.stack([np.cos(x[0]) * np.cos(2 * x[1]) * np.sin(x[2]),
                         -2 * np.sin(x[0]) * np.sin(2 * x[1]) * np.sin(x[2]),
                         np.sin(x[0]) * np.cos(2 * x[1]) * np.cos(x[2])])
    assert np.allclose(spectral.leray(grad_phi), 0.0, atol=1e-12)
    assert np.allclose(spectral.leray_parallel(grad_phi), grad_phi, atol=1e-12)
    # a divergence-free field (curl of (0, 0, cos(x1 + 2 x2)))
    psi = np.cos(x[0] + 2 * x[1])
    curl = np.stack([-2 * np.sin(x[0] + 2 * x[1]), np.sin(x[0] + 2 * x[1]), 0 * psi])
    assert np.allclose(spectral.leray(curl), curl, atol=1e-12)


def test_leray_is_an_orthogonal_projection():
    rng = np.random.default_rng(1)
    shape = (12, 10, 16)
    a = rng.standard_normal((3,) + shape)
    b = rng.standard_normal((3,) + shape)
    Pa = spectral.leray_parallel(a)
    assert np.allclose(spectral.leray_parallel(Pa), Pa, atol=1e-12)
    assert abs(np.sum(Pa * b) - np.sum(a * spectral.leray_parallel(b))) < 1e-10 * np.sum(np.abs(a * b))


def test_near_incompressible_term_limits():
    rng = np.random.default_rng(2)
    shape = (12, 12, 12)
    b = rng.standard_normal((3,) + shape)
    assert np.array_equal(spectral.near_incompressible_term(b, 1e-2, 0.0), np.zeros_like(b))
    big = spectral.near_incompressible_term(b, 1e-2, 1e14)
    assert np.allclose(big, spectral.leray_parallel(b), atol=1e-9)


def test_restrict_and_prolong_on_band_limited_fields():
    fine, coarse = (16, 20, 12), (8, 10, 6)
    f = lambda x: np.sin(x[0]) * np.cos(2 * x[1] + 0.3) + 0.5 * np.cos(x[2] - x[0]) + 0.2
    uf = f(_grid(fine))
    uc = f(_grid(coarse))
    assert np.allclose(spectral.restrict(uf, coarse), uc, atol=1e-12)
    assert np.allclose(spectral.prolong(uc, fine), uf, atol=1e-12)
    rng = np.random.default_rng(3)
    r = rng.standard_normal(coarse)
    rr = spectral.restrict(spectral.prolong(r, fine), coarse)
    # identity on every coarse mode except the coarse Nyquist planes
    R = np.fft.fftn(r)
    for a, n in enumerate(coarse):
        idx = [slice(None)] * 3
        idx[a] = n // 2
        R[tuple(idx)] = 0.0
    assert np.allclose(rr, np.real(np.fft.ifftn(R)), atol=1e-12)
