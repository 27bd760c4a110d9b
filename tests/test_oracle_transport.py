"""Pins for oracle.transport (Sec. 2.5.2): identity, exact shifts, adjointness, mass.

P-1 zero velocity, P-2 constant velocity (closed form of the discrete scheme on
a Fourier mode, exact periodic shift), P-6 adjoint identity, P-7 mass
conservation of the continuity (adjoint) equation, and the v = 0 closed forms
of the incremental solves that Sec. 2.5.6 (zero velocity approximation) works out.
"""

import numpy as np
import pytest

from oracle import transport as T
from oracle.interp import lagrange_weights, interp
from oracle.fd8 import grad8, div8


def _x(shape):
    return np.meshgrid(*[np.arange(n) * 2 * np.pi / n for n in shape], indexing="ij")


def _const_v(shape, shift_vox_per_step, nt):
    """Constant velocity whose per-step displacement is shift_vox_per_step voxels."""
    h = [2 * np.pi / n for n in shape]
    return np.stack([np.full(shape, s * h[a] * nt) for a, s in enumerate(shift_vox_per_step)])


def test_zero_velocity_is_the_identity_bitwise():
    rng = np.random.default_rng(0)
    shape = (16, 18, 20)
    m0 = rng.standard_normal(shape)
    v = np.zeros((3,) + shape)
    y = T.departure_points(v, 4, +1)
    assert np.array_equal(y, np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in shape],
                                                  indexing="ij")))
    assert np.array_equal(T.state_solve(m0, v, 4)[-1], m0)
    assert np.array_equal(T.adjoint_solve(m0, v, 4)[0], m0)


def test_constant_velocity_departure_points_are_a_plain_shift():
    shape = (16, 16, 16)
    nt = 4
    v = _const_v(shape, (0.37, -1.25, 2.0), nt)
    q = T.departure_points(v, nt, +1)
    base = np.stack(np.meshgrid(*[np.arange(16.0)] * 3, indexing="ij"))
    shift = np.array([0.37, -1.25, 2.0])[:, None, None, None]
    assert np.allclose(q, base - shift, atol=1e-12)
    assert np.allclose(T.departure_points(v, nt, -1), base + shift, atol=1e-12)


def test_integer_shift_per_step_is_an_exact_roll():
    rng = np.random.default_rng(1)
    shape = (16, 20, 18)
    m0 = rng.standard_normal(shape)
    nt = 4
    v = _const_v(shape, (1.0, -2.0, 3.0), nt)
    m1 = T.state_solve(m0, v, nt)[-1]
    ref = np.roll(m0, shift=(4 * 1, 4 * -2, 4 * 3), axis=(0, 1, 2))
    assert np.allclose(m1, ref, atol=1e-12)


def test_fractional_shift_matches_closed_form_on_a_fourier_mode():
    shape = (16, 20, 24)
    nt = 4
    s = (0.3, -0.55, 1.7)                       # per-step shift in voxels
    v = _const_v(shape, s, nt)
    kvec = (2, -3, 5)
    x = _x(shape)
    phase = kvec[0] * x[0] + kvec[1] * x[1] + kvec[2] * x[2]
    m0 = np.cos(phase)
    m1 = T.state_solve(m0, v, nt)[-1]
    G = 1.0 + 0j
    for a in range(3):
        h = 2 * np.pi / shape[a]
        d = -s[a]                               # departure displacement, voxels
        p = np.floor(d)
        f = d - p
        w = lagrange_weights(np.array(f))
        G *= np.exp(1j * kvec[a] * p * h) * sum(w[i] * np.exp(1j * kvec[a] * (i - 1) * h)
                                                 for i in range(4))
    expect = np.real(G ** nt * np.exp(1j * phase))
    assert np.allclose(m1, expect, atol=1e-12)
    # and it approximates the continuous shift m0(x - v) to the interpolation error
    exact = np.cos(phase - sum(kvec[a] * v[a] for a in range(3)))
    kh = max(abs(kvec[a]) * 2 * np.pi / shape[a] for a in range(3))
    assert np.max(np.abs(m1 - exact)) < nt * kh ** 4


def test_adjoint_identity_is_exact_for_constant_velocity():
    rng = np.random.default_rng(2)
    shape = (16, 16, 18)
    nt = 4
    v = _const_v(shape, (0.41, -0.73, 1.3), nt)
    a = rng.standard_normal(shape)
    b = rng.standard_normal(shape)
    Aa = T.state_solve(a, v, nt)[-1]
    ATb = T.adjoint_solve(b, v, nt)[0]
    assert abs(np.sum(Aa * b) - np.sum(a * ATb)) < 1e-12 * np.sum(np.abs(a * b)) * 10


def _smooth_v(shape, amp=1.0):
    x = _x(shape)
    return amp * (0.3 * np.stack([np.sin(x[0] + 0.3), np.sin(x[1]), 0.5 * np.sin(x[2] - 0.2)])
                  + 0.1 * np.stack([np.cos(x[1]), np.sin(x[2]), np.cos(x[0])]))


def test_adjoint_identity_holds_to_discretisation_error_for_variable_velocity():
    shape = (16, 16, 16)
    x = _x(shape)
    v = _smooth_v(shape)
    a = np.exp(np.cos(x[0]) * np.sin(x[1] + x[2]))
    b = np.cos(x[0] + 2 * x[2]) + np.sin(x[1]) ** 2
    lhs = np.sum(T.state_solve(a, v, 4)[-1] * b)
    rhs = np.sum(a * T.adjoint_solve(b, v, 4)[0])
    assert abs(lhs - rhs) / np.sqrt(np.sum(a * a) * np.sum(b * b)) < 1e-2


def _adjoint_mass_drift(n, nt, solve=T.adjoint_solve):
    x = _x((n, n, n))
    lam = np.exp(np.cos(x[0] + 0.4) + 0.5 * np.sin(x[1] + x[2]))
    L = solve(lam, _smooth_v((n, n, n)), nt)
    return abs(L[0].sum() - L[nt].sum()) / np.abs(L[nt]).sum()


def test_adjoint_conserves_mass():
    assert _adjoint_mass_drift(32, 4) < 2e-3


@pytest.mark.slow
def test_adjoint_mass_drift_vanishes_under_refinement():
    assert _adjoint_mass_drift(64, 16) < 2e-5


def test_mass_pin_detects_a_wrong_corrector_sign(monkeypatch):
    """Plant the paper's printed '-' corrector (reading C-5) and check the pin fails."""
    def planted(lam1, v, nt, y=None):
        ht = 1.0 / nt
        y = T.departure_points(v, nt, -1)
        D = div8(v)
        D_y = interp(D, y)
        lam = [None] * (nt + 1)
        lam[nt] = lam1
        for j in range(nt - 1, -1, -1):
            u_y = interp(lam[j + 1], y)
            f0 = u_y * D_y
            f1 = (u_y + ht * f0) * D
            lam[j] = u_y - 0.5 * ht * (f0 + f1)
        return lam
    assert _adjoint_mass_drift(32, 4, planted) > 5e-3


def test_state_conserves_mass_for_divergence_free_velocity():
    shape = (32, 32, 32)
    x = _x(shape)
    psi = np.cos(x[0] + 2 * x[1]) + 0.5 * np.sin(x[2] - x[1])
    # curl of (0, 0, psi) + curl of (psi2, 0, 0): divergence-free by construction
    v = 0.4 * np.stack([-2 * np.sin(x[0] + 2 * x[1]) + 0.5 * np.cos(x[2] - x[1]),
                        np.sin(x[0] + 2 * x[1]), 0.3 * np.cos(x[0])])
    assert np.max(np.abs(div8(v))) < 1e-6
    m0 = np.exp(np.sin(x[0]) * np.cos(x[1]) + 0.3 * np.cos(x[2]))
    m1 = T.state_solve(m0, v, 4)[-1]
    assert abs(m1.sum() - m0.sum()) / m0.sum() < 1e-3
    assert abs((m1 ** 2).sum() - (m0 ** 2).sum()) / (m0 ** 2).sum() < 1e-3


def test_incremental_solves_at_zero_velocity_match_closed_forms():
    """Sec. 2.5.6: at v = 0, m~(t) = -t grad m0 . v~ and lam~(t) = grad m0 . v~ (GN);
    with the lam terms (full Newton) lam~(t) = grad m0 . v~ + (1 - t) div(lam0 v~)."""
    rng = np.random.default_rng(5)
    shape = (16, 16, 16)
    x = _x(shape)
    m0 = np.sin(x[0]) * np.cos(x[1] + x[2]) + 0.2 * rng.standard_normal(shape)
    lam0 = np.cos(x[2]) + 0.1 * rng.standard_normal(shape)
    vt = rng.standard_normal((3,) + shape)
    v = np.zeros((3,) + shape)
    nt = 4
    s = np.sum(grad8(m0) * vt, axis=0)
    q = div8(lam0[None] * vt)
    mt = T.incremental_state_solve([m0] * (nt + 1), vt, v, nt)
    for j in range(nt + 1):
        assert np.allclose(mt[j], -(j / nt) * s, atol=1e-12)
    lt = T.incremental_adjoint_solve(mt[nt], v, nt)
    for j in range(nt + 1):
        assert np.allclose(lt[j], s, atol=1e-12)
    lt_full = T.incremental_adjoint_solve(mt[nt], v, nt, lam_hist=[lam0] * (nt + 1), vt=vt)
    for j in range(nt + 1):
        assert np.allclose(lt_full[j], s + (1 - j / nt) * q, atol=1e-12)


def test_trapezoid_weights():
    w = T.trapezoid_weights(4)
    assert np.allclose(w, [0.125, 0.25, 0.25, 0.25, 0.125])
    assert abs(w.sum() - 1.0) < 1e-15
