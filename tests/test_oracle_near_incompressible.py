"""Pin of the near-incompressible gradient term c(kappa) P_par b (Appendix,
"(near-)incompressible diffeomorphisms"; reading C-2).

The Appendix obtains the reduced gradient by eliminating the constraint
div v = w and its dual variable rho from the optimality system of a problem
with a second control w regularised with weight beta.  For a data term whose
gradient is a fixed body force b, that problem is the quadratic

    Phi(v) = <b, v> + (alpha / 2) <v, L v> + (beta / 2) <div v, B div v>,

and eliminating rho = beta B div v gives the gradient
alpha L v + b - grad (beta B)(alpha + beta B)^-1 Lap^-1 div b.  The printed
operator (alpha (beta (-Lap^-1 + id))^-1 + id)^-1 is (beta B)(alpha + beta B)^-1
with B = -Lap^-1 + id, whose symbol with kappa = |k|^2 is the oracle's
c(kappa) = beta (1 + kappa) / (beta (1 + kappa) + alpha kappa).

So the oracle's gradient alpha L v + b - c(kappa) P_par b must vanish at the
minimiser of Phi, computed here independently of the oracle (NumPy's complex
FFT, per-mode 3 x 3 solves of (alpha kappa I + beta (1 + kappa) / kappa k k^T)
v^ = -b^, L = -Lap).  Planted mistakes in c(kappa) (a dropped 1 + kappa, alpha
and beta exchanged, the H^1 operator id - Lap for B, the full Leray weight 1)
and a flipped sign of the term each leave a gradient far from zero.
"""

import numpy as np
import pytest

from oracle import spectral as OS

SHAPE = (12, 10, 14)
ALPHA = 1e-2


def _bandlimited_vector_field(seed, kmax=3):
    rng = np.random.default_rng(seed)
    k = [np.fft.fftfreq(n, 1.0 / n) for n in SHAPE]
    K = np.stack(np.meshgrid(*k, indexing="ij"))
    mask = (np.sum(K * K, axis=0) <= kmax ** 2) & (np.sum(K * K, axis=0) > 0)
    out = []
    for _ in range(3):
        c = (rng.standard_normal(SHAPE) + 1j * rng.standard_normal(SHAPE)) * mask
        out.append(np.real(np.fft.ifftn(c)))          # real part: a Hermitian spectrum
    return np.stack(out)


def _direct_minimiser(b, alpha, beta):
    """argmin Phi by one 3 x 3 solve per Fourier mode (the k = 0 mode of a
    zero-mean b stays zero)."""
    k = [np.fft.fftfreq(n, 1.0 / n) for n in SHAPE]
    K = np.stack(np.meshgrid(*k, indexing="ij"))
    Bh = np.stack([np.fft.fftn(b[a]) for a in range(3)])
    Vh = np.zeros_like(Bh)
    for idx in np.ndindex(SHAPE):
        kv = K[(slice(None),) + idx]
        kap = float(kv @ kv)
        if kap == 0.0:
            continue
        M = alpha * kap * np.eye(3) + beta * (1.0 + kap) / kap * np.outer(kv, kv)
        Vh[(slice(None),) + idx] = -np.linalg.solve(M, Bh[(slice(None),) + idx])
    return np.stack([np.real(np.fft.ifftn(Vh[a])) for a in range(3)])


def _gradient_residual(b, alpha, beta):
    v = _direct_minimiser(b, alpha, beta)
    g = OS.apply_reg(v, alpha, 1.0) + b - OS.near_incompressible_term(b, alpha, beta)
    return float(np.linalg.norm(g) / np.linalg.norm(b))


@pytest.mark.parametrize("beta", [1e-4, 1e-2, 1.0, 1e2])
def test_near_incompressible_gradient_vanishes_at_the_constrained_minimiser(beta):
    b = _bandlimited_vector_field(seed=int(1e4 * beta) % 97)
    assert _gradient_residual(b, ALPHA, beta) < 1e-12


def test_the_pin_sees_the_term_at_all():
    # the near-incompressible part is not negligible here: without it the
    # gradient at the minimiser is far from zero
    b = _bandlimited_vector_field(seed=3)
    v = _direct_minimiser(b, ALPHA, 1.0)
    g = OS.apply_reg(v, ALPHA, 1.0) + b
    assert np.linalg.norm(g) / np.linalg.norm(b) > 0.1


_PLANTED = {
    "dropped 1 + kappa": lambda kap, a, b: b / (b + a * kap),
    "alpha and beta exchanged": lambda kap, a, b: a * (1 + kap) / (a * (1 + kap) + b * kap),
    "B = id - Lap (H1)": lambda kap, a, b: b * (1 + kap) / (b * (1 + kap) + a),
    "full Leray weight": lambda kap, a, b: np.ones_like(kap),
}


@pytest.mark.parametrize("name", sorted(_PLANTED))
def test_planted_mistakes_in_the_weight_fail(monkeypatch, name):
    planted = _PLANTED[name]
    monkeypatch.setattr(OS, "near_incompressible_weight",
                        lambda shape, alpha, beta_w: planted(OS.kappa(shape), alpha, beta_w))
    b = _bandlimited_vector_field(seed=5)
    assert _gradient_residual(b, ALPHA, 1.0) > 1e-3          # beta != alpha


def test_planted_sign_flip_fails(monkeypatch):
    real = OS.near_incompressible_term
    monkeypatch.setattr(OS, "near_incompressible_term",
                        lambda b, alpha, beta_w: -real(b, alpha, beta_w))
    b = _bandlimited_vector_field(seed=7)
    assert _gradient_residual(b, ALPHA, 1e-2) > 1e-3
