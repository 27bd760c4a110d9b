"""Two-level zero-velocity preconditioner (Sec. 2.5.6, "Two-Level
Preconditioner" and "Zero Velocity Approximation"; the default of Sec. 2.6).

TEST INFRASTRUCTURE ONLY: plain FP64 restatement used to check the CUDA path.

Zero-velocity Hessian (Sec. 2.5.6): at v = 0 the state is constant in time,
the incremental state at t = 1 is -grad m . v~ and the Gauss-Newton
incremental adjoint is grad m . v~, so

    H0 v~ = alpha L v~ + (grad m (x) grad m) v~,

with m the current m(t = 1) in place of m0 (the paper's remedy for iterates
away from v = 0).

Two-level scheme, applied to the regularisation-preconditioned system
(I + R^-1/2 H_dat R^-1/2) w = -R^-1/2 g, w = R^1/2 v~ (R = H_reg):

    M^-1 r = Q_P (M~_L)^-1 Q_R F_L r + F_H r,

with spectral restriction Q_R / prolongation Q_P to the grid of half the
resolution, cut-off filters F_L + F_H = I, and the coarse operator M~_L the
directly discretised zero-velocity Hessian of the same system,
I + R_c^-1/2 (grad m_c (x) grad m_c) R_c^-1/2, inverted by a nested CG whose
relative tolerance is a tenth of the outer PCG's.

Readings (reading C-15):
* R = alpha L with the zero symbol set to one, the operator of the spectral
  preconditioner (reading C-3); R^-1/2 is its spectral square root.
* PCG stays in v~: preconditioning H with R^-1/2 M^-1 R^-1/2 generates the
  same iterates v~ = R^-1/2 w as PCG on the split system.
* m_c is the spectral restriction of m(1); grad m_c is FD8 on the coarse grid.
* The nested solver is unpreconditioned CG from zero, stopped at
  ||res|| <= rtol ||rhs|| or after max_iter iterations.
* Q_R F_L = restriction (modes |k_i| < n_i / 4), Q_P F_L = prolongation, and
  F_H t = t - Q_P Q_R t.  The near-incompressible term is not part of H0.
"""

import numpy as np

from .fd8 import grad8
from .spectral import _rfft, _irfft, reg_symbol, apply_L, restrict, prolong


def apply_reg_inv_sqrt(r, alpha, gamma):
    """R^-1/2 r, symbol (alpha |k|^(2 gamma))^-1/2 with the zero symbol set to one."""
    r = np.asarray(r, dtype=np.float64)
    shape = r.shape[1:]
    sig = reg_symbol(shape, gamma)
    sig = np.where(sig == 0.0, 1.0, sig)
    f = 1.0 / np.sqrt(alpha * sig)
    return np.stack([_irfft(f * _rfft(r[a]), shape) for a in range(3)])


def h0_apply(vt, m, alpha, gamma):
    """H0 v~ = alpha L v~ + grad m (grad m . v~) on the grid of m."""
    vt = np.asarray(vt, dtype=np.float64)
    gm = grad8(m)
    return alpha * apply_L(vt, gamma) + gm * np.sum(gm * vt, axis=0)[None]


def coarse_operator(x, gm_c, alpha, gamma):
    """(I + R^-1/2 (grad m_c (x) grad m_c) R^-1/2) x on the coarse grid."""
    q = apply_reg_inv_sqrt(x, alpha, gamma)
    w = gm_c * np.sum(gm_c * q, axis=0)[None]
    return x + apply_reg_inv_sqrt(w, alpha, gamma)


def cg(apply_A, b, rtol, max_iter):
    """Conjugate gradients for A x = b from x = 0; returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    stop = rtol * np.sqrt(rr)
    it = 0
    while it < max_iter and np.sqrt(rr) > stop:
        Ap = apply_A(p)
        pAp = float(np.sum(p * Ap))
        if pAp <= 0.0:
            break
        a = rr / pAp
        x = x + a * p
        r = r - a * Ap
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def coarse_shape(shape):
    return tuple(n // 2 for n in shape)


def coarse_gradient(m):
    """FD8 gradient of the spectrally restricted image on the coarse grid."""
    return grad8(restrict(m, coarse_shape(m.shape)))


def restrict3(u, shape):
    return np.stack([restrict(u[a], shape) for a in range(3)])


def prolong3(u, shape):
    return np.stack([prolong(u[a], shape) for a in range(3)])


def two_level_inverse(r, m, alpha, gamma, rtol, max_iter=100, gm_c=None):
    """z = R^-1/2 M^-1 R^-1/2 r; returns (z, inner CG iterations)."""
    r = np.asarray(r, dtype=np.float64)
    fine = r.shape[1:]
    cs = coarse_shape(fine)
    if gm_c is None:
        gm_c = coarse_gradient(m)
    t = apply_reg_inv_sqrt(r, alpha, gamma)
    t_c = restrict3(t, cs)                         # Q_R F_L t
    t_high = t - prolong3(t_c, fine)               # F_H t
    s_c, its = cg(lambda x: coarse_operator(x, gm_c, alpha, gamma), t_c, rtol, max_iter)
    z = apply_reg_inv_sqrt(prolong3(s_c, fine) + t_high, alpha, gamma)
    return z, its
