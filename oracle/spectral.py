"""Pseudo-spectral operators (Sec. 2.5.3, Sec. 2.5.5, Appendix).

Fields are expanded in the Fourier basis of the periodic grid with integer
wavenumbers (Sec. 2.5.3); a diagonal operator multiplies each coefficient by
its symbol.  Transforms are scipy.fft rfftn/irfftn (library routines).

* Regulariser L = (-Laplacian)^gamma, symbol |k|^(2 gamma)      (Sec. 2.2; gamma = 1
  is the H1 seminorm, L = -Laplacian; reading C-2 for the meaning of gamma).
* Preconditioner (alpha L)^-1 with zero symbols set to one before inverting
  (Sec. 2.5.5, reading C-3: the mean mode is scaled by 1/alpha).
* Leray projection: the gradient part P_par b = grad Lap^-1 div b, symbol
  k k^T / |k|^2, and its weighted near-incompressible form c(kappa) P_par b
  (Appendix, (near-)incompressible diffeomorphisms; reading C-2).
* Spectral restriction / prolongation between grids of n and n/2 points by
  truncating / zero-padding the Fourier coefficients (Sec. 2.5.6).
"""

import numpy as np
import scipy.fft as sfft

from .grid import rfft_wavenumbers, nyquist_zeroed, wavenumber

WORKERS = -1


def _rfft(u):
    return sfft.rfftn(u, workers=WORKERS)


def _irfft(U, shape):
    return sfft.irfftn(U, s=shape, workers=WORKERS)


def kappa(shape):
    """|k|^2 over the half spectrum (symbol of -Laplacian)."""
    k1, k2, k3 = rfft_wavenumbers(shape)
    return k1 * k1 + k2 * k2 + k3 * k3


def reg_symbol(shape, gamma):
    """Symbol of L = (-Laplacian)^gamma: |k|^(2 gamma), 0 at k = 0."""
    return kappa(shape) ** gamma


def apply_L(v, gamma):
    """L v for a vector field (3, n1, n2, n3), component by component."""
    v = np.asarray(v, dtype=np.float64)
    shape = v.shape[1:]
    sig = reg_symbol(shape, gamma)
    return np.stack([_irfft(sig * _rfft(v[a]), shape) for a in range(3)])


def apply_reg(v, alpha, gamma):
    """H_reg v = alpha L v (Sec. 2.5.6, regularisation part of the Hessian)."""
    return alpha * apply_L(v, gamma)


def apply_reg_inverse(r, alpha, gamma):
    """(alpha L)^-1 r with the zero symbol (k = 0) replaced by one (reading C-3)."""
    r = np.asarray(r, dtype=np.float64)
    shape = r.shape[1:]
    sig = reg_symbol(shape, gamma)
    sig = np.where(sig == 0.0, 1.0, sig)
    return np.stack([_irfft(_rfft(r[a]) / (alpha * sig), shape) for a in range(3)])


def _odd_wavenumbers(shape):
    """Wavenumber vector with Nyquist entries zeroed (keeps k k^T real-symmetric)."""
    n1, n2, n3 = shape
    k1 = nyquist_zeroed(wavenumber(n1), n1)[:, None, None]
    k2 = nyquist_zeroed(wavenumber(n2), n2)[None, :, None]
    k3 = nyquist_zeroed(np.arange(n3 // 2 + 1, dtype=np.float64), n3)[None, None, :]
    return k1, k2, k3


def leray_parallel(b):
    """P_par b = grad Lap^-1 div b: Fourier symbol k (k . b_hat) / |k|^2.

    Both grad and div carry a factor i k; their product with Lap^-1 = -1/|k|^2
    gives the real symbol k k^T / |k|^2.  Nyquist components of k are zeroed
    so the projection maps real fields to real fields; k = 0 maps to 0.
    """
    b = np.asarray(b, dtype=np.float64)
    shape = b.shape[1:]
    ks = _odd_wavenumbers(shape)
    kk = ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2
    B = [_rfft(b[a]) for a in range(3)]
    kdotb = ks[0] * B[0] + ks[1] * B[1] + ks[2] * B[2]
    inv = np.where(kk > 0.0, 1.0 / np.where(kk > 0.0, kk, 1.0), 0.0)
    return np.stack([_irfft(ks[a] * kdotb * inv, shape) for a in range(3)])


def leray(b):
    """Divergence-free part b - P_par b (Appendix, incompressible gradient)."""
    return np.asarray(b, dtype=np.float64) - leray_parallel(b)


def near_incompressible_weight(shape, alpha, beta_w):
    """c(kappa) = beta_w (1 + kappa) / (beta_w (1 + kappa) + alpha kappa).

    Reading C-2 of the Appendix's garbled near-incompressible gradient
    grad (alpha (beta (-Lap^-1 + id))^-1 + id)^-1 Lap^-1 div, with kappa = |k|^2.
    beta_w -> infinity gives 1 (full Leray), beta_w = 0 gives 0.  The printed
    operator is (beta B)(alpha + beta B)^-1 with B = -Lap^-1 + id: the weight of
    the gradient obtained by eliminating div v = w and its dual variable from a
    problem whose second control w is regularised by (beta / 2) <w, B w>.
    """
    kap = kappa(shape)
    num = beta_w * (1.0 + kap)
    return num / (num + alpha * kap)


def near_incompressible_term(b, alpha, beta_w):
    """c(kappa) P_par b: the term subtracted from the gradient when beta_w > 0."""
    b = np.asarray(b, dtype=np.float64)
    shape = b.shape[1:]
    if beta_w == 0.0:
        return np.zeros_like(b)
    c = near_incompressible_weight(shape, alpha, beta_w)
    ks = _odd_wavenumbers(shape)
    kk = ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2
    B = [_rfft(b[a]) for a in range(3)]
    kdotb = ks[0] * B[0] + ks[1] * B[1] + ks[2] * B[2]
    inv = np.where(kk > 0.0, 1.0 / np.where(kk > 0.0, kk, 1.0), 0.0)
    return np.stack([_irfft(c * ks[a] * kdotb * inv, shape) for a in range(3)])


def _band_mask(fine_shape, coarse_shape):
    """Fine-grid modes representable on the coarse grid (coarse Nyquist dropped)."""
    masks = []
    for nf, nc in zip(fine_shape, coarse_shape):
        k = wavenumber(nf)
        masks.append(np.abs(k) < nc // 2)
    return masks


def restrict(u, coarse_shape):
    """Spectral restriction of a scalar field to a coarser periodic grid.

    Keeps the Fourier coefficients with |k_i| < n_i^c / 2 on every axis (the
    coarse Nyquist mode is dropped) and evaluates them on the coarse nodes.
    """
    u = np.asarray(u, dtype=np.float64)
    fine_shape = u.shape
    U = sfft.fftn(u, workers=WORKERS)
    m = _band_mask(fine_shape, coarse_shape)
    Uc = np.zeros(coarse_shape, dtype=np.complex128)
    kc = [wavenumber(n) for n in coarse_shape]
    kf = [wavenumber(n) for n in fine_shape]
    src = [np.nonzero(m[a])[0] for a in range(3)]
    dst = [np.array([int(np.nonzero(kc[a] == kf[a][i])[0][0]) for i in src[a]]) for a in range(3)]
    Uc[np.ix_(dst[0], dst[1], dst[2])] = U[np.ix_(src[0], src[1], src[2])]
    scale = np.prod(coarse_shape) / np.prod(fine_shape)
    return np.real(sfft.ifftn(Uc * scale, workers=WORKERS))


def prolong(u, fine_shape):
    """Spectral prolongation (zero padding) of a scalar field to a finer grid."""
    u = np.asarray(u, dtype=np.float64)
    coarse_shape = u.shape
    U = sfft.fftn(u, workers=WORKERS)
    kc = [wavenumber(n) for n in coarse_shape]
    kf = [wavenumber(n) for n in fine_shape]
    keep = [np.nonzero(np.abs(kc[a]) < coarse_shape[a] // 2)[0] for a in range(3)]
    dst = [np.array([int(np.nonzero(kf[a] == kc[a][i])[0][0]) for i in keep[a]]) for a in range(3)]
    Uf = np.zeros(fine_shape, dtype=np.complex128)
    Uf[np.ix_(dst[0], dst[1], dst[2])] = U[np.ix_(keep[0], keep[1], keep[2])]
    scale = np.prod(fine_shape) / np.prod(coarse_shape)
    return np.real(sfft.ifftn(Uf * scale, workers=WORKERS))
