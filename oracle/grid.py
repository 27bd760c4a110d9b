"""Nodal periodic grid (Sec. 2.5.1 Discretization).

The domain is Omega = [-pi, pi)^3 with n_i nodes per axis and spacing
h_i = 2 pi / n_i; time is split into n_t steps of length h_t = 1 / n_t.

Reading C-1: the paper writes the node coordinates as ((n/2) - l) * h, which
decreases with the index while its printed FD8 stencil and its Fourier sign
assume the opposite orientation.  The oracle places x_l = l * h, increasing
with the array index, so "+x" along an axis is "+1" in the index.  Even-order
spectral operators do not depend on the orientation.

Arrays are C-ordered [n1][n2][n3] with x3 fastest (Sec. 2.5.3 keeps the
innermost x3 direction contiguous); vector fields are [3][n1][n2][n3].
"""

import numpy as np


def spacing(shape):
    """h_i = 2 pi / n_i for each axis (Sec. 2.5.1)."""
    return tuple(2.0 * np.pi / n for n in shape)


def cell_volume(shape):
    """h1 h2 h3: weight of the trapezoidal rule in space on a periodic grid."""
    h = spacing(shape)
    return h[0] * h[1] * h[2]


def index_coordinates(shape):
    """Node positions in grid units (x_l / h = l), shape (3, n1, n2, n3)."""
    return np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape],
                                indexing="ij"))


def wavenumber(n):
    """Integer wavenumbers of an n-point periodic axis in FFT order.

    The paper's expansion runs over k = -n/2+1 .. n/2 (Sec. 2.5.3).  Index n/2
    (even n) is the Nyquist mode; its magnitude is n/2 in either convention.
    """
    k = np.arange(n, dtype=np.float64)
    k[k > n // 2] -= n
    return k


def rfft_wavenumbers(shape):
    """(k1, k2, k3) broadcastable over the half spectrum of rfftn."""
    n1, n2, n3 = shape
    k1 = wavenumber(n1)[:, None, None]
    k2 = wavenumber(n2)[None, :, None]
    k3 = np.arange(n3 // 2 + 1, dtype=np.float64)[None, None, :]
    return k1, k2, k3


def nyquist_zeroed(k, n):
    """Wavenumber vector with the Nyquist entry set to 0 (for odd-order factors)."""
    out = np.array(k, dtype=np.float64, copy=True)
    if n % 2 == 0:
        out[np.abs(out) == n // 2] = 0.0
    return out
