"""3x3x3 periodic convolution and its adjoints in FP64 (learned warm start).

Not part of the paper's method: the U-Net that predicts an initial velocity
uses 3x3x3 convolutions with periodic padding on the periodic image grid.

  y[o](p) = sum_{c, t} w[o, c, t] x[c](p + off_t) + b[o]        (forward)
  dx[c](p) = sum_{o, t} w[o, c, t] dy[o](p - off_t)             (data gradient)
  dw[o, c, t] = sum_p dy[o](p) x[c](p + off_t)                   (weight gradient)
off_t = (dz, dy, dx) in {-1, 0, 1}^3, t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1);
arrays are x [C][D][H][W], w [O][C][27].  Written as one shifted sum per tap.
"""

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(a, off):
    """a(p + off) on the periodic grid (a has a leading channel axis)."""
    return np.roll(a, shift=(-off[0], -off[1], -off[2]), axis=(1, 2, 3))


def conv3d(x, w, b=None):
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    y = np.zeros((w.shape[0],) + x.shape[1:])
    for t, off in enumerate(OFFSETS):
        y += np.einsum("oc,czyx->ozyx", w[:, :, t], _shift(x, off))
    if b is not None:
        y += np.asarray(b, dtype=np.float64)[:, None, None, None]
    return y


def conv3d_data_grad(dy, w):
    dy = np.asarray(dy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dx = np.zeros((w.shape[1],) + dy.shape[1:])
    for t, off in enumerate(OFFSETS):
        dx += np.einsum("oc,ozyx->czyx", w[:, :, t], _shift(dy, (-off[0], -off[1], -off[2])))
    return dx


def conv3d_weight_grad(x, dy):
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    dw = np.zeros((dy.shape[0], x.shape[0], 27))
    for t, off in enumerate(OFFSETS):
        dw[:, :, t] = np.einsum("ozyx,czyx->oc", dy, _shift(x, off))
    return dw
