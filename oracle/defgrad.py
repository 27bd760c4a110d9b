"""Deformation gradient and det F1 (Appendix, Deformation Gradient, eq. def-grad).

  partial_t F + (v . grad) F = (grad v) F,   F(0) = I,   periodic,
with (grad v)_{ab} = d_b v_a (FD8).  In SL form d_t F = (grad v) F along +v;
one RK2 step per component (Sec. 2.5.2, reading C-5 for the corrector sign):
  f0 = (grad v)(y) F^j(y);  F~ = F^j(y) + h_t f0;  f1 = (grad v)(x) F~;
  F^{j+1}(x) = F^j(y) + (h_t / 2)(f0 + f1).
det F1 = det F(t = 1) is the surrogate for det grad y (reading C-12); the
admissibility bound is eps_D < det F1 < 1 / eps_D with eps_D = 0.1 (Sec. 2.6).
"""

import numpy as np

from .fd8 import grad8
from .interp import interp_many
from .transport import departure_points


def deformation_gradient(v, nt, y=None):
    """F(t = 1) as an array (3, 3, n1, n2, n3)."""
    v = np.asarray(v, dtype=np.float64)
    shape = v.shape[1:]
    ht = 1.0 / nt
    if y is None:
        y = departure_points(v, nt, +1)
    A = np.stack([grad8(v[a]) for a in range(3)])          # A[a, b] = d_b v_a
    A_y = np.stack(interp_many([A[a, b] for a in range(3) for b in range(3)], y)).reshape(
        (3, 3) + shape)
    F = np.zeros((3, 3) + shape)
    for a in range(3):
        F[a, a] = 1.0
    for _ in range(nt):
        F_y = np.stack(interp_many([F[a, b] for a in range(3) for b in range(3)], y)).reshape(
            (3, 3) + shape)
        f0 = np.einsum("ac...,cb...->ab...", A_y, F_y)
        F_tilde = F_y + ht * f0
        f1 = np.einsum("ac...,cb...->ab...", A, F_tilde)
        F = F_y + 0.5 * ht * (f0 + f1)
    return F


def det3(F):
    """Determinant of a field of 3x3 matrices (3, 3, ...) by cofactor expansion."""
    return (F[0, 0] * (F[1, 1] * F[2, 2] - F[1, 2] * F[2, 1])
            - F[0, 1] * (F[1, 0] * F[2, 2] - F[1, 2] * F[2, 0])
            + F[0, 2] * (F[1, 0] * F[2, 1] - F[1, 1] * F[2, 0]))


def det_deformation_gradient(v, nt):
    """det F1 on the grid, plus (min, max, mean)."""
    d = det3(deformation_gradient(v, nt))
    return d, (float(d.min()), float(d.max()), float(d.mean()))
