"""Semi-Lagrangian transport solves (Sec. 2.5.2 Time Integration).

Every PDE of the optimality system is brought into the form d_t u = f with
the material derivative d_t = partial_t + w . grad along a transport velocity
w (eq. matderiv).  One SL step from time level j to j+1:

  1. departure points: y~ = x - h_t w(x);  y = x - (h_t / 2)(w(x) + w(y~))
     (RK2 characteristic, traced once because v is stationary);
  2. homogeneous (f = 0):  u^{j+1}(x) = u^j(y);
  3. non-homogeneous, RK2 along the characteristic:
       f0 = f at (y, t^j) using u^j(y);  u~ = u^j(y) + h_t f0;
       f1 = f at (x, t^{j+1}) using u~;  u^{j+1}(x) = u^j(y) + (h_t / 2)(f0 + f1).
     Reading C-5: the paper prints "-" in the corrector, which contradicts its
     predictor and d_t u = f; the oracle uses "+" (Heun's method).
  Differential operators in f are applied on the regular grid and the results
  interpolated (Sec. 2.5.2, last paragraph; reading C-6: products such as
  grad m . v~ are formed on the grid and gathered as one scalar).

The four solves:
  state        d_t m = 0 along +v, forward, m(0) = m0                  (eq. transport)
  adjoint      -d_t lam - div(lam v) = 0, backward, lam(1) = -(m(1)-m1) (eq. adjoint)
  inc. state   d_t m~ = -grad m . v~ along +v, forward, m~(0) = 0       (eq. incstate)
  inc. adjoint -d_t lam~ - div(lam~ v + lam v~) = 0, backward,
               lam~(1) = -m~(1)                                          (eq. incadj)
Reading C-4: both adjoint equations carry "- div" (derived from the
Lagrangian, eq. lagrangian, by integration by parts).  In backward time
tau = 1 - t they are transport along -v with source lam div v (+ div(lam v~)).
"""

import numpy as np

from .grid import spacing, index_coordinates
from .interp import interp, interp_many
from .fd8 import grad8, div8


def departure_points(v, nt, direction=+1):
    """RK2 departure points in grid units for transport velocity w = direction * v.

    direction = +1: forward solves (state, incremental state);
    direction = -1: backward solves (adjoint, incremental adjoint).
    Returns q of shape (3, n1, n2, n3): y / h per axis (x_l / h = l).
    """
    v = np.asarray(v, dtype=np.float64)
    shape = v.shape[1:]
    h = spacing(shape)
    ht = 1.0 / nt
    x = index_coordinates(shape)
    w = direction * v
    # y~ = x - h_t w(x), expressed in grid units per axis
    y_tilde = np.stack([x[a] - ht * w[a] / h[a] for a in range(3)])
    w_at_ytilde = interp_many([w[0], w[1], w[2]], y_tilde)
    return np.stack([x[a] - 0.5 * ht * (w[a] + w_at_ytilde[a]) / h[a] for a in range(3)])


def state_solve(m0, v, nt, y=None):
    """m^j, j = 0..nt, of eq. (transport): homogeneous SL steps along +v."""
    if y is None:
        y = departure_points(v, nt, +1)
    m = [np.asarray(m0, dtype=np.float64)]
    for _ in range(nt):
        m.append(interp(m[-1], y))
    return m


def adjoint_solve(lam1, v, nt, y=None):
    """lam^j, j = 0..nt, of eq. (adjoint), solved backward from lam^nt = lam1.

    Backward step t^{j+1} -> t^j along -v with f = lam * D, D = div v (FD8):
      f0 = lam^{j+1}(y) D(y);  u~ = lam^{j+1}(y) + h_t f0;
      f1 = u~ D(x);            lam^j(x) = lam^{j+1}(y) + (h_t/2)(f0 + f1).
    """
    ht = 1.0 / nt
    if y is None:
        y = departure_points(v, nt, -1)
    D = div8(v)
    D_y = interp(D, y)
    lam = [None] * (nt + 1)
    lam[nt] = np.asarray(lam1, dtype=np.float64)
    for j in range(nt - 1, -1, -1):
        u_y = interp(lam[j + 1], y)
        f0 = u_y * D_y
        u_tilde = u_y + ht * f0
        f1 = u_tilde * D
        lam[j] = u_y + 0.5 * ht * (f0 + f1)
    return lam


def incremental_state_solve(m_hist, vt, v, nt, y=None):
    """m~^j, j = 0..nt, of eq. (incstate) with m~^0 = 0.

    f = -grad m . v~; s^j = grad8(m^j) . v~ is formed on the grid (reading C-6):
      f0 = -s^j(y);  u~ = m~^j(y) + h_t f0;  f1 = -s^{j+1}(x);
      m~^{j+1}(x) = m~^j(y) + (h_t/2)(f0 + f1).
    """
    ht = 1.0 / nt
    if y is None:
        y = departure_points(v, nt, +1)
    vt = np.asarray(vt, dtype=np.float64)
    s = [np.sum(grad8(mj) * vt, axis=0) for mj in m_hist]
    mt = [np.zeros_like(m_hist[0])]
    for j in range(nt):
        u_y = interp(mt[j], y)
        f0 = -interp(s[j], y)
        # the predictor u~ = m~^j(y) + h_t f0 is not needed: f1 does not depend on u
        f1 = -s[j + 1]
        mt.append(u_y + 0.5 * ht * (f0 + f1))
    return mt


def incremental_adjoint_solve(mt1, v, nt, lam_hist=None, vt=None, y=None, final=None):
    """lam~^j, j = 0..nt, of eq. (incadj), solved backward from lam~^nt = -m~(1)
    (or from the given final condition, e.g. the NCC one of the Appendix).

    Gauss-Newton (lam_hist is None): every lam term dropped (Sec. 2.5.5), so
    lam~ obeys the adjoint equation.  Full Newton: source q^j = div8(lam^j v~):
      f0 = lam~^{j+1}(y) D(y) + q^{j+1}(y);  u~ = lam~^{j+1}(y) + h_t f0;
      f1 = u~ D(x) + q^j(x);  lam~^j(x) = lam~^{j+1}(y) + (h_t/2)(f0 + f1).
    """
    ht = 1.0 / nt
    if y is None:
        y = departure_points(v, nt, -1)
    D = div8(v)
    D_y = interp(D, y)
    if lam_hist is not None:
        vt = np.asarray(vt, dtype=np.float64)
        q = [div8(lam_j[None] * vt) for lam_j in lam_hist]
    lt = [None] * (nt + 1)
    lt[nt] = -np.asarray(mt1, dtype=np.float64) if final is None else np.asarray(final, dtype=np.float64)
    for j in range(nt - 1, -1, -1):
        u_y = interp(lt[j + 1], y)
        f0 = u_y * D_y
        if lam_hist is not None:
            f0 = f0 + interp(q[j + 1], y)
        u_tilde = u_y + ht * f0
        f1 = u_tilde * D
        if lam_hist is not None:
            f1 = f1 + q[j]
        lt[j] = u_y + 0.5 * ht * (f0 + f1)
    return lt


def trapezoid_weights(nt):
    """h_t * (1/2, 1, ..., 1, 1/2): trapezoidal rule in time (Sec. 2.5.1)."""
    w = np.full(nt + 1, 1.0 / nt)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w
