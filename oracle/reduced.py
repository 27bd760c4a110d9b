"""Reduced-space objective, gradient and Hessian matvec (Sec. 2.2 - 2.4).

  J(v)  = 1/2 int (m(1) - m1)^2 dx + alpha/2 <L v, v>            (eq. varopt-claire)
  g(v)  = alpha L v + int_0^1 lam grad m dt                        (eq. rgrad)
  H v~  = alpha L v~ + int_0^1 (lam~ grad m + lam grad m~) dt      (eq. matvec)
Gauss-Newton (Sec. 2.5.5): drop every term with lam in eq. (matvec) and eq.
(incadj); this is the default (reading C-7).  Space integrals are h1 h2 h3 * sum
(trapezoid on a periodic grid), time integrals the trapezoidal rule with n_t
steps (Sec. 2.5.1).  grad is FD8 (Sec. 2.5.3), L is spectral.

Near-incompressible model (Appendix, reading C-2): with beta_w > 0 the data
part b of the gradient (and of the Hessian) is replaced by b - c(kappa) P_par b.
beta_w = 0 (the default) is the plain H1-seminorm problem of Sec. 2.2.

Distances (Problem.distance): "l2" is 1/2 ||m(1) - m1||^2 (eq. varopt-claire);
"ncc" is the normalised cross correlation of the Appendix,
1 - <m(1), m1>^2 / (<m1, m1> <m(1), m(1)>), which changes only the final
conditions lam(1) = -d dist / d m(1) and, for the Hessian, lam~(1) =
-(d^2 dist / d m(1)^2)[m~(1)] (reading C-16 for the sign of the printed q1).
"""

from dataclasses import dataclass, field

import numpy as np

from .grid import cell_volume
from .fd8 import grad8
from .spectral import apply_L, near_incompressible_term
from .transport import (departure_points, state_solve, adjoint_solve,
                        incremental_state_solve, incremental_adjoint_solve,
                        trapezoid_weights)


@dataclass
class Problem:
    """One registration problem: images, time steps and regularisation."""
    m0: np.ndarray
    m1: np.ndarray
    nt: int = 4
    beta_v: float = 1e-2      # alpha in the paper
    gamma: float = 1.0        # exponent of L = (-Laplacian)^gamma (reading C-2)
    beta_w: float = 0.0       # divergence penalty weight (Appendix)
    distance: str = "l2"      # or "ncc" (Appendix, normalised cross correlation)

    def __post_init__(self):
        self.m0 = np.asarray(self.m0, dtype=np.float64)
        self.m1 = np.asarray(self.m1, dtype=np.float64)

    @property
    def shape(self):
        return self.m0.shape

    @property
    def h3(self):
        return cell_volume(self.shape)


@dataclass
class Evaluation:
    """State of Algorithm 1 at one iterate v (lines 3-6)."""
    v: np.ndarray
    y_f: np.ndarray
    m: list
    J: float
    mismatch: float
    y_b: np.ndarray = None
    lam: list = None
    g: np.ndarray = None
    extra: dict = field(default_factory=dict)


def inner(prob, a, b):
    """L2 inner product <a, b> = h1 h2 h3 sum a b (Appendix, NCC)."""
    return prob.h3 * float(np.sum(np.asarray(a, dtype=np.float64) * b))


def distance(prob, m_end):
    """dist(m(1), m1): 1/2 ||m(1) - m1||^2 or the NCC distance of the Appendix."""
    if prob.distance == "ncc":
        a = inner(prob, m_end, prob.m1)
        return 1.0 - a * a / (inner(prob, prob.m1, prob.m1) * inner(prob, m_end, m_end))
    return 0.5 * prob.h3 * float(np.sum((m_end - prob.m1) ** 2))


def adjoint_final(prob, m_end):
    """lam(1) = -d dist / d m(1): m1 - m(1) (eq. adjfinal) or, for NCC (Appendix),
    -2 <m1, m> / (||m||^2 ||m1||^2) (<m1, m> / ||m||^2 m - m1)."""
    if prob.distance == "ncc":
        a = inner(prob, m_end, prob.m1)
        b = inner(prob, prob.m1, prob.m1)
        c = inner(prob, m_end, m_end)
        return -2.0 * a / (c * b) * (a / c * m_end - prob.m1)
    return -(m_end - prob.m1)


def incremental_adjoint_final(prob, m_end, mt_end):
    """lam~(1) = -(d^2 dist / d m(1)^2)[m~(1)] (Gauss-Newton and full Newton).

    L2: -m~(1).  NCC (Appendix): 2 (q1 m1 + q2 m(1) - q3 m~(1)) / ||m1||^2 with
    q2, q3 as printed and q1 = <m1, m~>/||m||^2 - 2 <m1, m><m, m~>/||m||^4, the
    negative of the printed q1 (reading C-16: the printed sign is not the
    derivative of the printed lam(1); the test suite checks both by finite
    differences).
    """
    mt_end = np.asarray(mt_end, dtype=np.float64)
    if prob.distance == "ncc":
        a = inner(prob, prob.m1, m_end)
        b = inner(prob, prob.m1, prob.m1)
        c = inner(prob, m_end, m_end)
        al = inner(prob, prob.m1, mt_end)
        ga = inner(prob, m_end, mt_end)
        q1 = al / c - 2.0 * a * ga / c ** 2
        q2 = 4.0 * a * a * ga / c ** 3 - 2.0 * a * al / c ** 2
        q3 = a * a / c ** 2
        return 2.0 * (q1 * prob.m1 + q2 * m_end - q3 * mt_end) / b
    return -mt_end


def objective_terms(prob, v, m_end):
    """(J, distance, regularisation) for m(1) = m_end at velocity v."""
    v = np.asarray(v, dtype=np.float64)
    dist = distance(prob, m_end)
    reg = 0.5 * prob.beta_v * prob.h3 * np.sum(v * apply_L(v, prob.gamma))
    return dist + reg, dist, reg


def evaluate_objective(prob, v):
    """State solve and objective (Algorithm 1, lines 3-4)."""
    v = np.asarray(v, dtype=np.float64)
    y_f = departure_points(v, prob.nt, +1)
    m = state_solve(prob.m0, v, prob.nt, y_f)
    J, dist, _ = objective_terms(prob, v, m[-1])
    return Evaluation(v=v, y_f=y_f, m=m, J=J, mismatch=dist)


def data_term(prob, b):
    """b or b - c(kappa) P_par b (near-incompressible model)."""
    if prob.beta_w == 0.0:
        return b
    return b - near_incompressible_term(b, prob.beta_v, prob.beta_w)


def complete_gradient(prob, ev):
    """Adjoint solve and reduced gradient (Algorithm 1, lines 5-6), in place."""
    nt = prob.nt
    ev.y_b = departure_points(ev.v, nt, -1)
    lam1 = adjoint_final(prob, ev.m[nt])               # eq. (adjfinal)
    ev.lam = adjoint_solve(lam1, ev.v, nt, ev.y_b)
    w = trapezoid_weights(nt)
    b = np.zeros_like(ev.v)
    for j in range(nt + 1):
        b += w[j] * ev.lam[j][None] * grad8(ev.m[j])
    ev.g = prob.beta_v * apply_L(ev.v, prob.gamma) + data_term(prob, b)
    return ev


def evaluate(prob, v):
    """J, g and the stored state/adjoint histories at v (Algorithm 1, lines 3-6)."""
    return complete_gradient(prob, evaluate_objective(prob, v))


def hessian_matvec(prob, ev, vt, full_newton=False):
    """H v~ at the evaluation point ev (eq. matvec; Gauss-Newton by default).

    Incremental state forward (eq. incstate), incremental adjoint backward
    (eq. incadj), then alpha L v~ + int (lam~ grad m [+ lam grad m~]) dt.
    """
    nt = prob.nt
    vt = np.asarray(vt, dtype=np.float64)
    mt = incremental_state_solve(ev.m, vt, ev.v, nt, ev.y_f)
    lt = incremental_adjoint_solve(mt[nt], ev.v, nt,
                                   ev.lam if full_newton else None, vt, ev.y_b,
                                   final=incremental_adjoint_final(prob, ev.m[nt], mt[nt]))
    w = trapezoid_weights(nt)
    bt = np.zeros_like(vt)
    for j in range(nt + 1):
        bt += w[j] * lt[j][None] * grad8(ev.m[j])
        if full_newton:
            bt += w[j] * ev.lam[j][None] * grad8(mt[j])
    return prob.beta_v * apply_L(vt, prob.gamma) + data_term(prob, bt)


def gradient_at_zero(prob):
    """g(v = 0): the relative-gradient denominator of reading C-10."""
    return evaluate(prob, np.zeros((3,) + prob.shape)).g
