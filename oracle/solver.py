"""Inexact Gauss-Newton-Krylov solver (Sec. 2.5.5, 2.5.6, 2.6; Algorithms 1 and 2).

* pcg        Algorithm 2: matrix-free PCG for H v~ = -g with the spectral
             regularisation preconditioner M = alpha L (Sec. 2.5.6), or the
             two-level zero-velocity preconditioner of oracle.precond
             (Options.precond = "two_level"; nested CG tolerance a tenth of
             the outer PCG's relative tolerance eta).
             Reading C-8: stop when ||r||_2 <= eta ||g||_2 with the superlinear
             forcing eta = min(1/2, sqrt(||g^k||_inf / ||g^0||_inf)) (quadratic:
             without the square root).  Negative curvature <s, H s> <= 0 ends
             PCG with the previous iterate (Sec. 2.5.5).
* armijo     backtracking line search (reading C-9: gamma_0 = 1, factor 1/2,
             c1 = 1e-4, directional derivative h^3 sum g . v~, at most 10 halvings).
* gauss_newton  Algorithm 1 with the stopping rule ||g^k||_inf <= eps_opt
             ||g^0||_inf or ||g^k||_inf <= 1e-6 (Sec. 2.5.5); g^0 is the gradient
             at v = 0 (reading C-10).
* continuation  solve for a decreasing sequence of beta_v, warm-starting each
             level from the previous one (Sec. 2.6).
Inner products are FP64 sums over all voxels and components.
"""

from dataclasses import dataclass, field

import numpy as np

from .reduced import evaluate, evaluate_objective, complete_gradient, hessian_matvec, distance
from .spectral import apply_reg_inverse
from .precond import two_level_inverse, coarse_gradient

OK, ENOTCONV, ENEGCURV, ELINESEARCH = 0, 5, 6, 7


@dataclass
class Options:
    eps_opt: float = 5e-2
    max_newton: int = 50
    max_pcg: int = 100
    fixed_iters: bool = False     # run exactly max_newton x max_pcg (parity runs)
    forcing: str = "superlinear"  # or "quadratic"
    full_newton: bool = False
    precond: str = "spectral"     # or "two_level" (Sec. 2.5.6)
    max_inner: int = 100          # nested CG iterations per two-level application
    c1: float = 1e-4
    max_halvings: int = 10
    gabs_tol: float = 1e-6


@dataclass
class Stats:
    newton_iters: int = 0
    pcg_iters: int = 0
    matvecs: int = 0
    pde_solves: int = 0
    linesearch_halvings: int = 0
    inner_iters: int = 0
    J0: float = 0.0
    J: float = 0.0
    mismatch_rel: float = 0.0
    grad_rel: float = 0.0
    status: int = OK
    history: list = field(default_factory=list)


def dot(a, b):
    return float(np.sum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))


def pcg(apply_H, apply_Minv, g, tol, max_iter, fixed=False):
    """Algorithm 2: PCG for H v~ = -g starting from v~ = 0.

    Returns (v~, iterations, matvecs, status).  tol is the absolute 2-norm
    threshold on the residual (the caller forms eta ||g||_2).
    """
    vt = np.zeros_like(g)
    r = -g
    z = apply_Minv(r)
    s = z.copy()
    rz = dot(r, z)
    matvecs = 0
    it = 0
    status = OK
    for it in range(1, max_iter + 1):
        Hs = apply_H(s)
        matvecs += 1
        sHs = dot(s, Hs)
        if sHs <= 0.0:
            status = ENEGCURV
            if it == 1:
                vt = s          # no previous iterate: take the preconditioned gradient
            it -= 1
            break
        kappa = rz / sHs
        vt = vt + kappa * s
        r = r - kappa * Hs
        if not fixed and np.sqrt(dot(r, r)) < tol:
            break
        z = apply_Minv(r)
        rz_new = dot(z, r)
        mu = rz_new / rz
        rz = rz_new
        s = z + mu * s
    return vt, it, matvecs, status


def armijo(prob, ev, vt, opts):
    """Backtracking on J(v + gamma v~) <= J(v) + c1 gamma h^3 <g, v~> (reading C-9)."""
    slope = prob.h3 * dot(ev.g, vt)
    gamma = 1.0
    for halvings in range(opts.max_halvings + 1):
        trial = evaluate_objective(prob, ev.v + gamma * vt)
        if trial.J <= ev.J + opts.c1 * gamma * slope:
            return gamma, trial, halvings, True
        gamma *= 0.5
    return 0.0, None, opts.max_halvings, False


def gauss_newton(prob, v0=None, opts=None, gnorm0=None, stats=None):
    """Algorithm 1 (outer iterations) with Algorithm 2 for each Newton step."""
    opts = opts or Options()
    stats = stats or Stats()
    v = np.zeros((3,) + prob.shape) if v0 is None else np.asarray(v0, dtype=np.float64)
    ev = evaluate(prob, v)
    stats.pde_solves += 2
    if gnorm0 is None:
        if np.any(v != 0.0):
            gnorm0 = float(np.max(np.abs(evaluate(prob, np.zeros_like(v)).g)))
            stats.pde_solves += 2
        else:
            gnorm0 = float(np.max(np.abs(ev.g)))
    if stats.newton_iters == 0 and stats.J0 == 0.0:
        stats.J0 = ev.J
    mis0 = distance(prob, prob.m0)
    k = 0
    while k < opts.max_newton:
        gnorm = float(np.max(np.abs(ev.g)))
        if not opts.fixed_iters and (gnorm <= opts.eps_opt * gnorm0 or gnorm <= opts.gabs_tol):
            break
        ratio = gnorm / gnorm0
        eta = min(0.5, np.sqrt(ratio) if opts.forcing == "superlinear" else ratio)
        tol = eta * np.sqrt(dot(ev.g, ev.g))
        if opts.precond == "two_level":
            gm_c = coarse_gradient(ev.m[prob.nt])    # H0 at the current m(1)

            def apply_Minv(r):
                z, inner = two_level_inverse(r, None, prob.beta_v, prob.gamma, 0.1 * eta,
                                             opts.max_inner, gm_c=gm_c)
                stats.inner_iters += inner
                return z
        else:
            def apply_Minv(r):
                return apply_reg_inverse(r, prob.beta_v, prob.gamma)
        vt, its, mv, st = pcg(lambda s: hessian_matvec(prob, ev, s, opts.full_newton),
                              apply_Minv, ev.g, tol, opts.max_pcg, opts.fixed_iters)
        stats.pcg_iters += its
        stats.matvecs += mv
        stats.pde_solves += 2 * mv
        gamma, trial, halvings, ok = armijo(prob, ev, vt, opts)
        stats.linesearch_halvings += halvings
        stats.pde_solves += halvings + 1
        if not ok:
            stats.status = ELINESEARCH
            break
        ev = complete_gradient(prob, trial)
        stats.pde_solves += 1
        k += 1
        stats.newton_iters += 1
        stats.history.append((k, ev.J, float(np.max(np.abs(ev.g))) / gnorm0, its, gamma))
    stats.J = ev.J
    stats.mismatch_rel = float(ev.mismatch / mis0) if mis0 > 0 else 0.0
    stats.grad_rel = float(np.max(np.abs(ev.g)) / gnorm0)
    if stats.status == OK and not opts.fixed_iters and stats.grad_rel > opts.eps_opt \
            and float(np.max(np.abs(ev.g))) > opts.gabs_tol:
        stats.status = ENOTCONV
    return ev.v, stats, ev


def continuation(prob, betas, opts=None, v0=None):
    """Parameter continuation in beta_v (Sec. 2.6), warm-started level to level."""
    opts = opts or Options()
    stats = Stats()
    v = v0
    gnorm0 = None
    ev = None
    for beta in betas:
        prob.beta_v = beta
        if gnorm0 is None:
            # g(v = 0) has no regularisation part, so one value serves every level
            gnorm0 = float(np.max(np.abs(evaluate(prob, np.zeros((3,) + prob.shape)).g)))
            stats.pde_solves += 2
        stats.status = OK
        v, stats, ev = gauss_newton(prob, v, opts, gnorm0=gnorm0, stats=stats)
    return v, stats, ev


def beta_search(solve, detf_bounds, eps_d=0.1, beta0=1.0, beta_min=1e-8, rtol=0.1,
                max_bisect=10):
    """Regularisation-parameter search with det-F bounds (Sec. 2.6, "Parameter
    Selection"): eps_d < det grad y < 1/eps_d must hold (eq. ddgradbound).

    Starting at beta0 the parameter drops by decades until the bound fails;
    then a bisection runs between the last admissible value and the failing
    one.  Every trial warm-starts from the previous trial's velocity.  Reading
    C-17: the bisection takes the arithmetic midpoint and stops once the
    bracket is narrower than rtol times its admissible end, or after
    max_bisect steps; the result is the smallest admissible value found.

    solve(beta, v0) -> v (v0 None: zero initial guess); detf_bounds(v) ->
    (min det F1, max det F1).  Returns (beta*, v*, trials) with trials a list
    of (beta, admissible, min det, max det); beta* is None when beta0 itself
    violates the bound.
    """
    trials = []

    def trial(beta, v0):
        v = solve(beta, v0)
        mn, mx = detf_bounds(v)
        ok = eps_d < mn and mx < 1.0 / eps_d
        trials.append((beta, ok, mn, mx))
        return v, ok

    beta, v = beta0, None
    ok_beta, ok_v = None, None
    while True:
        v, ok = trial(beta, v)
        if not ok:
            break
        ok_beta, ok_v = beta, v
        if beta / 10.0 < beta_min * (1.0 - 1e-9):
            return ok_beta, ok_v, trials
        beta /= 10.0
    if ok_beta is None:
        return None, None, trials
    lo, hi = beta, ok_beta
    for _ in range(max_bisect):
        if hi - lo <= rtol * hi:
            break
        mid = 0.5 * (lo + hi)
        v, ok = trial(mid, v)
        if ok:
            hi, ok_v = mid, v
        else:
            lo = mid
    return hi, ok_v, trials
