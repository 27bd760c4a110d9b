"""Pins of the oracle's Armijo line search and beta_v continuation (Sec. 2.5.5,
Algorithm 1; Sec. 2.6; readings C-9 and C-10).

armijo: on a stand-in objective that is an exact quadratic along the search
line, phi(gamma) = J + gamma h^3 s + gamma^2 q / 2 with s = <g, v~>, the rule
"accept the first gamma in 1, 1/2, 1/4, ... with phi(gamma) <= J + c1 gamma
h^3 s" has a closed-form answer.  Each case below is built so that one
plausible mistake changes the accepted step or the halving count: a flipped
slope sign, a slope without the h^3 quadrature weight, c1 = 1, no halving,
an off-by-one cap on the halvings.  The planted versions at the end are such
mistakes written into a copy of the oracle's function; each must fail a pin.

continuation: with stand-in evaluate / gauss_newton that only record their
arguments, the level loop must solve the levels in the given order, start each
level from the previous level's result, and divide by one denominator,
||g(v = 0)||_inf, computed once (reading C-10).
"""

import types

import numpy as np
import pytest

from oracle import solver as S

H3 = 40.0          # quadrature weight of the stand-in grid (>1, so a missing h^3 matters)


class _Quadratic:
    """J(v) = J0 + h^3 (<g0, v - v0> + <v - v0, a (v - v0)> / 2): an exact
    quadratic along every line, with the oracle's convention that the
    directional derivative is h^3 <g, v~>."""

    def __init__(self, v0, g0, a, J0=1.0):
        self.v0, self.g0, self.a, self.J0 = v0, g0, a, J0
        self.calls = []

    def __call__(self, prob, v):
        self.calls.append(v.copy())
        dv = v - self.v0
        J = self.J0 + H3 * (np.sum(self.g0 * dv) + 0.5 * np.sum(self.a * dv * dv))
        return types.SimpleNamespace(J=float(J), v=v)


def _case(direction_scale, curvature_scale, monkeypatch, seed=0):
    """A stand-in problem whose line phi(gamma) has slope h^3 s (s < 0) and
    curvature q = h^3 <v~, a v~> set relative to |s|."""
    rng = np.random.default_rng(seed)
    shape = (3, 2, 3, 2)
    v0 = rng.standard_normal(shape)
    g0 = rng.standard_normal(shape)
    vt = -direction_scale * g0                      # descent direction, s = -scale |g0|^2
    s = float(np.sum(g0 * vt))
    a = np.full(shape, curvature_scale * abs(s) / float(np.sum(vt * vt)))
    obj = _Quadratic(v0, g0, a)
    monkeypatch.setattr(S, "evaluate_objective", obj)
    prob = types.SimpleNamespace(h3=H3)
    ev = types.SimpleNamespace(v=v0, g=g0, J=obj.J0)
    return prob, ev, vt, obj, s


def _phi(obj, s, gamma, q):
    return obj.J0 + gamma * H3 * s + 0.5 * gamma ** 2 * q


def _pins(armijo, monkeypatch):
    """Run every closed-form case through `armijo`; returns the failed pins."""
    failed = []
    opts = S.Options()
    c1 = opts.c1

    # 1. phi(1) = phi(0): the minimiser of the line is at gamma = 1/2.  The
    #    correct rule rejects gamma = 1 (no decrease) and accepts 1/2.
    prob, ev, vt, obj, s = _case(1.0, 2.0, monkeypatch)   # curvature 2 |s|: phi(1) = phi(0)
    gamma, trial, halvings, ok = armijo(prob, ev, vt, opts)
    if not (ok and gamma == 0.5 and halvings == 1 and len(obj.calls) == 2):
        failed.append("equal-objective step")

    # 2. at gamma = 1 the decrease is half of c1 h^3 |s|: rejected; accepted at 1/2.
    #    q chosen so that phi(1) = J - c1 h^3 |s| / 2.
    prob, ev, vt, obj, s = _case(1.0, 1.0, monkeypatch, seed=1)
    q = 2.0 * H3 * abs(s) * (1.0 - 0.5 * c1)
    obj.a = obj.a * (q / (H3 * float(np.sum(obj.a * vt * vt))))
    assert abs(_phi(obj, s, 1.0, q) - (obj.J0 - 0.5 * c1 * H3 * abs(s))) < 1e-9 * H3 * abs(s)
    gamma, trial, halvings, ok = armijo(prob, ev, vt, opts)
    if not (ok and gamma == 0.5 and halvings == 1):
        failed.append("half-sufficient decrease at the full step")

    # 3. a sharply curved line (minimiser at gamma = 1/20): the first accepted
    #    step is 1/16 after exactly four halvings, trial steps 1, 1/2, 1/4, 1/8, 1/16.
    prob, ev, vt, obj, s = _case(1.0, 20.0, monkeypatch, seed=2)
    gamma, trial, halvings, ok = armijo(prob, ev, vt, opts)
    steps = [float(np.linalg.norm(c - ev.v) / np.linalg.norm(vt)) for c in obj.calls]
    if not (ok and gamma == 1.0 / 16 and halvings == 4 and
            np.allclose(steps, [1, 0.5, 0.25, 0.125, 0.0625], rtol=1e-12)):
        failed.append("four halvings")
    if ok and trial is not None and not np.allclose(trial.v, ev.v + gamma * vt):
        failed.append("accepted trial point")

    # 4. an ascent direction is never accepted: exactly max_halvings + 1 trials
    prob, ev, vt, obj, s = _case(-1.0, 1.0, monkeypatch, seed=3)
    gamma, trial, halvings, ok = armijo(prob, ev, vt, opts)
    if not (not ok and gamma == 0.0 and trial is None and halvings == opts.max_halvings and
            len(obj.calls) == opts.max_halvings + 1):
        failed.append("ascent direction")

    # 5. a full Newton step on an exact quadratic model (minimiser at gamma = 1)
    #    is accepted at once
    prob, ev, vt, obj, s = _case(1.0, 1.0, monkeypatch, seed=4)
    gamma, trial, halvings, ok = armijo(prob, ev, vt, opts)
    if not (ok and gamma == 1.0 and halvings == 0):
        failed.append("full step")
    return failed


def test_armijo_matches_the_closed_form_cases(monkeypatch):
    assert _pins(S.armijo, monkeypatch) == []


# -- planted mistakes (copies of the oracle's armijo with one change each) ---------------

def _flipped_slope(prob, ev, vt, opts):
    slope = -prob.h3 * S.dot(ev.g, vt)
    gamma = 1.0
    for halvings in range(opts.max_halvings + 1):
        trial = S.evaluate_objective(prob, ev.v + gamma * vt)
        if trial.J <= ev.J + opts.c1 * gamma * slope:
            return gamma, trial, halvings, True
        gamma *= 0.5
    return 0.0, None, opts.max_halvings, False


def _no_h3(prob, ev, vt, opts):
    slope = S.dot(ev.g, vt)
    gamma = 1.0
    for halvings in range(opts.max_halvings + 1):
        trial = S.evaluate_objective(prob, ev.v + gamma * vt)
        if trial.J <= ev.J + opts.c1 * gamma * slope:
            return gamma, trial, halvings, True
        gamma *= 0.5
    return 0.0, None, opts.max_halvings, False


def _c1_one(prob, ev, vt, opts):
    slope = prob.h3 * S.dot(ev.g, vt)
    gamma = 1.0
    for halvings in range(opts.max_halvings + 1):
        trial = S.evaluate_objective(prob, ev.v + gamma * vt)
        if trial.J <= ev.J + 1.0 * gamma * slope:
            return gamma, trial, halvings, True
        gamma *= 0.5
    return 0.0, None, opts.max_halvings, False


def _no_halving(prob, ev, vt, opts):
    slope = prob.h3 * S.dot(ev.g, vt)
    gamma = 1.0
    for halvings in range(opts.max_halvings + 1):
        trial = S.evaluate_objective(prob, ev.v + gamma * vt)
        if trial.J <= ev.J + opts.c1 * gamma * slope:
            return gamma, trial, halvings, True
    return 0.0, None, opts.max_halvings, False


def _one_halving_short(prob, ev, vt, opts):
    slope = prob.h3 * S.dot(ev.g, vt)
    gamma = 1.0
    for halvings in range(opts.max_halvings):
        trial = S.evaluate_objective(prob, ev.v + gamma * vt)
        if trial.J <= ev.J + opts.c1 * gamma * slope:
            return gamma, trial, halvings, True
        gamma *= 0.5
    return 0.0, None, opts.max_halvings, False


@pytest.mark.parametrize("planted", [_flipped_slope, _no_h3, _c1_one, _no_halving,
                                     _one_halving_short])
def test_armijo_pins_detect_planted_mistakes(monkeypatch, planted):
    assert _pins(planted, monkeypatch) != []


# -- continuation -------------------------------------------------------------------------

def _run_continuation(continuation, monkeypatch, betas, v0):
    """continuation() with stand-ins that record each level's beta_v, initial
    guess and denominator; a level's 'solve' returns its initial guess + beta."""
    levels, evaluations = [], []

    def fake_evaluate(prob, v):
        evaluations.append((prob.beta_v, v.copy()))
        g = np.full((3,) + prob.shape, 2.5)
        g[0, 0, 0, 0] = -7.0                           # ||g(0)||_inf = 7
        return types.SimpleNamespace(g=g)

    def fake_gauss_newton(prob, v, opts, gnorm0=None, stats=None):
        levels.append((prob.beta_v, None if v is None else np.array(v), gnorm0, stats.status))
        stats.newton_iters += 1
        stats.status = S.ENOTCONV                      # must not leak into the next level
        start = np.zeros((3,) + prob.shape) if v is None else np.asarray(v)
        return start + prob.beta_v, stats, types.SimpleNamespace(level=prob.beta_v)

    monkeypatch.setattr(S, "evaluate", fake_evaluate)
    monkeypatch.setattr(S, "gauss_newton", fake_gauss_newton)
    prob = types.SimpleNamespace(beta_v=None, shape=(2, 2, 2))
    v, stats, ev = continuation(prob, betas, S.Options(), v0=v0)
    return levels, evaluations, v, stats, ev


def _continuation_pins(continuation, monkeypatch):
    failed = []
    betas = [1e-1, 1e-2, 1e-3, 1e-4]
    levels, evaluations, v, stats, ev = _run_continuation(continuation, monkeypatch, betas,
                                                          None)
    if [lv[0] for lv in levels] != betas:
        failed.append("level order")
    if levels and levels[0][1] is not None:
        failed.append("first level starts from the given guess")
    for i in range(1, len(levels)):          # level i starts where level i - 1 ended
        expect = np.full((3, 2, 2, 2), sum(betas[:i]))
        if levels[i][1] is None or not np.allclose(levels[i][1], expect):
            failed.append(f"warm start of level {i}")
    # one denominator for every level: ||g(v = 0)||_inf, from one evaluation at v = 0
    if [lv[2] for lv in levels] != [7.0] * len(betas):
        failed.append("denominator")
    if len(evaluations) != 1 or np.any(evaluations[0][1] != 0.0):
        failed.append("denominator evaluated once at v = 0")
    if any(lv[3] != S.OK for lv in levels):
        failed.append("status reset per level")
    if not np.allclose(v, sum(betas)) or stats.newton_iters != len(betas) or ev.level != 1e-4:
        failed.append("result of the last level")
    # an explicit initial guess is the first level's start
    v0 = np.full((3, 2, 2, 2), 0.25)
    levels, _, v, _, _ = _run_continuation(continuation, monkeypatch, [1e-2, 1e-3], v0)
    if levels[0][1] is None or not np.allclose(levels[0][1], 0.25) or \
            not np.allclose(v, 0.25 + 1e-2 + 1e-3):
        failed.append("given initial guess")
    return failed


def test_continuation_levels_warm_start_with_one_denominator(monkeypatch):
    assert _continuation_pins(S.continuation, monkeypatch) == []


def _cold_levels(prob, betas, opts=None, v0=None):
    opts = opts or S.Options()
    stats = S.Stats()
    gnorm0 = float(np.max(np.abs(S.evaluate(prob, np.zeros((3,) + prob.shape)).g)))
    for beta in betas:
        prob.beta_v = beta
        stats.status = S.OK
        v, stats, ev = S.gauss_newton(prob, v0, opts, gnorm0=gnorm0, stats=stats)
    return v, stats, ev


def _denominator_per_level(prob, betas, opts=None, v0=None):
    opts = opts or S.Options()
    stats = S.Stats()
    v = v0
    for beta in betas:
        prob.beta_v = beta
        stats.status = S.OK
        v, stats, ev = S.gauss_newton(prob, v, opts, gnorm0=None, stats=stats)
    return v, stats, ev


def _reversed_levels(prob, betas, opts=None, v0=None):
    opts = opts or S.Options()
    betas = betas[::-1]
    stats = S.Stats()
    v, gnorm0 = v0, None
    for beta in betas:
        prob.beta_v = beta
        if gnorm0 is None:
            gnorm0 = float(np.max(np.abs(S.evaluate(prob, np.zeros((3,) + prob.shape)).g)))
        stats.status = S.OK
        v, stats, ev = S.gauss_newton(prob, v, opts, gnorm0=gnorm0, stats=stats)
    return v, stats, ev


def _status_carried(prob, betas, opts=None, v0=None):
    opts = opts or S.Options()
    stats = S.Stats()
    v, gnorm0 = v0, None
    for beta in betas:
        prob.beta_v = beta
        if gnorm0 is None:
            gnorm0 = float(np.max(np.abs(S.evaluate(prob, np.zeros((3,) + prob.shape)).g)))
        v, stats, ev = S.gauss_newton(prob, v, opts, gnorm0=gnorm0, stats=stats)
    return v, stats, ev


@pytest.mark.parametrize("planted", [_cold_levels, _denominator_per_level, _reversed_levels,
                                     _status_carried])
def test_continuation_pins_detect_planted_mistakes(monkeypatch, planted):
    assert _continuation_pins(planted, monkeypatch) != []
