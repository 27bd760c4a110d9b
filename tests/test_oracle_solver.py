"""Pins for oracle.solver: Algorithm 2 is textbook PCG (P-11, checked against
scipy.sparse.linalg.cg), negative-curvature exit (Sec. 2.5.5), and Algorithm 1
decreasing J and the relative gradient on a small registration."""

import numpy as np
import scipy.sparse.linalg as spla

from oracle import solver as S
from oracle import reduced as R
from paper_2401_17493_b300 import synth


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, 4))
    return np.diag(rng.uniform(1.0, 50.0, n)) + U @ U.T


def test_pcg_iterates_match_scipy_cg():
    n = 60
    A = _spd(n, 0)
    d = 1.0 / np.diag(A)
    g = np.random.default_rng(1).standard_normal(n)
    for k in (1, 3, 7, 12):
        ours, its, mv, st = S.pcg(lambda s: A @ s, lambda r: d * r, g, 0.0, k, fixed=True)
        iters = []
        spla.cg(A, -g, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=k,
                M=spla.LinearOperator((n, n), matvec=lambda r: d * r),
                callback=lambda xk: iters.append(xk.copy()))
        assert its == k and mv == k and st == S.OK
        assert np.allclose(ours, iters[-1], rtol=1e-10, atol=1e-12)


def test_pcg_stops_on_the_residual_tolerance():
    A = _spd(40, 2)
    g = np.ones(40)
    x, its, mv, st = S.pcg(lambda s: A @ s, lambda r: r, g, 1e-6 * np.linalg.norm(g), 200)
    assert its < 40
    assert np.linalg.norm(A @ x + g) < 1e-6 * np.linalg.norm(g)


def test_pcg_negative_curvature_returns_previous_iterate():
    g = np.array([1.0, 1.0, 1.0])
    # <s, A s> = 0 on the first direction s = -g: no previous iterate, fall back to s
    A = np.diag([3.0, 2.0, -5.0])
    x, its, mv, st = S.pcg(lambda s: A @ s, lambda r: r, g, 0.0, 10, fixed=True)
    assert st == S.ENEGCURV and its == 0 and np.allclose(x, -g)
    # first step fine (kappa = 3/4), second direction has <s, A s> < 0: keep x_1
    A2 = np.diag([3.0, 2.0, -1.0])
    x2, its2, mv2, st2 = S.pcg(lambda s: A2 @ s, lambda r: r, g, 0.0, 10, fixed=True)
    assert st2 == S.ENEGCURV and its2 == 1 and mv2 == 2
    assert np.allclose(x2, -0.75 * g)


def test_gauss_newton_decreases_objective_and_gradient():
    m0, m1, v = synth.blob_pair((16, 16, 16), seed=3, kmax=2, max_disp_voxels=1.0)
    p = R.Problem(m0, m1, nt=4, beta_v=1e-2)
    vs, st, ev = S.gauss_newton(p, None, S.Options(max_newton=3, max_pcg=5, fixed_iters=True))
    assert st.newton_iters == 3 and st.matvecs == 15
    assert st.J < st.J0
    assert st.grad_rel < 0.5
    Js = [h[1] for h in st.history]
    assert all(b <= a for a, b in zip(Js, Js[1:]))


def test_gauss_newton_reaches_the_relative_gradient_tolerance():
    m0, m1, v = synth.blob_pair((16, 16, 16), seed=4, kmax=2, max_disp_voxels=1.0)
    p = R.Problem(m0, m1, nt=4, beta_v=1e-1)
    vs, st, ev = S.gauss_newton(p, None, S.Options(eps_opt=5e-2))
    assert st.status == S.OK
    assert st.grad_rel <= 5e-2
    # each Newton iteration costs 2 PDE solves per matvec + line-search state solves + adjoint
    assert st.pde_solves >= 2 + 2 * st.matvecs + 2 * st.newton_iters


def test_beta_search_sequence_on_a_known_threshold():
    """Brute force of the search rule with a stand-in solver: admissible iff
    beta >= 3.7e-3 (decades 1 .. 1e-2 pass, 1e-3 fails, then bisection)."""
    calls = []

    def solve(beta, v0):
        calls.append((beta, v0))
        return beta                                  # the 'velocity' carries beta

    def bounds(v):
        return (0.5, 1.5) if v >= 3.7e-3 else (0.05, 3.0)

    beta, v, trials = S.beta_search(solve, bounds, eps_d=0.1, rtol=0.1)
    seq = [t[0] for t in trials]
    expect = [1.0, 0.1, 0.01, 1e-3]
    lo, hi = 1e-3, 1e-2
    while hi - lo > 0.1 * hi:
        mid = 0.5 * (lo + hi)
        expect.append(mid)
        if mid >= 3.7e-3:
            hi = mid
        else:
            lo = mid
    assert np.allclose(seq, expect)
    assert beta == hi and v == hi and 3.7e-3 <= beta < 3.7e-3 / 0.9
    # warm starts: each trial starts from the previous trial's velocity
    assert calls[0][1] is None and all(calls[i][1] == calls[i - 1][0] for i in range(1, len(calls)))


def test_beta_search_edge_cases():
    solve = lambda b, v0: b
    beta, _, trials = S.beta_search(solve, lambda v: (0.01, 2.0), eps_d=0.1)
    assert beta is None and len(trials) == 1                # beta0 already violates
    beta, _, trials = S.beta_search(solve, lambda v: (0.9, 1.1), eps_d=0.1, beta_min=1e-3)
    assert abs(beta - 1e-3) < 1e-15 and len(trials) == 4    # never violated down to beta_min
    beta, _, trials = S.beta_search(solve, lambda v: (0.5, 20.0) if v < 0.05 else (0.5, 2.0),
                                    eps_d=0.1)
    assert trials[2][1] is False and 0.05 <= beta <= 0.1      # upper bound 1/eps_d checked


def test_beta_search_on_a_registration_keeps_det_f_in_bounds():
    from oracle import defgrad as D
    m0, m1, v = synth.blob_pair((16, 16, 16), seed=5, kmax=2, max_disp_voxels=2.5)
    p = R.Problem(m0, m1, nt=4, beta_v=1.0)
    gnorm0 = float(np.max(np.abs(R.gradient_at_zero(p))))

    def solve(beta, v0):
        p.beta_v = beta
        vs, _, _ = S.gauss_newton(p, v0, S.Options(eps_opt=5e-2), gnorm0=gnorm0)
        return vs

    def bounds(v):
        _, (mn, mx, _) = D.det_deformation_gradient(v, 4)
        return mn, mx

    beta, vb, trials = S.beta_search(solve, bounds, eps_d=0.5, rtol=0.2, max_bisect=4)
    assert beta is not None and any(not t[1] for t in trials)
    mn, mx = bounds(vb)
    assert 0.5 < mn and mx < 2.0
