"""Pins for oracle.precond, the two-level zero-velocity preconditioner (Sec. 2.5.6).

* H0's closed form equals the transport-based Gauss-Newton Hessian matvec of
  oracle.reduced at v = 0 (the special case the paper works out): two
  independent code paths.
* With a constant image grad m = 0, the nested system is the identity and the
  two-level preconditioner reduces to the spectral one, (alpha L)^-1.
* Purely high-frequency residuals (no mode with every |k_i| < n_i / 4) skip the
  coarse solve: M^-1 r = (alpha L)^-1 r for any image.
* The nested CG reaches the solution of the coarse system assembled as a dense
  matrix on a tiny grid (brute force).
* With an exact nested solve, R^-1/2 M^-1 R^-1/2 is symmetric positive definite
  (a transposed or one-sided R^-1/2 breaks it).
"""

import numpy as np

from oracle import precond as P
from oracle import reduced as R
from oracle import spectral as Sp
from oracle import solver as S
from paper_2401_17493_b300 import synth


def _images(n=16, seed=5):
    m0, m1, _ = synth.blob_pair((n, n, n), seed=seed, kmax=2, max_disp_voxels=1.0)
    return m0.astype(np.float64), m1.astype(np.float64)


def _field(shape, seed, kmax=5):
    return synth.bandlimited_velocity(shape, kmax, 1.0, seed).astype(np.float64)


def test_h0_equals_gauss_newton_hessian_at_zero_velocity():
    m0, m1 = _images()
    p = R.Problem(m0, m1, nt=4, beta_v=3e-2)
    ev = R.evaluate(p, np.zeros((3,) + p.shape))
    vt = _field(p.shape, 11)
    H = R.hessian_matvec(p, ev, vt)
    H0 = P.h0_apply(vt, m0, p.beta_v, p.gamma)
    assert np.max(np.abs(H - H0)) <= 1e-10 * np.max(np.abs(H))


def test_constant_image_reduces_to_the_spectral_preconditioner():
    shape = (16, 16, 16)
    r = _field(shape, 12, kmax=7)
    m = np.full(shape, 0.4)
    z, its = P.two_level_inverse(r, m, 1e-2, 1.0, 1e-12)
    ref = Sp.apply_reg_inverse(r, 1e-2, 1.0)
    assert its <= 1
    assert np.max(np.abs(z - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_high_frequency_residual_skips_the_coarse_solve():
    m0, _ = _images()
    shape = m0.shape
    r = _field(shape, 13, kmax=8)
    r = r - P.prolong3(P.restrict3(r, P.coarse_shape(shape)), shape)   # F_H r
    z, its = P.two_level_inverse(r, m0, 1e-3, 1.0, 1e-12)
    ref = Sp.apply_reg_inverse(r, 1e-3, 1.0)
    assert np.max(np.abs(z - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_nested_cg_matches_a_dense_solve_of_the_coarse_system():
    m0, _ = _images()
    gm_c = P.coarse_gradient(m0)
    cs = gm_c.shape[1:]
    n = 3 * int(np.prod(cs))
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = P.coarse_operator(e.reshape((3,) + cs), gm_c, 1e-3, 1.0).ravel()
    assert np.allclose(A, A.T, atol=1e-10 * np.abs(A).max())
    b = _field(cs, 14, kmax=3)
    x_ref = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    x, its = P.cg(lambda u: P.coarse_operator(u, gm_c, 1e-3, 1.0), b, 1e-13, 2000)
    assert np.max(np.abs(x - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))


def test_two_level_inverse_is_symmetric_positive_definite():
    m0, _ = _images()
    a = _field(m0.shape, 15, kmax=6)
    b = _field(m0.shape, 16, kmax=6)
    Ma, _ = P.two_level_inverse(a, m0, 1e-3, 1.0, 1e-13, 500)
    Mb, _ = P.two_level_inverse(b, m0, 1e-3, 1.0, 1e-13, 500)
    lhs, rhs = float(np.sum(a * Mb)), float(np.sum(Ma * b))
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), abs(rhs))
    assert float(np.sum(a * Ma)) > 0.0 and float(np.sum(b * Mb)) > 0.0


def test_gauss_newton_with_the_two_level_preconditioner_converges():
    m0, m1 = _images(seed=4)
    p = R.Problem(m0, m1, nt=4, beta_v=1e-3)
    _, st_s, _ = S.gauss_newton(p, None, S.Options(eps_opt=5e-2))
    _, st_t, _ = S.gauss_newton(p, None, S.Options(eps_opt=5e-2, precond="two_level"))
    assert st_t.status == S.OK and st_t.grad_rel <= 5e-2
    assert st_t.inner_iters > 0
    # the coarse zero-velocity Hessian captures the data term's low modes
    assert st_t.matvecs < st_s.matvecs
