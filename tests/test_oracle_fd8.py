"""Pins for oracle.fd8 (Sec. 2.5.3): the printed stencil, closed forms, adjointness."""

import os

import numpy as np

from oracle.fd8 import d8, grad8, div8

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd8_stencil.txt")


def _load_stencil():
    rows = [l.split("#")[0].split() for l in open(GOLDEN)]
    rows = [r for r in rows if r]
    den = float(rows[0][1])
    return den, {int(k): float(c) for k, c in rows[1:]}


def test_impulse_response_reproduces_printed_coefficients():
    den, coef = _load_stencil()
    n, h = 16, 0.37
    for axis in range(3):
        u = np.zeros((n, n, n))
        u[5, 6, 7] = 1.0
        d = d8(u, axis, h) * den * h
        idx = [5, 6, 7]
        for k, c in coef.items():
            # the stencil at node l uses u_{l+k}; the impulse sits at l + k = idx
            at = list(idx)
            at[axis] = (idx[axis] - k) % n
            assert abs(d[tuple(at)] - c) < 1e-9, (axis, k)
        assert np.count_nonzero(np.abs(d) > 1e-12) == 8


def test_sine_mode_closed_form_and_orientation():
    n = 32
    h = 2 * np.pi / n
    x = np.arange(n) * h
    for kap in (1, 3, 7):
        kt = (2.0 / h) * (4 / 5 * np.sin(kap * h) - 1 / 5 * np.sin(2 * kap * h)
                          + 4 / 105 * np.sin(3 * kap * h) - 1 / 280 * np.sin(4 * kap * h))
        for axis in range(3):
            shp = [1, 1, 1]
            shp[axis] = n
            u = np.broadcast_to(np.sin(kap * x).reshape(shp), (n, n, n)).copy()
            g = grad8(u)
            expect = np.broadcast_to((kt * np.cos(kap * x)).reshape(shp), (n, n, n))
            assert np.allclose(g[axis], expect, atol=1e-12)
            for other in range(3):
                if other != axis:
                    assert np.allclose(g[other], 0.0, atol=1e-12)
        assert abs(kt - kap) / kap < (kap * h) ** 8          # 8th-order accurate


def test_exact_for_degree_8_polynomials_in_the_interior():
    n = 24
    h = 0.5
    l = np.arange(n, dtype=float)
    x = l * h
    p = np.poly1d(np.random.default_rng(0).standard_normal(9))
    u = np.broadcast_to(p(x)[None, None, :], (4, 4, n)).copy()
    d = d8(u, 2, h)[0, 0, 4:n - 4]
    ref = p.deriv()(x[4:n - 4])
    assert np.allclose(d, ref, rtol=1e-9, atol=1e-7 * np.max(np.abs(ref)))


def test_gradient_and_divergence_are_negative_adjoints():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((12, 10, 14))
    w = rng.standard_normal((3, 12, 10, 14))
    lhs = np.sum(grad8(u) * w)
    rhs = -np.sum(u * div8(w))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_threaded_slabs_give_bitwise_the_serial_values():
    from oracle import fd8 as F
    rng = np.random.default_rng(3)
    u = rng.standard_normal((72, 64, 80))
    w = rng.standard_normal((3, 72, 64, 80))
    serial_g, serial_d = F.grad8(u), F.div8(w)
    try:
        F.set_threads(5)
        threaded_g, threaded_d = F.grad8(u), F.div8(w)
    finally:
        F.set_threads(1)
    assert np.array_equal(serial_g, threaded_g) and np.array_equal(serial_d, threaded_d)
