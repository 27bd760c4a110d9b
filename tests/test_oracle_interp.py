"""Pins for oracle.interp (Sec. 2.5.4): brute force, library route, closed forms."""

import numpy as np
import pytest

from oracle import interp as OI
from oracle.interp import interp, interp_many, lagrange_weights


def _poly_route(u, q):
    """Independent route: sequential 1D cubic fits (numpy.polyfit) through 4 nodes per axis."""
    n = u.shape
    out = np.empty(q.shape[1])
    for p in range(q.shape[1]):
        base = [int(np.floor(q[a, p])) for a in range(3)]
        nodes = np.arange(-1, 3)
        # x3 first: 16 rows -> 4x4 values at the query's x3
        vals12 = np.empty((4, 4))
        for a in range(4):
            for b in range(4):
                row = [u[(base[0] + nodes[a]) % n[0], (base[1] + nodes[b]) % n[1],
                         (base[2] + c) % n[2]] for c in nodes]
                coef = np.polyfit(base[2] + nodes.astype(float), row, 3)
                vals12[a, b] = np.polyval(coef, q[2, p])
        vals1 = np.empty(4)
        for a in range(4):
            coef = np.polyfit(base[1] + nodes.astype(float), vals12[a], 3)
            vals1[a] = np.polyval(coef, q[1, p])
        coef = np.polyfit(base[0] + nodes.astype(float), vals1, 3)
        out[p] = np.polyval(coef, q[0, p])
    return out


def test_matches_sequential_polyfit_route_on_tiny_grid():
    rng = np.random.default_rng(0)
    u = rng.standard_normal((5, 6, 7))
    q = rng.uniform(-9.0, 15.0, size=(3, 40))          # includes wrap-around
    ref = _poly_route(u, q)
    assert np.allclose(interp(u, q), ref, rtol=0, atol=1e-10)


def test_grid_points_are_reproduced_exactly():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((8, 9, 10))
    q = np.stack(np.meshgrid(np.arange(8.0), np.arange(9.0), np.arange(10.0), indexing="ij"))
    assert np.array_equal(interp(u, q), u)


def test_tensor_cubic_polynomials_are_exact_away_from_the_wrap():
    n = (16, 16, 16)
    x = np.meshgrid(*[np.arange(m, dtype=float) for m in n], indexing="ij")
    P = lambda a, b, c: (0.3 * a ** 3 - a * b + 0.1 * b ** 3 * c - 2 * c ** 2 + 0.05 * a * b * c
                         + 0.01 * a ** 3 * b ** 3 * c ** 3)
    u = P(*x)
    rng = np.random.default_rng(2)
    q = rng.uniform(1.0, 12.999, size=(3, 200))        # nodes floor-1 .. floor+2 stay in [0, 15]
    assert np.allclose(interp(u, q), P(q[0], q[1], q[2]), rtol=1e-12, atol=1e-9)


def test_weights_partition_of_unity_and_mirror_symmetry():
    t = np.linspace(0.0, 1.0, 101)
    w = lagrange_weights(t)
    assert np.allclose(sum(w), 1.0, atol=1e-15)
    wm = lagrange_weights(1.0 - t)
    for k in range(4):                                  # w_{1-k}(1-t) = w_k(t), nodes -1..2
        assert np.allclose(wm[3 - k], w[k], atol=1e-15)
    # closed forms of the four cubic Lagrange polynomials on {-1, 0, 1, 2}
    assert np.allclose(w[0], -t * (t - 1) * (t - 2) / 6)
    assert np.allclose(w[1], (t + 1) * (t - 1) * (t - 2) / 2)
    assert np.allclose(w[2], -(t + 1) * t * (t - 2) / 2)
    assert np.allclose(w[3], (t + 1) * t * (t - 1) / 6)


def test_many_fields_match_single_field_calls():
    rng = np.random.default_rng(3)
    fs = [rng.standard_normal((6, 6, 8)) for _ in range(3)]
    q = rng.uniform(0, 8, size=(3, 4, 5))
    many = interp_many(fs, q)
    for f, m in zip(fs, many):
        assert np.array_equal(interp(f, q), m)


def test_threaded_chunks_give_bitwise_the_serial_values():
    rng = np.random.default_rng(5)
    shape = (40, 36, 48)
    u = rng.standard_normal(shape)
    q = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij"))
    q = q + rng.uniform(-5.0, 5.0, size=(3,) + shape)
    serial = OI.interp_many([u, -u], q)
    try:
        OI.set_threads(4)
        threaded = OI.interp_many([u, -u], q)
    finally:
        OI.set_threads(1)
    assert all(np.array_equal(a, b) for a, b in zip(serial, threaded))
