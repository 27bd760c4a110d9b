"""8th-order central finite differences (Sec. 2.5.3 Differentiation).

d_i u(x_l) ~= (u^-_i + u^+_i) / (840 h_i) with
  u^-_i = 3 u_{l-4} - 32 u_{l-3} + 168 u_{l-2} - 672 u_{l-1}
  u^+_i = 672 u_{l+1} - 168 u_{l+2} + 32 u_{l+3} - 3 u_{l+4}
on the periodic grid, with +x along +index (reading C-1).  The gradient of a
scalar and the divergence of a vector field both use this first derivative.

set_threads(n) lets d8 work on n slabs at once, cut along an axis other than
the derivative's: each slab sees the same periodic shifts along the derivative
axis, so the values are bitwise those of the whole-array expression; only wall
time changes.  Used to time the oracle on all host cores.
"""

from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .grid import spacing

_THREADS = 1


def set_threads(n):
    """Number of slabs d8 evaluates concurrently (>= 1)."""
    global _THREADS
    _THREADS = max(1, int(n))


def _shift(u, k, axis):
    """u_{l+k} along axis (periodic)."""
    return np.roll(u, -k, axis=axis)


def _d8(u, axis, h):
    u_minus = (3.0 * _shift(u, -4, axis) - 32.0 * _shift(u, -3, axis)
               + 168.0 * _shift(u, -2, axis) - 672.0 * _shift(u, -1, axis))
    u_plus = (672.0 * _shift(u, 1, axis) - 168.0 * _shift(u, 2, axis)
              + 32.0 * _shift(u, 3, axis) - 3.0 * _shift(u, 4, axis))
    return (u_minus + u_plus) / (840.0 * h)


def d8(u, axis, h):
    """First derivative along one axis, written as the paper's u^- + u^+."""
    if _THREADS == 1 or u.size < 1 << 18:
        return _d8(u, axis, h)
    cut = 1 if axis == 0 else 0                   # slabs along an axis != the derivative's
    edges = np.linspace(0, u.shape[cut], min(_THREADS, u.shape[cut]) + 1).astype(int)
    out = np.empty_like(u, dtype=np.float64)

    def slab(i):
        sl = [slice(None)] * u.ndim
        sl[cut] = slice(edges[i], edges[i + 1])
        out[tuple(sl)] = _d8(u[tuple(sl)], axis, h)

    with ThreadPoolExecutor(_THREADS) as ex:
        list(ex.map(slab, range(len(edges) - 1)))
    return out


def grad8(u):
    """FD8 gradient of a scalar field (n1, n2, n3) -> (3, n1, n2, n3)."""
    u = np.asarray(u, dtype=np.float64)
    h = spacing(u.shape)
    return np.stack([d8(u, a, h[a]) for a in range(3)])


def div8(w):
    """FD8 divergence of a vector field (3, n1, n2, n3) -> (n1, n2, n3)."""
    w = np.asarray(w, dtype=np.float64)
    h = spacing(w.shape[1:])
    return d8(w[0], 0, h[0]) + d8(w[1], 1, h[1]) + d8(w[2], 2, h[2])
