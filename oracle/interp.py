"""Periodic tricubic Lagrange interpolation (Sec. 2.5.4 Interpolation).

The paper evaluates u(x) = sum_k c_k prod_i phi_{k_i}(x_i) with p + 1 basis
polynomials per axis; for Lagrange interpolation the coefficients are the grid
values and the phi are Lagrange polynomials.  CLAIRE uses cubic (p = 3).

Here a query coordinate q (in grid units, i.e. x / h) is split into the cell
index i = floor(q) and the offset t = q - i in [0, 1); the four nodes are
i-1, i, i+1, i+2, wrapped periodically; the 1D weights are the Lagrange
polynomials on the nodes {-1, 0, 1, 2} evaluated at t, written as the plain
product formula; the 3D value is the tensor product over the 64 taps.

Reading C-11: at an integer coordinate either neighbouring cell gives the same
value (the cubic is continuous across cells), so floor() is used as is.

set_threads(n) lets interp_many evaluate independent chunks of query points
on n threads (NumPy releases the interpreter lock inside take and the
element-wise products).  Every point is still computed by the same operations
in the same order, so the values are bitwise those of the serial loop; only
wall time changes.  Used to time the oracle on all host cores.
"""

from concurrent.futures import ThreadPoolExecutor

import numpy as np

_THREADS = 1


def set_threads(n):
    """Number of threads interp_many spreads its point chunks over (>= 1)."""
    global _THREADS
    _THREADS = max(1, int(n))


def get_threads():
    return _THREADS


NODES = (-1, 0, 1, 2)


def lagrange_weights(t):
    """phi_k(t) = prod_{j != k} (t - j) / (k - j) for k in NODES."""
    t = np.asarray(t, dtype=np.float64)
    weights = []
    for k in NODES:
        w = np.ones_like(t)
        for j in NODES:
            if j != k:
                w = w * (t - j) / (k - j)
        weights.append(w)
    return weights


def _axis_taps(q, n):
    base = np.floor(q)
    t = q - base
    base = base.astype(np.int64)
    idx = [np.mod(base + k, n) for k in NODES]
    return idx, lagrange_weights(t)


def interp_many(fields, q, chunk=1 << 21):
    """Interpolate several scalar fields on the same periodic grid at points q.

    fields : sequence of arrays of shape (n1, n2, n3)
    q      : array (3, ...) of query coordinates in grid units
    returns a list of arrays of shape q.shape[1:]
    """
    fields = [np.asarray(f, dtype=np.float64) for f in fields]
    shape = fields[0].shape
    n1, n2, n3 = shape
    pts_shape = q.shape[1:]
    qf = q.reshape(3, -1)
    m = qf.shape[1]
    flats = [f.ravel() for f in fields]
    outs = [np.empty(m, dtype=np.float64) for _ in fields]

    def one_chunk(s):
        e = min(m, s + chunk)
        i1, w1 = _axis_taps(qf[0, s:e], n1)
        i2, w2 = _axis_taps(qf[1, s:e], n2)
        i3, w3 = _axis_taps(qf[2, s:e], n3)
        acc = [np.zeros(e - s) for _ in fields]
        for a in range(4):
            for b in range(4):
                row = (i1[a] * n2 + i2[b]) * n3
                wab = w1[a] * w2[b]
                for c in range(4):
                    flat = row + i3[c]
                    w = wab * w3[c]
                    for f, fl in enumerate(flats):
                        acc[f] += w * np.take(fl, flat)
        for f in range(len(fields)):
            outs[f][s:e] = acc[f]

    if _THREADS > 1 and m > 1 << 16:
        chunk = min(chunk, max(1 << 14, -(-m // (8 * _THREADS))))
        with ThreadPoolExecutor(_THREADS) as ex:
            list(ex.map(one_chunk, range(0, m, chunk)))
    else:
        for s in range(0, m, chunk):
            one_chunk(s)
    return [o.reshape(pts_shape) for o in outs]


def interp(u, q):
    """Interpolate one scalar field u (n1, n2, n3) at coordinates q (3, ...)."""
    return interp_many([u], q)[0]
