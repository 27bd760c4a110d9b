"""Parity at the benchmark's full size (256^3 ellipsoid phantom pair, seed 2,
the launch configuration `bench.py` times), on sampled outputs the oracle
computes point by point, and properties that hold at any size.

* RK2 departure points (forward and backward) at 4096 sampled nodes: the
  oracle evaluates v and v(y~) at exactly those nodes (relative 1e-5 of the
  displacement scale).
* SL gather at 4096 sampled nodes, at the GPU's departure points (1e-5).
* FD8 gradient of m0 at the sampled nodes (1e-5 of the gradient scale).
* J and g: central differences of J against <g, w> (5e-2, optimize-then-
  discretize), and H positive along random directions.
* The two-level continuation solve of the benchmark converges on every level,
  decreases J, and keeps det F1 positive.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import interp as OI
from paper_2401_17493_b300 import synth

N = 256
SHAPE = (N, N, N)


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


@pytest.fixture(scope="module")
def workload():
    m0, m1, _ = synth.ellipsoid_pair(SHAPE, seed=2)
    v = synth.bandlimited_velocity(SHAPE, 8, 4.0, 3).astype(np.float32)
    rng = np.random.default_rng(7)
    idx = rng.integers(0, N, size=(3, 4096))
    return m0, m1, v, idx


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _at(field, idx):
    return field[..., idx[0], idx[1], idx[2]]


def test_trace_at_sampled_nodes(claire, workload):
    m0, m1, v, idx = workload
    with claire.Context(SHAPE, nt=4) as ctx:
        df, db = ctx.trace(dev(v))
        df, db = df.cpu().numpy(), db.cpu().numpy()
    h = 2 * np.pi / N
    ht = 0.25
    x = idx.astype(np.float64)
    vv = v.astype(np.float64)
    for sgn, d in ((+1, df), (-1, db)):
        w = sgn * vv
        w_x = _at(w, idx)
        y_t = x - ht * w_x / h
        w_yt = np.stack(OI.interp_many([w[0], w[1], w[2]], y_t))
        y = x - 0.5 * ht * (w_x + w_yt) / h
        err = np.abs(_at(d, idx) - (y - x))
        assert err.max() <= 1e-5 * np.abs(y - x).max() + 1e-6


def test_sl_gather_at_sampled_nodes(claire, workload):
    m0, m1, v, idx = workload
    with claire.Context(SHAPE, nt=4) as ctx:
        df, _ = ctx.trace(dev(v))
        out = ctx.interp(dev(m0), df).cpu().numpy()
        d = df.cpu().numpy()
    q = idx.astype(np.float64) + _at(d, idx).astype(np.float64)
    ref = OI.interp(m0.astype(np.float64), q)
    assert np.abs(_at(out, idx) - ref).max() <= 1e-5 * np.abs(m0).max()


def test_fd8_gradient_at_sampled_nodes(claire, workload):
    m0, _, _, idx = workload
    with claire.Context(SHAPE, nt=4) as ctx:
        g = ctx.grad8(dev(m0)).cpu().numpy()
    h = 2 * np.pi / N
    c = np.array([672.0, -168.0, 32.0, -3.0]) / (840.0 * h)
    u = m0.astype(np.float64)
    for a in range(3):
        ref = np.zeros(idx.shape[1])
        for k in range(1, 5):
            ip, im = idx.copy(), idx.copy()
            ip[a] = (ip[a] + k) % N
            im[a] = (im[a] - k) % N
            ref += c[k - 1] * (_at(u, ip) - _at(u, im))
        assert np.abs(g[a][idx[0], idx[1], idx[2]] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_gradient_and_hessian_properties_at_full_size(claire, workload):
    m0, m1, v, _ = workload
    v = 0.3 * v
    w = synth.bandlimited_velocity(SHAPE, 6, 1.0, 11).astype(np.float32)
    eps = 1e-2
    with claire.Context(SHAPE, nt=4, beta_v=1e-3) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        Jp, _ = ctx.objective_gradient(dev(v + eps * w), want_gradient=False)
        Jm, _ = ctx.objective_gradient(dev(v - eps * w), want_gradient=False)
        J, g = ctx.objective_gradient(dev(v))
        Hw = ctx.hessian_matvec(dev(w))
        h3 = (2 * np.pi / N) ** 3
        gw = h3 * float(torch.sum(g.double() * dev(w).double()))
        wHw = float(torch.sum(Hw.double() * dev(w).double()))
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - gw) <= 5e-2 * abs(fd)
    assert wHw > 0.0


def test_benchmark_solve_converges_and_stays_diffeomorphic(claire, workload):
    m0, m1, _, _ = workload
    betas = [1e-1, 1e-2, 1e-3, 1e-4]
    with claire.Context(SHAPE, nt=4, beta_v=betas[0], precond=1, max_inner=10,
                        max_pcg=200) as ctx:
        ctx.set_images(dev(m0), dev(m1))
        v, st = ctx.solve_continuation(betas)
        (mn, mx, mean), _ = ctx.det_deformation_gradient(v)
    assert st.status == claire.OK and st.grad_rel <= 5e-2
    assert st.J < st.J0 and 0.0 < st.mismatch_rel < 0.5
    assert mn > 0.0 and abs(mean - 1.0) < 0.05
