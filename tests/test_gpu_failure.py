"""Failure detection without a GPU fault: the bounded tensor-core waits.

* claire_wait_selftest polls an mbarrier that nothing arrives at: every thread
  gives up after max_polls polls, the call returns ETIMEOUT, and the device
  counter read by claire_wait_status holds its 32 timeouts and then resets.
* With an arrival the same wait succeeds and nothing is counted.
* Afterwards the device is usable: a tensor-core convolution (halo-tile forward
  and tcgen05 weight gradient) matches the oracle and counts no timeout.
* Invalid budgets are rejected before any launch.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import conv3d as OC


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _bf(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64)).to(torch.bfloat16).double().numpy()


def _cl(x):
    return torch.from_numpy(np.ascontiguousarray(np.moveaxis(x, 0, -1).reshape(-1, x.shape[0]))).to(
        torch.bfloat16).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_wait_that_nothing_completes_reports_timeout(claire):
    assert claire.wait_status() == 0                 # no earlier kernel timed out
    assert claire.wait_selftest(max_polls=1000, arrive=False) == claire.ETIMEOUT
    assert claire.wait_status() == 32                # one per thread of the CTA
    assert claire.wait_status() == 0                 # the read reset the counter


def test_completed_wait_succeeds(claire):
    stream = torch.cuda.current_stream().cuda_stream
    assert claire.wait_selftest(max_polls=1000, arrive=True, stream=stream) == claire.OK
    assert claire.wait_status() == 0


def test_device_stays_usable_after_a_timeout(claire):
    assert claire.wait_selftest(max_polls=10, arrive=False) == claire.ETIMEOUT
    assert claire.wait_status() == 32
    cin, cout, shape = 16, 32, (2, 16, 8)
    rng = np.random.default_rng(7)
    x = _bf(rng.standard_normal((cin,) + shape))
    w = _bf(rng.standard_normal((cout, cin, 27)) * 0.2)
    dy = _bf(rng.standard_normal((cout,) + shape))
    L = claire.load_library()
    D, H, W = shape
    V = D * H * W
    xg, dyg = _cl(x), _cl(dy)
    wg = torch.from_numpy(np.ascontiguousarray(np.transpose(w, (0, 2, 1)))).to(torch.bfloat16).cuda()
    y32 = torch.empty((V, cout), device="cuda")
    assert L.claire_conv3d_forward(_p(xg), 1, D, H, W, cin, _p(wg), None, cout, 0, None,
                                   _p(y32), None) == claire.OK
    part = torch.empty(4 * cout * 27 * cin, device="cuda")
    dw = torch.empty((cout, 27, cin), device="cuda")
    assert L.claire_conv3d_wgrad(_p(xg), 1, D, H, W, cin, _p(dyg), cout, _p(part), 4,
                                 _p(dw), None) == claire.OK
    assert claire.wait_status() == 0
    y = np.moveaxis(y32.cpu().numpy().astype(np.float64).reshape(D, H, W, cout), -1, 0)
    assert rel(y, OC.conv3d(x, w)) < 1e-4
    assert rel(np.transpose(dw.cpu().numpy(), (0, 2, 1)), OC.conv3d_weight_grad(x, dy)) < 1e-4


def test_invalid_budgets_are_rejected(claire):
    L = claire.load_library()
    for polls in (0, -1, (1 << 20) + 1):
        assert L.claire_wait_selftest(polls, 0, None) == claire.EINVAL
