"""The largest grid the benchmark runs (768^3, about 453 M voxels, the
single-registration workload of `bench.py`'s `scale_768`), checked by a
property that holds at any size.

A constant velocity of a whole number of voxels per time step moves the
template by an exact periodic shift: with v_i = k_i h_i (h_i = 2 pi / n_i) the
solution of the transport equation is m(1)(x) = m0(x - v), i.e. m0 rolled by
k_i nodes along axis i.  The RK2 departure points of a constant field are
x - h_t v up to rounding, and a tricubic interpolant at (almost) integer
offsets returns the node values, so every SL step reproduces the shift to
rounding.  The template is FP16-representable, so the mixed form, which stores
the state in FP16 between the steps, must give the same shift.  This covers
the 64-bit offsets, the TMA tensor maps (589,824 brick rows) and the tile grids
at the maximum size; the oracle parity of the same kernels is pinned on smaller
grids.
"""

import math

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 768
SHAPE = (N, N, N)
SHIFT = (4, -8, 12)            # voxels over unit time: 1, -2, 3 per step at nt = 4


@pytest.fixture(scope="module")
def claire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 170e9:
        pytest.skip("needs about 170 GB of free device memory")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    C.load_library()
    return C


def _template():
    gen = torch.Generator(device="cuda").manual_seed(768)
    return torch.rand(SHAPE, device="cuda", generator=gen).half().float()


@pytest.mark.parametrize("precision", [0, 1])
def test_integer_shift_is_exact_at_768(claire, precision):
    m0 = _template()
    h = 2.0 * math.pi / N
    v = torch.empty((3,) + SHAPE, device="cuda")
    for a in range(3):
        v[a].fill_(SHIFT[a] * h)
    with claire.Context(SHAPE, nt=4, beta_v=1e-3, precision=precision) as ctx:
        ctx.set_images(m0, m0)
        m1 = ctx.transport(v)
    expected = torch.roll(m0, shifts=SHIFT, dims=(0, 1, 2))
    err = (m1 - expected).abs().max().item()
    assert err < 2e-5, err
    del v, m1, expected, m0
    torch.cuda.empty_cache()
    assert claire.wait_status() == 0
