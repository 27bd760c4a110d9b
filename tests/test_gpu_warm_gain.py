"""What the trained warm start gains over the plain zero-initialised solve.

A U-Net is trained on the GPU (the library's BF16 tensor-core convolutions) on
pairs the solver itself generated: 64^3 phantom pairs, their zero-initialised
solutions as targets.  On held-out pairs every solve is run twice at the same
relative-gradient tolerance with the same denominator ||g(v = 0)||_inf: from
v = 0, and from the network's prediction (with the solver's J(v_pred) <= J(0)
check).  The warm-started solves must need fewer Hessian matvecs on average,
fall back on no pair, converge, and end at the same mismatch.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 64
BETA = 1e-2
TRAIN = 192
EPOCHS = 20
HELD_OUT = 16


@pytest.fixture(scope="module")
def unet():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import unet as U
    return U


def test_trained_warm_start_needs_fewer_matvecs_on_held_out_pairs(unet):
    U = unet
    inputs, targets = [], []
    seeds = list(range(30000, 30000 + TRAIN))
    for i in range(0, TRAIN, 64):
        pairs = U.make_pairs(seeds[i:i + 64], N)
        vs = U.solve_targets(pairs, N, BETA)
        for (m0, m1), v in zip(pairs, vs):
            inputs.append(torch.stack([m0, m1]).contiguous())
            targets.append(v.contiguous())
    model = U.UNet3D(seed=0)
    hist = U.train(model, inputs, targets, EPOCHS, warmup=100)
    assert np.isfinite(hist).all() and hist[-1] < 0.5 * hist[0]
    res = U.evaluate(model, U.make_pairs(list(range(40000, 40000 + HELD_OUT)), N), N, BETA)
    mv_zero = np.mean([r["matvecs_zero"] for r in res])
    mv_warm = np.mean([r["matvecs_warm"] for r in res])
    print(f"held-out matvecs: zero-init {mv_zero:.2f}, warm start {mv_warm:.2f}")
    assert mv_warm < mv_zero
    assert not any(r["fallback"] for r in res)
    assert all(r["grad_rel_zero"] <= 5e-2 and r["grad_rel_warm"] <= 5e-2 for r in res)
    mis_zero = np.mean([r["mismatch_zero"] for r in res])
    mis_warm = np.mean([r["mismatch_warm"] for r in res])
    assert abs(mis_warm - mis_zero) <= 0.05 * mis_zero
