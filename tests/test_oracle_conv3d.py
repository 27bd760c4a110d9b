"""Pins for oracle.conv3d: torch's float64 conv3d with circular padding and its
autograd (library route), adjoint identities, brute force at one voxel."""

import numpy as np
import torch

from oracle import conv3d as C


def _case(seed=0, ci=3, co=4, shape=(5, 6, 7)):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((ci,) + shape)
    w = rng.standard_normal((co, ci, 27))
    b = rng.standard_normal(co)
    return x, w, b


def _torch_weight(w):
    return torch.from_numpy(w.reshape(w.shape[0], w.shape[1], 3, 3, 3))


def test_forward_matches_torch_circular_conv3d():
    x, w, b = _case()
    xt = torch.nn.functional.pad(torch.from_numpy(x)[None], (1, 1, 1, 1, 1, 1), mode="circular")
    ref = torch.nn.functional.conv3d(xt, _torch_weight(w), torch.from_numpy(b))[0].numpy()
    assert np.allclose(C.conv3d(x, w, b), ref, atol=1e-12)


def test_gradients_match_torch_autograd():
    x, w, b = _case(1)
    dy = np.random.default_rng(2).standard_normal((w.shape[0],) + x.shape[1:])
    xt = torch.from_numpy(x)[None].requires_grad_(True)
    wt = _torch_weight(w).clone().requires_grad_(True)
    y = torch.nn.functional.conv3d(torch.nn.functional.pad(xt, (1,) * 6, mode="circular"), wt)
    (y * torch.from_numpy(dy)[None]).sum().backward()
    assert np.allclose(C.conv3d_data_grad(dy, w), xt.grad[0].numpy(), atol=1e-11)
    assert np.allclose(C.conv3d_weight_grad(x, dy), wt.grad.numpy().reshape(w.shape), atol=1e-11)


def test_adjoint_identities():
    x, w, _ = _case(3)
    dy = np.random.default_rng(4).standard_normal((w.shape[0],) + x.shape[1:])
    lhs = np.sum(C.conv3d(x, w) * dy)
    assert abs(lhs - np.sum(x * C.conv3d_data_grad(dy, w))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * C.conv3d_weight_grad(x, dy))) < 1e-10 * abs(lhs)


def test_single_voxel_brute_force():
    x, w, b = _case(5, ci=2, co=2, shape=(4, 4, 4))
    y = C.conv3d(x, w, b)
    p = (0, 3, 1)
    acc = b[1]
    for t, (dz, dy, dx) in enumerate(C.OFFSETS):
        for c in range(2):
            acc += w[1, c, t] * x[c, (p[0] + dz) % 4, (p[1] + dy) % 4, (p[2] + dx) % 4]
    assert abs(y[1][p] - acc) < 1e-12
