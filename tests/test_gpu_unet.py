"""Learned warm start: the U-Net kernels against FP64 references.

Convolutions (forward, data gradient via flipped weights, weight gradient)
against oracle.conv3d on the same BF16-rounded inputs (the GPU accumulates in
FP32: tolerance 1e-4 relative); layer ops against numpy; spectral resampling
against oracle.spectral.restrict / prolong; the whole network's loss and
weight gradients against a float64 torch CPU reference that rounds every
stored activation and gradient to BF16 like the GPU path and uses the GPU's
ReLU masks (tolerance 3e-2).
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import conv3d as OC, spectral as OS


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire as C
    return C


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _bf(a):
    """numpy float64 -> BF16-rounded float64."""
    return torch.from_numpy(np.asarray(a, dtype=np.float64)).to(torch.bfloat16).double().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _to_cl(x):
    """[C][B*D..] planar (per sample [C][D][H][W]) -> channels-last [V][C] bf16 CUDA."""
    return torch.from_numpy(np.ascontiguousarray(np.moveaxis(x, 0, -1).reshape(-1, x.shape[0]))).to(
        torch.bfloat16).cuda()


# shapes with H % 16 == 0 and W % 8 == 0 take the halo-tile forward kernel (one
# chunk group, weights resident or streamed; several groups for 96 input channels
# and, in the data gradient, 80 and 128), the first three the per-tap gather kernel.
# Weight gradient: tcgen05 with the output channels as MMA rows where W % 8 == 0,
# H % 16 == 0 and cin <= cout <= 128; else, with W % 8 == 0, H % 8 == 0 and
# cout <= 32 or H % 16 != 0, tcgen05 with the input channels as MMA rows (48 -> 16,
# 64 -> 32, 96 -> 32, the 8^3 and H = 8 shapes, two row blocks for 192 -> 32);
# else mma.sync (192 -> 64)
@pytest.mark.parametrize("cin,cout,shape", [(16, 16, (8, 6, 10)), (48, 32, (6, 6, 6)),
                                            (32, 64, (4, 8, 4)), (16, 16, (4, 16, 8)),
                                            (48, 16, (3, 16, 16)), (64, 32, (2, 32, 8)),
                                            (32, 128, (5, 16, 24)), (16, 80, (2, 16, 8)),
                                            (96, 32, (3, 16, 8)), (48, 16, (2, 8, 16)),
                                            (128, 128, (8, 8, 8)), (64, 128, (4, 8, 8)),
                                            (192, 32, (2, 16, 8)), (192, 64, (2, 16, 8))])
def test_conv_forward_dgrad_wgrad_match_oracle(lib, cin, cout, shape):
    rng = np.random.default_rng(cin + cout)
    x = _bf(rng.standard_normal((cin,) + shape))
    w = _bf(rng.standard_normal((cout, cin, 27)) * 0.2)
    b = rng.standard_normal(cout)
    dy = _bf(rng.standard_normal((cout,) + shape))
    L = lib.load_library()
    D, H, W = shape
    V = D * H * W
    xg, dyg = _to_cl(x), _to_cl(dy)
    wg = torch.from_numpy(np.ascontiguousarray(np.transpose(w, (0, 2, 1)))).to(torch.bfloat16).cuda()
    bg = torch.from_numpy(b).float().cuda()
    y32 = torch.empty((V, cout), device="cuda")
    assert L.claire_conv3d_forward(_p(xg), 1, D, H, W, cin, _p(wg), _p(bg), cout, 0, None,
                                   _p(y32), None) == 0
    wf = torch.empty((cin, 27, cout), device="cuda", dtype=torch.bfloat16)
    assert L.claire_conv3d_flip_weights(_p(wg), cout, cin, _p(wf), None) == 0
    dx32 = torch.empty((V, cin), device="cuda")
    assert L.claire_conv3d_forward(_p(dyg), 1, D, H, W, cout, _p(wf), None, cin, 0, None,
                                   _p(dx32), None) == 0
    nsplit = 3
    part = torch.empty(nsplit * cout * 27 * cin, device="cuda")
    dw = torch.empty((cout, 27, cin), device="cuda")
    assert L.claire_conv3d_wgrad(_p(xg), 1, D, H, W, cin, _p(dyg), cout, _p(part), nsplit,
                                 _p(dw), None) == 0
    torch.cuda.synchronize()
    cl = lambda t, c: np.moveaxis(t.cpu().numpy().astype(np.float64).reshape(D, H, W, c), -1, 0)
    assert rel(cl(y32, cout), OC.conv3d(x, w, b)) < 1e-4
    assert rel(cl(dx32, cin), OC.conv3d_data_grad(dy, w)) < 1e-4
    assert rel(np.transpose(dw.cpu().numpy(), (0, 2, 1)), OC.conv3d_weight_grad(x, dy)) < 1e-4


@pytest.mark.parametrize("B,D,H,W,cin,cout", [(3, 6, 6, 6, 16, 16),      # V = 648, ragged
                                              (2, 4, 16, 8, 32, 16)])    # halo-tile kernel
def test_conv_batch_and_ragged_voxel_count(lib, B, D, H, W, cin, cout):
    _batch_case(lib, B, D, H, W, cin, cout)


def test_tensor_core_weight_gradient_on_many_tiles(lib):
    """The tcgen05 weight gradient with persistent CTAs that each accumulate several
    8 x 16 tiles (128 tiles over 32 CTAs) against the FP64 oracle."""
    rng = np.random.default_rng(11)
    B, D, H, W, cin, cout = 2, 8, 32, 32, 32, 48
    xs = [_bf(rng.standard_normal((cin, D, H, W))) for _ in range(B)]
    dys = [_bf(rng.standard_normal((cout, D, H, W))) for _ in range(B)]
    xg = torch.cat([_to_cl(x) for x in xs])
    dyg = torch.cat([_to_cl(d) for d in dys])
    nsplit = 32
    part = torch.empty(nsplit * cout * 27 * cin, device="cuda")
    dw = torch.empty((cout, 27, cin), device="cuda")
    L = lib.load_library()
    assert L.claire_conv3d_wgrad(_p(xg), B, D, H, W, cin, _p(dyg), cout, _p(part), nsplit,
                                 _p(dw), None) == 0
    torch.cuda.synchronize()
    ref = sum(OC.conv3d_weight_grad(x, d) for x, d in zip(xs, dys))
    assert rel(np.transpose(dw.cpu().numpy(), (0, 2, 1)), ref) < 1e-4


def _batch_case(lib, B, D, H, W, cin, cout):
    rng = np.random.default_rng(7)
    xs = [_bf(rng.standard_normal((cin, D, H, W))) for _ in range(B)]
    w = _bf(rng.standard_normal((cout, cin, 27)) * 0.2)
    xg = torch.cat([_to_cl(x) for x in xs])
    wg = torch.from_numpy(np.ascontiguousarray(np.transpose(w, (0, 2, 1)))).to(torch.bfloat16).cuda()
    y32 = torch.empty((B * D * H * W, cout), device="cuda")
    L = lib.load_library()
    assert L.claire_conv3d_forward(_p(xg), B, D, H, W, cin, _p(wg), None, cout, 1, None,
                                   _p(y32), None) == 0
    torch.cuda.synchronize()
    y = y32.cpu().numpy().reshape(B, D, H, W, cout)
    for bi, x in enumerate(xs):                          # periodic padding within each sample
        ref = np.maximum(OC.conv3d(x, w), 0.0)
        assert rel(np.moveaxis(y[bi], -1, 0), ref) < 1e-4


def test_layer_ops_match_numpy(lib):
    rng = np.random.default_rng(8)
    L = lib.load_library()
    B, D, C = 2, 8, 16
    x = torch.from_numpy(rng.standard_normal((B, D, D, D, C))).to(torch.bfloat16).cuda()
    xp = torch.empty((B, D // 2, D // 2, D // 2, C), device="cuda", dtype=torch.bfloat16)
    assert L.claire_unet_op(1, _p(x), _p(xp), 0, C, 0, 0, B, D, D, D, None) == 0
    up = torch.zeros((B, D, D, D, 2 * C), device="cuda", dtype=torch.bfloat16)
    assert L.claire_unet_op(3, _p(xp), _p(up), 0, C, 2 * C, C, B, D // 2, D // 2, D // 2, None) == 0
    torch.cuda.synchronize()
    xn = x.double().cpu().numpy()
    pooled = xn.reshape(B, D // 2, 2, D // 2, 2, D // 2, 2, C).mean(axis=(2, 4, 6))
    assert np.allclose(xp.double().cpu().numpy(), pooled, rtol=1e-2, atol=1e-2)
    upn = up.double().cpu().numpy()
    ref_up = np.repeat(np.repeat(np.repeat(xp.double().cpu().numpy(), 2, 1), 2, 2), 2, 3)
    assert np.array_equal(upn[..., C:], ref_up) and np.all(upn[..., :C] == 0)


@pytest.mark.parametrize("src,dst", [((32, 24, 16), (16, 12, 8)), ((16, 12, 8), (32, 24, 16))])
def test_spectral_resample_matches_oracle(lib, src, dst):
    from paper_2401_17493_b300 import synth
    f = np.stack([synth.smooth_field(src, 5, s) for s in (1, 2, 3)]).astype(np.float32)
    out = torch.empty((3,) + dst, device="cuda")
    L = lib.load_library()
    assert L.claire_resample(*src, _p(torch.from_numpy(f).cuda()), *dst, _p(out), 3, None) == 0
    op = OS.restrict if np.prod(dst) < np.prod(src) else OS.prolong
    ref = np.stack([op(f[i].astype(np.float64), dst) for i in range(3)])
    assert rel(out.cpu().numpy(), ref) < 1e-5


class _BF(torch.autograd.Function):
    """Round to BF16 in the forward pass and the gradient in the backward pass,
    where the GPU path stores an activation and its gradient in BF16."""

    @staticmethod
    def forward(ctx, x):
        return x.to(torch.bfloat16).double()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).double()


class _BFGrad(torch.autograd.Function):
    """Identity forward; BF16-rounded gradient (FP32 output, BF16 gradient)."""

    @staticmethod
    def forward(ctx, x):
        return x.clone()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).double()


# GPU activation holding each layer's output (its ReLU mask)
_OUT_ACT = {"e0a": "e0a", "e0b": "e0", "e1a": "e1a", "e1b": "e1", "e2a": "e2a", "e2b": "e2",
            "ba": "ba", "bb": "b", "d2a": "d2a", "d2b": "d2", "d1a": "d1a", "d1b": "d1",
            "d0a": "d0a", "d0b": "d0"}


def _torch_unet_reference(model, fields, target):
    """float64 CPU torch network that rounds every tensor the GPU path stores in
    BF16 (activations and their gradients) to BF16, with the ReLU masks of the
    GPU's forward pass: a forward value that differs by one BF16 rounding can sit
    on the other side of zero, and a flipped mask element changes the gradient by
    O(1) at that voxel, so the two backward passes are compared under one mask."""
    import torch.nn.functional as F
    rb = _BF.apply
    B = len(fields)
    n = fields[0].shape[-1]

    def mask(layer):
        a = model.acts[_OUT_ACT[layer]].float().cpu()
        m = n >> __import__("paper_2401_17493_b300.unet", fromlist=["x"]).LAYER_LEVEL[layer]
        return (a.reshape(B, m, m, m, -1).permute(0, 4, 1, 2, 3) > 0).double()
    W = {}
    for k, l in model.layers.items():
        w = l.w.double().cpu().reshape(l.cout, 3, 3, 3, l.cin).permute(0, 4, 1, 2, 3).contiguous()
        W[k] = (w.requires_grad_(True), l.b32.double().cpu().requires_grad_(True))

    def conv(x, k, relu=True):
        y = F.conv3d(F.pad(x, (1,) * 6, mode="circular"), W[k][0], W[k][1])
        return rb(y * mask(k)) if relu else _BFGrad.apply(y)

    x = torch.stack([torch.from_numpy(f) for f in fields]).double()      # [B][2][n][n][n]
    x = rb(F.pad(x, (0, 0, 0, 0, 0, 0, 0, 14)))
    e0 = conv(conv(x, "e0a"), "e0b")
    e1 = conv(conv(rb(F.avg_pool3d(e0, 2)), "e1a"), "e1b")
    e2 = conv(conv(rb(F.avg_pool3d(e1, 2)), "e2a"), "e2b")
    b = conv(conv(rb(F.avg_pool3d(e2, 2)), "ba"), "bb")
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    d2 = conv(conv(rb(torch.cat([up(b), e2], 1)), "d2a"), "d2b")
    d1 = conv(conv(rb(torch.cat([up(d2), e1], 1)), "d1a"), "d1b")
    d0 = conv(conv(rb(torch.cat([up(d1), e0], 1)), "d0a"), "d0b")
    out = conv(d0, "head", relu=False)[:, :3]                           # [B][3][n][n][n]
    loss = ((out - target) ** 2).mean()
    loss.backward()
    return loss.item(), {k: (w.grad.permute(0, 2, 3, 4, 1).reshape(w.shape[0], 27, -1).numpy(),
                             bb.grad.numpy()) for k, (w, bb) in W.items()}


def test_unet_loss_and_gradients_match_float64_reference(lib):
    from paper_2401_17493_b300 import unet
    n, B = 16, 2
    rng = np.random.default_rng(9)
    fields = [rng.random((2, n, n, n)).astype(np.float32) for _ in range(B)]
    target = rng.standard_normal((B, 3, n, n, n)).astype(np.float32) * 0.3
    model = unet.UNet3D(seed=3)
    out = model.forward([torch.from_numpy(f).cuda() for f in fields], B, n=n)
    tgt = torch.from_numpy(np.ascontiguousarray(np.moveaxis(target, 1, 0).reshape(3, -1))).cuda()
    loss = float(model.loss_and_backward(out, tgt))
    torch.cuda.synchronize()
    ref_loss, ref_grads = _torch_unet_reference(model, fields, torch.from_numpy(target).double())
    assert abs(loss - ref_loss) / ref_loss < 1e-2
    errs = {k: (rel(l.dw.cpu().numpy(), ref_grads[k][0]), rel(l.db.cpu().numpy(), ref_grads[k][1]))
            for k, l in model.layers.items()}
    print("weight / bias gradient errors:", {k: (f"{a:.1e}", f"{b:.1e}") for k, (a, b) in errs.items()})
    for k, (ew, eb) in errs.items():
        assert ew < 3e-2 and eb < 3e-2, (k, ew, eb)


def test_a_few_training_steps_lower_the_loss(lib):
    from paper_2401_17493_b300 import unet
    n, B = 16, 2
    rng = np.random.default_rng(10)
    fields = [torch.from_numpy(rng.random((2, n, n, n)).astype(np.float32)).cuda() for _ in range(B)]
    # a target the network can represent: fixed combinations of the two input images
    tgt = torch.stack([torch.stack([f[0] - f[1], 0.5 * f[0], -0.5 * f[1]]) for f in fields], 1)
    tgt = tgt.reshape(3, -1).contiguous()
    model = unet.UNet3D(seed=4)
    losses = []
    for _ in range(60):
        out = model.forward(fields, B, n=n)
        losses.append(float(model.loss_and_backward(out, tgt)))
        model.step(1e-3)
    assert losses[-1] < 0.8 * losses[0]


@pytest.mark.parametrize("V,C", [(1, 16), (1000, 16), (262147, 32), (70001, 128), (5003, 512)])
def test_bias_gradient_matches_a_float64_sum(lib, V, C):
    """db[c] = sum_v dy[v][c] for ragged voxel counts, several channel counts and
    fewer voxels than reduction CTAs; invalid arguments are refused."""
    from paper_2401_17493_b300 import claire as C_
    L = C_.load_library()
    gen = torch.Generator(device="cuda").manual_seed(V + C)
    dy = torch.randn((V, C), device="cuda", generator=gen).to(torch.bfloat16)
    db = torch.empty(C, device="cuda")
    part = torch.empty(592 * C, device="cuda", dtype=torch.float64)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.claire_unet_bias_grad(ctypes.c_void_p(dy.data_ptr()), V, C,
                                   ctypes.c_void_p(db.data_ptr()),
                                   ctypes.c_void_p(part.data_ptr()), 592, st) == C_.OK
    ref = dy.double().sum(0)
    err = (db.double() - ref).abs().max().item() / max(1.0, ref.abs().max().item())
    assert err < 1e-6
    # odd channel counts, too many channels, no scratch
    for bad in [(C + 1, 592, part), (514, 592, part), (C, 592, None), (C, 0, part)]:
        c_, nb, p = bad
        assert L.claire_unet_bias_grad(ctypes.c_void_p(dy.data_ptr()), V, c_,
                                       ctypes.c_void_p(db.data_ptr()),
                                       None if p is None else ctypes.c_void_p(p.data_ptr()),
                                       nb, st) == C_.EINVAL
