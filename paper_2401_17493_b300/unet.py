"""Learned warm start: a 3D U-Net that predicts the registration velocity.

Not part of the paper (which cites learning only as related work): a small
U-Net (4 levels, 16/32/64/128 channels, BF16 weights and activations, FP32
accumulation, 3x3x3 periodic convolutions) maps the image pair (m0, m1),
spectrally restricted to 64^3, to a velocity on 64^3 that is spectrally
prolonged to the registration grid and used as the solver's initial guess.
The plain zero-initialised solve is both the fallback (taken when the
prediction raises the objective) and the accuracy reference (same
relative-gradient tolerance, denominator ||g(v = 0)||_inf for both).

Every layer runs in the library's kernels (claire_conv3d_forward / wgrad /
flip_weights, claire_unet_op / bias_grad / pack / mse / adam,
claire_resample); this module only sequences them and owns the buffers
(torch CUDA tensors).

    python -m paper_2401_17493_b300.unet --train 2000 --eval 200 --epochs 40 --out results.json
"""

import argparse
import ctypes
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))

from paper_2401_17493_b300 import claire as C  # noqa: E402

IN_CH = 16          # (m0, m1) padded to one 16-channel k-chunk
OUT_CH = 16         # velocity in channels 0..2, padded to 16
V_SCALE = 0.1       # network output * V_SCALE = velocity (physical units)
PRECOND = 1         # registration solves: two-level zero-velocity preconditioner (Sec. 2.6)
MAX_INNER = 10      # nested CG cap of that preconditioner


def wgrad_splits(V):
    """Voxel splits of a weight gradient over V voxels (its partial buffer holds this
    many copies of dW): at least one tensor-core weight-gradient CTA per SM."""
    return max(1, min(160, V // 128))


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


BIAS_BLOCKS = 592           # CTAs of the bias-gradient reduction (4 per SM of a B300)


def _check(st, what):
    if st != C.OK:
        raise C.ClaireError(st, what)


class Conv:
    """One 3x3x3 periodic conv layer: FP32 master weights, BF16 copies, Adam state."""

    def __init__(self, cin, cout, relu, gen, scale=1.0):
        import torch
        self.cin, self.cout, self.relu = cin, cout, relu
        std = scale * math.sqrt(2.0 / (27 * cin))
        self.w32 = (torch.randn((cout, 27, cin), generator=gen, device="cuda") * std).contiguous()
        self.b32 = torch.zeros(cout, device="cuda")
        self.w = self.w32.to(torch.bfloat16)
        self.wf = torch.empty((cin, 27, cout), device="cuda", dtype=torch.bfloat16)
        self.dw = torch.zeros_like(self.w32)
        self.db = torch.zeros_like(self.b32)
        self.mw, self.vw = torch.zeros_like(self.w32), torch.zeros_like(self.w32)
        self.mb, self.vb = torch.zeros_like(self.b32), torch.zeros_like(self.b32)

    def forward(self, x, vol, y=None, y32=None):
        import torch
        V = vol[0] * vol[1] * vol[2] * vol[3]
        if y is None and y32 is None:
            y = torch.empty((V, self.cout), device="cuda", dtype=torch.bfloat16)
        _check(C.load_library().claire_conv3d_forward(
            _p(x), *vol, self.cin, _p(self.w), _p(self.b32), self.cout, int(self.relu),
            _p(y), _p(y32), _stream()), "conv3d_forward")
        return y

    def backward(self, x, y, dy, vol, need_dx=True, partial=None, bias_part=None):
        """dy: gradient w.r.t. this layer's (post-activation) output, BF16 [V][cout]
        (overwritten); accumulates nothing: sets dw, db; returns dx or None.
        partial: scratch of the weight gradient; bias_part: FP64 scratch of the
        bias gradient (BIAS_BLOCKS x cout doubles)."""
        import torch
        L = C.load_library()
        V = vol[0] * vol[1] * vol[2] * vol[3]
        s = _stream()
        if self.relu:
            _check(L.claire_unet_op(0, _p(y), _p(dy), V, self.cout, 0, 0, 0, 0, 0, 0, s),
                   "relu_bwd")
        nsplit = wgrad_splits(V)
        need = nsplit * self.cout * 27 * self.cin
        if partial is None or partial.numel() < need:
            raise ValueError("wgrad partial buffer too small")
        _check(L.claire_conv3d_wgrad(_p(x), *vol, self.cin, _p(dy), self.cout, _p(partial),
                                     nsplit, _p(self.dw), s), "wgrad")
        if bias_part is None or bias_part.numel() < BIAS_BLOCKS * self.cout:
            raise ValueError("bias-gradient scratch buffer too small")
        _check(L.claire_unet_bias_grad(_p(dy), V, self.cout, _p(self.db), _p(bias_part),
                                       BIAS_BLOCKS, s), "bias_grad")
        if not need_dx:
            return None
        _check(L.claire_conv3d_flip_weights(_p(self.w), self.cout, self.cin, _p(self.wf), s),
               "flip")
        dx = torch.empty((V, self.cin), device="cuda", dtype=torch.bfloat16)
        _check(L.claire_conv3d_forward(_p(dy), *vol, self.cout, _p(self.wf), None, self.cin, 0,
                                       _p(dx), None, s), "dgrad")
        return dx

    def adam(self, lr, step, b1=0.9, b2=0.999, eps=1e-8):
        L = C.load_library()
        s = _stream()
        _check(L.claire_unet_adam(self.w32.numel(), _p(self.w32), _p(self.dw), _p(self.mw),
                                  _p(self.vw), lr, b1, b2, eps, step, _p(self.w), s), "adam")
        _check(L.claire_unet_adam(self.b32.numel(), _p(self.b32), _p(self.db), _p(self.mb),
                                  _p(self.vb), lr, b1, b2, eps, step, None, s), "adam")

    def state(self):
        return {"w": self.w32, "b": self.b32}


# grid level (0 = 64^3 ... 3 = 8^3) at which each layer runs
LAYER_LEVEL = {"e0a": 0, "e0b": 0, "e1a": 1, "e1b": 1, "e2a": 2, "e2b": 2, "ba": 3, "bb": 3,
               "d2a": 2, "d2b": 2, "d1a": 1, "d1b": 1, "d0a": 0, "d0b": 0, "head": 0}


class UNet3D:
    """enc 16-32-64-128 (two convs per level, 2x2x2 average pooling), decoder with
    nearest upsampling + skip concatenation, 3x3x3 head to 3 velocity channels."""

    def __init__(self, seed=0, base=16):
        import torch
        gen = torch.Generator(device="cuda").manual_seed(seed)
        c = [base, 2 * base, 4 * base, 8 * base]
        self.c = c
        self.layers = {
            "e0a": Conv(IN_CH, c[0], True, gen), "e0b": Conv(c[0], c[0], True, gen),
            "e1a": Conv(c[0], c[1], True, gen), "e1b": Conv(c[1], c[1], True, gen),
            "e2a": Conv(c[1], c[2], True, gen), "e2b": Conv(c[2], c[2], True, gen),
            "ba": Conv(c[2], c[3], True, gen), "bb": Conv(c[3], c[3], True, gen),
            "d2a": Conv(c[3] + c[2], c[2], True, gen), "d2b": Conv(c[2], c[2], True, gen),
            "d1a": Conv(c[2] + c[1], c[1], True, gen), "d1b": Conv(c[1], c[1], True, gen),
            "d0a": Conv(c[1] + c[0], c[0], True, gen), "d0b": Conv(c[0], c[0], True, gen),
            "head": Conv(c[0], OUT_CH, False, gen, scale=0.1),
        }
        self.step_count = 0
        self.partial = None
        self.wpart = None
        self.bpart = None           # FP64 scratch of the bias gradients

    @property
    def parameters(self):
        return sum(l.w32.numel() + l.b32.numel() for l in self.layers.values())

    # ---------------------------------------------------------------- helpers
    @staticmethod
    def _op(op, a, b, V=0, C_=0, Cdst=0, off=0, vol=(0, 0, 0, 0)):
        _check(C.load_library().claire_unet_op(op, _p(a), _p(b), V, C_, Cdst, off, *vol,
                                               _stream()), f"unet_op {op}")

    @staticmethod
    def _empty(V, ch):
        import torch
        return torch.empty((V, ch), device="cuda", dtype=torch.bfloat16)

    def forward(self, fields, B, n=64):
        """fields: FP32 [B][2][n][n][n] (m0, m1 per sample, stacked as planar
        per-sample fields).  Returns the FP32 network output [V][OUT_CH] and keeps
        the activations for backward."""
        import torch
        L = self.layers
        c = self.c
        vols = [(B, n >> k, n >> k, n >> k) for k in range(4)]
        Vs = [v[0] * v[1] * v[2] * v[3] for v in vols]
        a = {}
        # channels-last input: per sample pack its 2 planar fields
        x0 = self._empty(Vs[0], IN_CH)
        per = Vs[0] // B
        for b in range(B):
            _check(C.load_library().claire_unet_pack(per, 2, _p(fields[b]), 1.0, IN_CH,
                                                     ctypes.c_void_p(x0.data_ptr() + 2 * per * IN_CH * b),
                                                     _stream()), "pack")
        a["x0"] = x0
        a["e0a"] = L["e0a"].forward(x0, vols[0])
        a["e0"] = L["e0b"].forward(a["e0a"], vols[0])
        a["p0"] = self._empty(Vs[1], c[0]); self._op(1, a["e0"], a["p0"], C_=c[0], vol=vols[0])
        a["e1a"] = L["e1a"].forward(a["p0"], vols[1])
        a["e1"] = L["e1b"].forward(a["e1a"], vols[1])
        a["p1"] = self._empty(Vs[2], c[1]); self._op(1, a["e1"], a["p1"], C_=c[1], vol=vols[1])
        a["e2a"] = L["e2a"].forward(a["p1"], vols[2])
        a["e2"] = L["e2b"].forward(a["e2a"], vols[2])
        a["p2"] = self._empty(Vs[3], c[2]); self._op(1, a["e2"], a["p2"], C_=c[2], vol=vols[2])
        a["ba"] = L["ba"].forward(a["p2"], vols[3])
        a["b"] = L["bb"].forward(a["ba"], vols[3])
        # decoder: concat(up(coarse), skip)
        for lvl, (coarse, skip, ca, cs, la, lb) in enumerate(
                [("b", "e2", c[3], c[2], "d2a", "d2b"), ("d2", "e1", c[2], c[1], "d1a", "d1b"),
                 ("d1", "e0", c[1], c[0], "d0a", "d0b")]):
            k = 2 - lvl                                          # fine level index
            cat = self._empty(Vs[k], ca + cs)
            self._op(3, a[coarse], cat, C_=ca, Cdst=ca + cs, off=0, vol=vols[k + 1])
            self._op(5, a[skip], cat, V=Vs[k], C_=cs, Cdst=ca + cs, off=ca)
            a[f"c{k}"] = cat
            a[la] = L[la].forward(cat, vols[k])
            a[f"d{k}"] = L[lb].forward(a[la], vols[k])
        out = torch.empty((Vs[0], OUT_CH), device="cuda")
        L["head"].forward(a["d0"], vols[0], y=None, y32=out)
        self.acts, self.vols, self.Vs = a, vols, Vs
        return out

    def loss_and_backward(self, out, target):
        """Mean squared error against target (FP32 planar [3][V0], in network
        units: velocity / V_SCALE) and the gradients of every layer."""
        import torch
        L, a, vols, Vs, c = self.layers, self.acts, self.vols, self.Vs, self.c
        V0 = Vs[0]
        nb = 1024
        if self.partial is None:
            self.partial = torch.empty(nb + 1, device="cuda", dtype=torch.float64)
        dout = self._empty(V0, OUT_CH)
        _check(C.load_library().claire_unet_mse(V0, OUT_CH, _p(out), _p(target), 1.0,
                                                _p(dout), None, _p(self.partial), nb,
                                                ctypes.c_void_p(self.partial.data_ptr() + 8 * nb),
                                                _stream()), "mse")
        loss = self.partial[nb]
        need = max(wgrad_splits(V) * l.cout * 27 * l.cin
                   for l, V in [(L[k], Vs[lv]) for k, lv in LAYER_LEVEL.items()])
        if self.wpart is None or self.wpart.numel() < need:
            self.wpart = torch.empty(need, device="cuda")
        wp = self.wpart
        if self.bpart is None:
            self.bpart = torch.empty(BIAS_BLOCKS * max(l.cout for l in L.values()),
                                     device="cuda", dtype=torch.float64)
        bp = self.bpart

        def bwd(name, x, y, dy, lvl, need_dx=True):
            return L[name].backward(x, y, dy, vols[lvl], need_dx=need_dx, partial=wp,
                                    bias_part=bp)

        def split(gcat, lvl, ca, cs):
            """d(concat(up(coarse), skip)) -> (d coarse, d skip)."""
            gs = self._empty(Vs[lvl], cs)
            self._op(6, gcat, gs, V=Vs[lvl], C_=cs, Cdst=ca + cs, off=ca)
            gc = self._empty(Vs[lvl + 1], ca)
            self._op(4, gcat, gc, C_=ca, Cdst=ca + cs, off=0, vol=vols[lvl + 1])
            return gc, gs

        def into_encoder(gpool, gskip, lvl, ch):
            """d(e_lvl) = pool adjoint of d(p_lvl) + skip gradient."""
            ge = self._empty(Vs[lvl], ch)
            self._op(2, gpool, ge, C_=ch, vol=vols[lvl])
            self._op(7, gskip, ge, V=Vs[lvl], C_=ch)
            return ge

        g = bwd("head", a["d0"], None, dout, 0)                 # d(d0)
        g = bwd("d0b", a["d0a"], a["d0"], g, 0)                  # d(d0a)
        g = bwd("d0a", a["c0"], a["d0a"], g, 0)                  # d(c0)
        g, gs0 = split(g, 0, c[1], c[0])                         # d(d1), d(e0) skip
        g = bwd("d1b", a["d1a"], a["d1"], g, 1)
        g = bwd("d1a", a["c1"], a["d1a"], g, 1)                  # d(c1)
        g, gs1 = split(g, 1, c[2], c[1])                         # d(d2), d(e1) skip
        g = bwd("d2b", a["d2a"], a["d2"], g, 2)
        g = bwd("d2a", a["c2"], a["d2a"], g, 2)                  # d(c2)
        g, gs2 = split(g, 2, c[3], c[2])                         # d(b), d(e2) skip
        g = bwd("bb", a["ba"], a["b"], g, 3)
        g = bwd("ba", a["p2"], a["ba"], g, 3)                    # d(p2)
        g = into_encoder(g, gs2, 2, c[2])                        # d(e2)
        g = bwd("e2b", a["e2a"], a["e2"], g, 2)
        g = bwd("e2a", a["p1"], a["e2a"], g, 2)                  # d(p1)
        g = into_encoder(g, gs1, 1, c[1])                        # d(e1)
        g = bwd("e1b", a["e1a"], a["e1"], g, 1)
        g = bwd("e1a", a["p0"], a["e1a"], g, 1)                  # d(p0)
        g = into_encoder(g, gs0, 0, c[0])                        # d(e0)
        g = bwd("e0b", a["e0a"], a["e0"], g, 0)
        bwd("e0a", a["x0"], a["e0a"], g, 0, need_dx=False)
        return loss

    def step(self, lr):
        self.step_count += 1
        for l in self.layers.values():
            l.adam(lr, self.step_count)

    def predict(self, fields, B, n=64):
        """Velocity (planar FP32 [B][3][n][n][n]) for a batch of restricted pairs."""
        import torch
        out = self.forward(fields, B, n)
        V0 = out.shape[0]
        pred = torch.empty((3, V0), device="cuda")
        _check(C.load_library().claire_unet_mse(V0, OUT_CH, _p(out), None, V_SCALE, None,
                                                _p(pred), None, 1024, None, _stream()), "pred")
        per = V0 // B
        return pred.reshape(3, B, per).permute(1, 0, 2).reshape(B, 3, n, n, n).contiguous()


def resample(x, shape_in, shape_out, ncomp):
    import torch
    out = torch.empty((ncomp,) + tuple(shape_out), device="cuda")
    _check(C.load_library().claire_resample(*shape_in, _p(x), *shape_out, _p(out), ncomp,
                                            _stream()), "resample")
    return out


# ---------------------------------------------------------------- pipeline

def make_pairs(seeds, n):
    """Seeded 128^3 phantom pairs (generated on the GPU, same family as the bench)."""
    from paper_2401_17493_b300 import synth
    return [synth.ellipsoid_pair_torch((n, n, n), seed=s) for s in seeds]


def solve_targets(pairs, n, beta, eps_opt=5e-2, batch=8):
    """Zero-initialised solves of every pair (the training targets)."""
    import torch
    out = []
    for i in range(0, len(pairs), batch):
        chunk = pairs[i:i + batch]
        ctxs = []
        for m0, m1 in chunk:
            ctx = C.Context((n, n, n), nt=4, beta_v=beta, eps_opt=eps_opt, graphs=1,
                            precond=PRECOND, max_inner=MAX_INNER)
            ctx.set_images(m0, m1)
            ctxs.append(ctx)
        vs, stats = C.solve_batch(ctxs)
        out.extend(vs)
        for c in ctxs:
            c.close()
    torch.cuda.synchronize()
    return out


def symmetry(fields, target, g):
    """Element g (0..47) of the cube's symmetry group applied to a training
    sample: the axes are permuted (g // 8 indexes the 6 permutations) and
    flipped (bits of g % 8).  The registration problem is covariant under it
    (L = -Lap and the L2 distance are invariant; transport commutes with it),
    so the relabelled pair has the relabelled velocity: components permuted
    with the axes and negated along flipped axes.  torch.flip maps index i to
    n - 1 - i, a reflection composed with a one-voxel shift, which the periodic
    problem also commutes with."""
    import itertools
    perm = list(itertools.permutations(range(3)))[g // 8]
    flips = [d for d in range(3) if (g % 8) >> d & 1]
    sp = (0, 1 + perm[0], 1 + perm[1], 1 + perm[2])
    f = fields.permute(*sp)
    t = target[list(perm)].permute(*sp)
    if flips:
        f = f.flip([1 + d for d in flips])
        t = t.flip([1 + d for d in flips])
        sign = t.new_ones(3)
        sign[flips] = -1.0
        t = t * sign.reshape(3, 1, 1, 1)
    return f.contiguous(), t.contiguous()


def train(model, inputs, targets, epochs, lr=5e-4, batch=4, seed=0, log=None, warmup=250,
          augment=False):
    """Adam with a linear warm-up over the first `warmup` steps, then a cosine
    decay per epoch (the warm-up keeps the first large Adam steps from
    silencing the ReLUs, which left the loss at the zero-prediction plateau).
    With augment, every sample of every step is relabelled by a random element
    of the cube's symmetry group (`symmetry`)."""
    import torch
    rng = np.random.default_rng(seed)
    n_in = len(inputs)
    hist = []
    step = 0
    for ep in range(epochs):
        order = rng.permutation(n_in)
        tot = 0.0
        nb = 0
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / max(1, epochs)))
        for i in range(0, n_in - batch + 1, batch):
            idx = order[i:i + batch]
            if augment:
                pairs = [symmetry(inputs[j], targets[j], int(rng.integers(0, 48))) for j in idx]
                fields = [p[0] for p in pairs]
                tgts = [p[1] for p in pairs]
            else:
                fields = [inputs[j] for j in idx]
                tgts = [targets[j] for j in idx]
            tgt = torch.cat([t.reshape(3, 1, -1) for t in tgts], dim=1).reshape(3, -1)
            out = model.forward(fields, len(idx))
            loss = model.loss_and_backward(out, (tgt / V_SCALE).contiguous())  # network units
            step += 1
            model.step(lr_ep * min(1.0, step / max(1, warmup)))
            tot += float(loss)
            nb += 1
        hist.append(tot / max(1, nb))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def _predict_batch(model, pairs, n):
    """Warm-start velocities of a list of (m0, m1) pairs on the n^3 grid: one batched
    restriction of all images to 64^3, one network pass, one batched prolongation."""
    import torch
    B = len(pairs)
    imgs = torch.stack([f for mm in pairs for f in mm]).contiguous()          # (2B, n, n, n)
    small = resample(imgs, (n, n, n), (64, 64, 64), 2 * B).reshape(B, 2, 64, 64, 64)
    v64 = model.predict([small[k] for k in range(B)], B)                     # (B, 3, 64^3)
    v = resample(v64.reshape(3 * B, 64, 64, 64).contiguous(), (64, 64, 64), (n, n, n), 3 * B)
    return list(v.reshape(B, 3, n, n, n))


def evaluate(model, pairs, n, beta, eps_opt=5e-2):
    """Zero-init vs warm-started solves of each pair, one pair at a time (same tolerance
    and denominator).  The warm arm's cost includes the prediction; its J(v_pred) <= J(0)
    test runs inside the solve (options.warm_check)."""
    import torch
    res = []
    for m0, m1 in pairs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v0 = _predict_batch(model, [(m0, m1)], n)[0].clone()
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t0
        with C.Context((n, n, n), nt=4, beta_v=beta, eps_opt=eps_opt, precond=PRECOND,
                       max_inner=MAX_INNER) as ctx:
            ctx.set_images(m0, m1)
            z = torch.zeros((3, n, n, n), device="cuda")
            # |g(0)| is shared by both arms (the same stopping test); the relative
            # gradient at the prediction is a diagnostic (outside the timings)
            _, g0 = ctx.objective_gradient(z)
            gnorm0 = float(g0.abs().max())
            ctx.set_options(gnorm0=gnorm0)
            _, gp = ctx.objective_gradient(v0)
            grad_rel_pred = float(gp.abs().max()) / gnorm0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vz, sz = ctx.solve(torch.zeros_like(z))
            torch.cuda.synchronize()
            tz = time.perf_counter() - t0
            # the representation floor (diagnostic): the zero-init solution restricted to
            # 64^3 and prolonged back, as the network's output is
            vr = resample(resample(vz.contiguous(), (n, n, n), (64, 64, 64), 3).contiguous(),
                          (64, 64, 64), (n, n, n), 3).contiguous()
            _, gr = ctx.objective_gradient(vr)
            grad_rel_floor = float(gr.abs().max()) / gnorm0
            ctx.set_options(warm_check=1)
            t0 = time.perf_counter()
            vw, sw = ctx.solve(v0)
            torch.cuda.synchronize()
            tw = time.perf_counter() - t0 + t_pred      # the prediction is part of the cost
        res.append({"t_zero": tz, "t_warm": tw, "t_predict": t_pred, "matvecs_zero": sz.matvecs,
                    "matvecs_warm": sw.matvecs, "newton_zero": sz.newton_iters,
                    "newton_warm": sw.newton_iters, "grad_rel_zero": sz.grad_rel,
                    "grad_rel_warm": sw.grad_rel, "mismatch_zero": sz.mismatch_rel,
                    "mismatch_warm": sw.mismatch_rel, "fallback": bool(sw.warm_fallback),
                    "grad_rel_pred": grad_rel_pred, "grad_rel_floor": grad_rel_floor})
    return res


def combined_chunks(npairs, batch):
    """Index chunks of the combined arm: batch / 8 and batch / 2 pairs, then
    `batch` pairs at a time (the last chunk takes the rest)."""
    sizes, out, k = [max(1, batch // 8), max(1, batch // 2)], [], 0
    while k < npairs:
        m = min(sizes.pop(0) if sizes else batch, npairs - k)
        out.append(list(range(k, k + m)))
        k += m
    return out


def evaluate_combined(model, pairs, n, beta, eps_opt=5e-2, batch=16):
    """The plain method against the combined form on the same pairs.

    plain:    FP32 storage, zero initial guess, one pair after the other;
    combined: mixed precision (FP16 field storage), U-Net warm start with the
              J(v_pred) <= J(0) fallback inside the solver (options.warm_check), and
              the pairs solved up to `batch` at a time by claire_solve_batch with
              graph-captured PCG iterations; the prediction of the next chunk runs
              on a side stream while the current chunk is solved.  The chunks ramp
              up (batch / 8, batch / 2, then batch pairs, `combined_chunks`), so
              only the first, small chunk's prediction is not hidden behind solves:
              a pair's prediction costs a fraction of its solve.
    Both arms stop at the same relative gradient with the same denominator
    |g(0)|_inf (from an FP32 evaluation at v = 0).  Context creation, one untimed
    set-up solve, one untimed prediction per chunk size (cuFFT plans) and g(0)
    are outside both timings; both arms reuse their contexts
    and load each pair's images (set_images) inside their timings (one context for
    the plain arm, `batch` for the combined one), and the combined time is the
    wall time from the first prediction to the last solve."""
    import torch
    opts = dict(nt=4, beta_v=beta, eps_opt=eps_opt, precond=PRECOND, max_inner=MAX_INNER)
    res = {k: [] for k in ("matvecs_plain", "matvecs_combined", "mismatch_plain",
                           "mismatch_combined", "grad_rel_plain", "grad_rel_combined")}
    zeros = lambda: torch.zeros((3, n, n, n), device="cuda")
    # plain arm (one context, set up by an untimed solve of the first pair), and the
    # shared denominators
    gnorm0s, t_plain = [], 0.0
    with C.Context((n, n, n), **opts) as cp:
        cp.set_images(*pairs[0])
        cp.solve(zeros())
        for (m0, m1) in pairs:                       # the denominators, untimed
            cp.set_images(m0, m1)
            _, g0 = cp.objective_gradient(zeros())
            gnorm0s.append(float(g0.abs().max()))
        for (m0, m1), gn0 in zip(pairs, gnorm0s):
            v0 = zeros()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cp.set_images(m0, m1)
            cp.set_options(gnorm0=gn0)
            _, st = cp.solve(v0)
            torch.cuda.synchronize()
            t_plain += time.perf_counter() - t0
            res["matvecs_plain"].append(st.matvecs)
            res["mismatch_plain"].append(st.mismatch_rel)
            res["grad_rel_plain"].append(st.grad_rel)
    # combined arm: a pool of `batch` contexts (workspace, cuFFT plans and captured
    # graphs set up once, outside the timing, by one untimed zero-initialised solve
    # of the first batch), then the timed pipeline over all pairs
    chunks = combined_chunks(len(pairs), batch)
    width = max(len(c) for c in chunks)
    pool = [C.Context((n, n, n), precision=1, graphs=1, warm_check=1, **opts)
            for _ in range(width)]

    def load(idx):
        for i, cc in zip(idx, pool):
            cc.set_images(*pairs[i])
            cc.set_options(gnorm0=gnorm0s[i])      # host-side option: graphs are kept
        return pool[:len(idx)]

    C.solve_batch(load(list(range(width))), [zeros() for _ in range(width)])
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    # set-up, untimed: the resampling plans are cached per stream and batch size, so
    # each chunk size is predicted once on the side stream first; then the
    # diagnostic prediction of one full chunk on its own
    with torch.cuda.stream(side):
        for size in sorted(set(len(c) for c in chunks)):
            _predict_batch(model, [pairs[i] for i in range(size)], n)
    torch.cuda.synchronize()
    tp = time.perf_counter()
    with torch.cuda.stream(side):
        _predict_batch(model, [pairs[i] for i in range(width)], n)
    torch.cuda.synchronize()
    t_pred_pair = (time.perf_counter() - tp) / width

    def predict(idx):
        side.wait_stream(main)
        with torch.cuda.stream(side):
            v0s = [v.clone() for v in _predict_batch(model, [pairs[i] for i in idx], n)]
            ev = side.record_event()
        return v0s, ev

    fallbacks = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nxt = predict(chunks[0])
    for k, idx in enumerate(chunks):
        v0s, ev = nxt
        main.wait_event(ev)
        if k + 1 < len(chunks):
            nxt = predict(chunks[k + 1])           # overlaps the solves of this chunk
        _, stats = C.solve_batch(load(idx), v0s)
        for st in stats:
            res["matvecs_combined"].append(st.matvecs)
            res["mismatch_combined"].append(st.mismatch_rel)
            res["grad_rel_combined"].append(st.grad_rel)
            fallbacks += st.warm_fallback
    torch.cuda.synchronize()
    t_comb = time.perf_counter() - t0
    for c in pool:
        c.close()
    npairs = len(pairs)
    summ = {"pairs": npairs, "batch": batch, "chunks": [len(c) for c in chunks],
            "t_plain_per_pair": t_plain / npairs,
            "t_combined_per_pair": t_comb / npairs, "speedup": t_plain / t_comb,
            "t_prediction_per_pair": t_pred_pair, "fallbacks": fallbacks}
    for k in ("matvecs", "mismatch", "grad_rel"):
        for arm in ("plain", "combined"):
            summ[f"mean_{k}_{arm}"] = float(np.mean(res[f"{k}_{arm}"]))
    summ["max_grad_rel"] = float(max(res["grad_rel_plain"] + res["grad_rel_combined"]))
    return summ


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--beta", type=float, default=1e-2)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--batch", type=int, default=4, help="training samples per Adam step")
    ap.add_argument("--warmup", type=int, default=250, help="linear learning-rate warm-up steps")
    ap.add_argument("--augment", type=int, default=0, choices=[0, 1],
                    help="relabel training samples by random symmetries of the cube")
    ap.add_argument("--precond", type=int, default=PRECOND,
                    help="registration preconditioner: 0 spectral, 1 two-level")
    ap.add_argument("--combined-batch", default="16",
                    help="comma-separated pairs per concurrent batch of the plain-vs-combined "
                         "comparison (0 skips it)")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    globals()["PRECOND"] = args.precond
    from paper_2401_17493_b300 import build
    build.build()
    n = args.n
    t_start = time.perf_counter()
    log = lambda m: print(f"[{time.perf_counter() - t_start:7.1f}s] {m}", flush=True)
    train_seeds = list(range(10000, 10000 + args.train))
    eval_seeds = list(range(20000, 20000 + args.eval))
    inputs, targets = [], []
    chunk = 64
    for i in range(0, len(train_seeds), chunk):
        pairs = make_pairs(train_seeds[i:i + chunk], n)
        vs = solve_targets(pairs, n, args.beta)
        for (m0, m1), v in zip(pairs, vs):
            inputs.append(resample(torch.stack([m0, m1]).contiguous(), (n,) * 3, (64,) * 3, 2))
            targets.append(resample(v.contiguous(), (n,) * 3, (64,) * 3, 3))
        del pairs, vs
    log(f"{len(inputs)} training pairs solved and restricted")
    model = UNet3D(seed=0)
    log(f"U-Net parameters: {model.parameters}")
    t0 = time.perf_counter()
    hist = train(model, inputs, targets, args.epochs, lr=args.lr, batch=args.batch, log=log,
                 warmup=args.warmup, augment=bool(args.augment))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = evaluate(model, make_pairs(eval_seeds, n), n, args.beta)
    summary = {
        "train_pairs": len(inputs), "eval_pairs": len(res), "epochs": args.epochs,
        "train_seconds": t_train, "loss_history": hist, "parameters": model.parameters,
        "grid": n, "beta_v": args.beta,
        "mean_t_zero": float(np.mean([r["t_zero"] for r in res])),
        "mean_t_warm": float(np.mean([r["t_warm"] for r in res])),
        "mean_matvecs_zero": float(np.mean([r["matvecs_zero"] for r in res])),
        "mean_matvecs_warm": float(np.mean([r["matvecs_warm"] for r in res])),
        "mean_mismatch_zero": float(np.mean([r["mismatch_zero"] for r in res])),
        "mean_mismatch_warm": float(np.mean([r["mismatch_warm"] for r in res])),
        "fallbacks": int(sum(r["fallback"] for r in res)),
        "median_grad_rel_pred": float(np.median([r["grad_rel_pred"] for r in res])),
        "frac_pred_within_tol": float(np.mean([r["grad_rel_pred"] <= 5e-2 for r in res])),
        "median_grad_rel_floor": float(np.median([r["grad_rel_floor"] for r in res])),
        "all_converged": bool(all(r["grad_rel_zero"] <= 5e-2 and r["grad_rel_warm"] <= 5e-2
                                  for r in res)),
    }
    summary["speedup_time"] = summary["mean_t_zero"] / summary["mean_t_warm"]
    summary["speedup_matvecs"] = summary["mean_matvecs_zero"] / max(1e-9, summary["mean_matvecs_warm"])
    log(json.dumps(summary))
    summary["combined"] = []
    for b in (int(x) for x in args.combined_batch.split(",")):
        if b > 0:
            summary["combined"].append(evaluate_combined(model, make_pairs(eval_seeds, n), n,
                                                         args.beta, batch=b))
            log("plain vs combined: " + json.dumps(summary["combined"][-1]))
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"summary": summary, "pairs": res}, f, indent=1)


if __name__ == "__main__":
    main()
