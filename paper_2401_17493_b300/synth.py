"""Seeded synthetic inputs: phantoms and band-limited velocities.

These generators stand in for the NIREP brain MRI pairs (256 x 300 x 256, T1)
that the paper registers; they reproduce the size class and smooth intensity
classes in [0, 1] of that workload.  They hold none of the registration
method's arithmetic: the reference image m1 is the analytic phantom evaluated
at warped coordinates x - u(x) (u a seeded band-limited displacement), not a
numerical transport of m0.  Both the CUDA path and the CPU oracle receive the
same float32 arrays from here.

RNG: numpy PCG64 (``np.random.default_rng(seed)``).  All coordinates are in
voxel units on the periodic grid [0, n_i).
"""

import math

import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def _wrap(d, n):
    """Periodic difference in (-n/2, n/2]."""
    return d - n * np.round(d / n)


def bandlimited_field(shape, kmax, rng, ncomp=3):
    """Real random field(s) with Hermitian Fourier coefficients supported on |k| <= kmax."""
    n1, n2, n3 = shape
    k1 = np.fft.fftfreq(n1, 1.0 / n1)[:, None, None]
    k2 = np.fft.fftfreq(n2, 1.0 / n2)[None, :, None]
    k3 = np.arange(n3 // 2 + 1, dtype=np.float64)[None, None, :]
    mask = (k1 ** 2 + k2 ** 2 + k3 ** 2) <= kmax ** 2
    out = []
    for _ in range(ncomp):
        coef = (rng.standard_normal(mask.shape) + 1j * rng.standard_normal(mask.shape)) * mask
        out.append(np.fft.irfftn(coef, s=shape, axes=(0, 1, 2)))   # Hermitian by construction
    return np.stack(out)


def bandlimited_velocity(shape, kmax, max_disp_voxels, seed):
    """Velocity (3, n1, n2, n3) in physical units with max |v| / h = max_disp_voxels."""
    rng = _rng(seed)
    u_vox = bandlimited_field(shape, kmax, rng, 3)     # read as a displacement in voxels
    u_vox *= max_disp_voxels / np.max(np.sqrt(np.sum(u_vox ** 2, axis=0)))
    h = np.array([2.0 * np.pi / n for n in shape])
    return u_vox * h[:, None, None, None]


def solenoidal_velocity(shape, kmax, max_disp_voxels, seed):
    """Divergence-free velocity: spectral curl of a band-limited vector potential."""
    rng = _rng(seed)
    psi = bandlimited_field(shape, kmax, rng, 3)
    n1, n2, n3 = shape
    k = [np.fft.fftfreq(n1, 1.0 / n1)[:, None, None],
         np.fft.fftfreq(n2, 1.0 / n2)[None, :, None],
         np.fft.rfftfreq(n3, 1.0 / n3)[None, None, :]]
    P = [np.fft.rfftn(psi[a]) for a in range(3)]
    curl = [1j * (k[1] * P[2] - k[2] * P[1]),
            1j * (k[2] * P[0] - k[0] * P[2]),
            1j * (k[0] * P[1] - k[1] * P[0])]
    v = np.stack([np.fft.irfftn(c, s=shape, axes=(0, 1, 2)) for c in curl])
    h = np.array([2.0 * np.pi / n for n in shape])
    vox = v / h[:, None, None, None]
    v *= max_disp_voxels / np.max(np.sqrt(np.sum(vox ** 2, axis=0)))
    return v


def _voxel_grid(shape):
    return np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")


# ----------------------------------------------------------------- blob phantom

def blob_params(shape, seed, nblobs=20, sigma=(3.0, 8.0), amp=(0.2, 1.0)):
    rng = _rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(nblobs, 3)) * np.array(shape, dtype=np.float64)
    sig = rng.uniform(sigma[0], sigma[1], size=nblobs)
    a = rng.uniform(amp[0], amp[1], size=nblobs)
    return centres, sig, a


def blob_image(params, shape, coords):
    """Sum of periodic Gaussian blobs evaluated at voxel coordinates (3 arrays)."""
    centres, sig, a = params
    out = np.zeros(coords[0].shape)
    for c, s, A in zip(centres, sig, a):
        r2 = sum(_wrap(coords[i] - c[i], shape[i]) ** 2 for i in range(3))
        out += A * np.exp(-0.5 * r2 / (s * s))
    return out


def blob_pair(shape=(64, 64, 64), seed=1, kmax=4, max_disp_voxels=3.0):
    """Template m0, reference m1 and the generating velocity (parity workload).

    m0: 20 periodic Gaussian blobs (sigma U[3, 8] voxels, amplitude U[0.2, 1],
    centres U[0, n)), min-max normalised to [0, 1].  v: random Fourier
    coefficients on |k| <= 4 scaled to max |v| / h = 3 voxels.  m1: the same
    blobs evaluated at x - v(x) (voxel units) with m0's normalisation.
    """
    params = blob_params(shape, seed)
    x = _voxel_grid(shape)
    raw0 = blob_image(params, shape, x)
    v = bandlimited_velocity(shape, kmax, max_disp_voxels, seed + 7919)
    h = [2.0 * np.pi / n for n in shape]
    xw = [x[i] - v[i] / h[i] for i in range(3)]
    raw1 = blob_image(params, shape, xw)
    lo, hi = raw0.min(), raw0.max()
    m0 = (raw0 - lo) / (hi - lo)
    m1 = (raw1 - lo) / (hi - lo)
    return m0.astype(np.float32), m1.astype(np.float32), v.astype(np.float32)


# ------------------------------------------------------------ ellipsoid phantom

def ellipsoid_params(shape, seed):
    rng = _rng(seed)
    n = np.array(shape, dtype=np.float64)
    centre = n / 2.0 + rng.uniform(-0.03, 0.03, size=3) * n
    outer = rng.uniform(0.6, 0.85, size=3) * n / 2.0
    middle = outer * rng.uniform(0.68, 0.78, size=3)
    core = outer * rng.uniform(0.38, 0.48, size=3)
    return centre, (outer, middle, core), (0.3, 0.6, 0.9)


def ellipsoid_image(params, shape, coords, edge_voxels=2.0):
    """Nested ellipsoids with smooth tanh edges: shell 0.3, middle 0.6, core 0.9."""
    centre, axes, levels = params
    d = [_wrap(coords[i] - centre[i], shape[i]) for i in range(3)]
    out = np.zeros(coords[0].shape)
    prev = 0.0
    for ax, lev in zip(axes, levels):
        rho = np.sqrt(sum((d[i] / ax[i]) ** 2 for i in range(3)))
        dist = (rho - 1.0) * float(np.mean(ax))        # approx. signed distance in voxels
        inside = 0.5 * (1.0 - np.tanh(dist / edge_voxels))
        out += (lev - prev) * inside
        prev = lev
    return out


def gaussian_smooth(u, sigma_voxels):
    """Periodic Gaussian smoothing via FFT (input preparation only)."""
    shape = u.shape
    k = [np.fft.fftfreq(shape[0])[:, None, None], np.fft.fftfreq(shape[1])[None, :, None],
         np.fft.rfftfreq(shape[2])[None, None, :]]
    g = np.exp(-2.0 * (np.pi * sigma_voxels) ** 2 * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2))
    return np.fft.irfftn(np.fft.rfftn(u) * g, s=shape, axes=(0, 1, 2))


def ellipsoid_pair(shape=(256, 256, 256), seed=2, kmax=8, max_disp_voxels=4.0,
                   noise=0.02, smooth_voxels=1.0):
    """Brain-like phantom pair (headline workload).

    Three nested ellipsoids (intensities 0.3 / 0.6 / 0.9, tanh edges of 2
    voxels, outer semi-axes U[0.6, 0.85] n/2 with seeded jitter), Gaussian
    noise N(0, 0.02^2), periodic Gaussian smoothing sigma = 1 voxel.  m1 is the
    phantom at x - u(x), u a seeded |k| <= 8 displacement with max 4 voxels,
    with its own noise draw.  Returns float32 (m0, m1, u as a velocity).
    """
    rng = _rng(seed)
    params = ellipsoid_params(shape, seed)
    v = bandlimited_velocity(shape, kmax, max_disp_voxels, seed + 7919)
    h = [2.0 * np.pi / n for n in shape]
    out = []
    for warp in (False, True):
        x = _voxel_grid(shape)
        if warp:
            x = [x[i] - v[i] / h[i] for i in range(3)]
        img = ellipsoid_image(params, shape, x)
        img = img + noise * rng.standard_normal(shape)
        img = gaussian_smooth(img, smooth_voxels)
        out.append(img.astype(np.float32))
        del x, img
    return out[0], out[1], v.astype(np.float32)


def smooth_field(shape, kmax, seed, amplitude=1.0):
    """A band-limited scalar field (for operator-level tests)."""
    f = bandlimited_field(shape, kmax, _rng(seed), 1)[0]
    return (amplitude * f / np.max(np.abs(f))).astype(np.float64)


# ------------------------------------------------ GPU generator (torch)

def ellipsoid_pair_torch(shape, seed, kmax=8, max_disp_voxels=4.0, noise=0.02,
                         smooth_voxels=1.0, device="cuda"):
    """The ellipsoid phantom pair of ellipsoid_pair, evaluated on the GPU.

    Same formulas; the ellipsoid parameters come from numpy's PCG64 with
    `seed`, the noise and the band-limited displacement from a torch
    generator seeded with `seed` (so the arrays differ from ellipsoid_pair's
    for the same seed, but the family is the same).  For large seeded data
    sets (training pairs of the learned warm start).  Returns float32 CUDA
    tensors (m0, m1).
    """
    import torch
    gen = torch.Generator(device=device).manual_seed(int(seed))
    n = torch.tensor(shape, dtype=torch.float64)
    centre, axes, levels = ellipsoid_params(shape, seed)
    n1, n2, n3 = shape
    # band-limited displacement (voxel units), max norm max_disp_voxels
    k1 = torch.fft.fftfreq(n1, 1.0 / n1, device=device)[:, None, None]
    k2 = torch.fft.fftfreq(n2, 1.0 / n2, device=device)[None, :, None]
    k3 = torch.arange(n3 // 2 + 1, device=device, dtype=torch.float32)[None, None, :]
    mask = (k1 ** 2 + k2 ** 2 + k3 ** 2) <= kmax ** 2
    u = []
    for _ in range(3):
        re = torch.randn(mask.shape, generator=gen, device=device)
        im = torch.randn(mask.shape, generator=gen, device=device)
        u.append(torch.fft.irfftn(torch.complex(re, im) * mask, s=shape, dim=(0, 1, 2)))
    u = torch.stack(u)
    u *= max_disp_voxels / torch.sqrt((u ** 2).sum(0)).max()
    grid = torch.meshgrid(*[torch.arange(m, device=device, dtype=torch.float32) for m in shape],
                          indexing="ij")
    kf = [torch.fft.fftfreq(n1, device=device)[:, None, None],
          torch.fft.fftfreq(n2, device=device)[None, :, None],
          torch.fft.rfftfreq(n3, device=device)[None, None, :]]
    gauss = torch.exp(-2.0 * (math.pi * smooth_voxels) ** 2 * (kf[0] ** 2 + kf[1] ** 2 + kf[2] ** 2))
    out = []
    for warp in (False, True):
        x = [grid[i] - u[i] if warp else grid[i] for i in range(3)]
        d = []
        for i in range(3):
            di = x[i] - float(centre[i])
            d.append(di - shape[i] * torch.round(di / shape[i]))
        img = torch.zeros(shape, device=device)
        prev = 0.0
        for ax, lev in zip(axes, levels):
            rho = torch.sqrt(sum((d[i] / float(ax[i])) ** 2 for i in range(3)))
            dist = (rho - 1.0) * float(np.mean(ax))
            img += (lev - prev) * 0.5 * (1.0 - torch.tanh(dist / 2.0))
            prev = lev
        img += noise * torch.randn(shape, generator=gen, device=device)
        img = torch.fft.irfftn(torch.fft.rfftn(img) * gauss, s=shape, dim=(0, 1, 2))
        out.append(img.float().contiguous())
    del n
    return out[0], out[1]
