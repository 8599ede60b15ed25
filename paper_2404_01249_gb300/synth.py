"""Seeded synthetic registration pairs (stand-ins for the paper's MRI and
microscopy data, which are not available here).

This module only draws inputs.  It holds none of the registration method's
arithmetic: image intensities are evaluated analytically at warped
coordinates (no resampling of voxel data), smooth random fields are made by
spectral filtering of white noise (numpy FFT, periodic), image blur uses
``scipy.ndimage.gaussian_filter`` and the scaling-and-squaring integration of
a velocity field uses ``scipy.ndimage.map_coordinates``.  Both the CUDA path
and the FP64 oracle consume the same arrays.

Recipes (shapes and statistics follow the workloads the paper evaluates):

* ``blobs_pair``      -- 32^3: 8 Gaussian blobs (sigma 3 vox, centres
  uniform, amplitudes U(0.5, 1)); moving = fixed evaluated at x + w(x), w a
  smoothed white-noise displacement (sigma 4) scaled to max |w| = 2 vox.
* ``voronoi_pair``    -- brain-MRI-shaped 160x192x224: 36-region random
  Voronoi partition with region means U(0.1, 1), plus N(0, 0.02) voxel noise,
  blurred with sigma 1; moving = the same partition evaluated at psi(x),
  psi = exp(v) by 7 scaling-and-squaring steps of a smoothed-noise velocity
  field (sigma 8) scaled to max |v| = 8 vox (scaled before integration), with
  its own noise draw.
* ``microscopy_pair`` -- 512x512x256: Poisson(1e-3 per voxel) cells drawn as
  Gaussian spots (sigma 1.5) with lognormal(0, 0.5) amplitudes over an
  N(0.05, 0.01) background; moving = the same cells evaluated at x + w(x),
  w smoothed noise (sigma 16) scaled to max 12 vox.
* ``uneven_shapes``   -- per-axis uniform integer sizes between 96x112x96 and
  192x224x192 for batched runs.

All arrays are float32, volumes [D, H, W], fields [3, D, H, W] (channel 0 is
the z component), in voxel units.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _grid(shape):
    D, H, W = shape
    return np.meshgrid(np.arange(D, dtype=np.float64), np.arange(H, dtype=np.float64),
                       np.arange(W, dtype=np.float64), indexing="ij")


def smooth_noise_field(shape, sigma: float, rng: np.random.Generator, channels: int = 3):
    """White noise N(0,1) per channel, low-passed by a Gaussian transfer
    function exp(-2 pi^2 sigma^2 |f|^2) in the periodic Fourier domain."""
    D, H, W = shape
    fz = np.fft.fftfreq(D)[:, None, None]
    fy = np.fft.fftfreq(H)[None, :, None]
    fx = np.fft.rfftfreq(W)[None, None, :]
    tf = np.exp(-2.0 * np.pi ** 2 * sigma ** 2 * (fz ** 2 + fy ** 2 + fx ** 2))
    out = np.empty((channels, D, H, W), dtype=np.float64)
    for c in range(channels):
        n = rng.standard_normal((D, H, W))
        out[c] = np.fft.irfftn(np.fft.rfftn(n) * tf, s=(D, H, W), axes=(0, 1, 2))
    return out


def _scale_to_max(field: np.ndarray, max_norm: float) -> np.ndarray:
    nrm = np.sqrt((field ** 2).sum(axis=0)).max()
    return field * (max_norm / nrm) if nrm > 0 else field


def blobs_pair(shape=(32, 32, 32), n_blobs=8, sigma=3.0, field_sigma=4.0, max_disp=2.0,
               seed=1000):
    """Returns (fixed, moving, w) with moving(x) = F(x + w(x))."""
    rng = _rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n_blobs, 3)) * np.asarray(shape, dtype=np.float64)
    amps = rng.uniform(0.5, 1.0, size=n_blobs)
    w = _scale_to_max(smooth_noise_field(shape, field_sigma, _rng(seed + 1000)), max_disp)

    def F(z, y, x):
        out = np.zeros_like(z)
        for c, a in zip(centres, amps):
            out += a * np.exp(-((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2)
                              / (2.0 * sigma ** 2))
        return out

    z, y, x = _grid(shape)
    fixed = F(z, y, x)
    moving = F(z + w[0], y + w[1], x + w[2])
    return fixed.astype(np.float32), moving.astype(np.float32), w.astype(np.float32)


def translated_blob_pair(shape=(24, 24, 24), shift=(0.6, -0.4, 0.8), sigma=3.5, seed=7):
    """Two blobs and their copy shifted by a constant vector: moving(x) = F(x + shift)."""
    rng = _rng(seed)
    centres = np.asarray(shape, dtype=np.float64) * rng.uniform(0.35, 0.65, size=(2, 3))
    z, y, x = _grid(shape)

    def F(z, y, x):
        out = np.zeros_like(z)
        for c in centres:
            out += np.exp(-((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2) / (2 * sigma ** 2))
        return out

    s = shift
    return (F(z, y, x).astype(np.float32), F(z + s[0], y + s[1], x + s[2]).astype(np.float32))


def _voronoi_labels(points: np.ndarray, seeds: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    """Index of the nearest seed for each point (ties to the lowest index)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(seeds)
    out = np.empty(points.shape[0], dtype=np.int64)
    for s in range(0, points.shape[0], chunk):
        _, idx = tree.query(points[s:s + chunk], k=1)
        out[s:s + chunk] = idx
    return out


def exp_svf(v: np.ndarray, steps: int) -> np.ndarray:
    """Displacement of exp(v) by scaling and squaring (u <- u + u o (id + u)),
    interpolation by scipy.ndimage.map_coordinates (order 1, nearest edge)."""
    from scipy.ndimage import map_coordinates
    shape = v.shape[1:]
    z, y, x = _grid(shape)
    u = v / float(2 ** steps)
    for _ in range(steps):
        coords = np.stack([z + u[0], y + u[1], x + u[2]])
        comp = np.stack([map_coordinates(u[c], coords, order=1, mode="nearest") for c in range(3)])
        u = u + comp
    return u


def voronoi_pair(shape=(160, 192, 224), n_regions=36, noise=0.02, blur=1.0, v_sigma=8.0,
                 max_v=8.0, ss_steps=7, seed=1000):
    """Returns (fixed, moving, psi_disp) with moving ~ fixed o psi, psi = exp(v)."""
    from scipy.ndimage import gaussian_filter
    rng = _rng(seed)
    seeds = rng.uniform(0.0, 1.0, size=(n_regions, 3)) * np.asarray(shape, dtype=np.float64)
    means = rng.uniform(0.1, 1.0, size=n_regions)
    v = _scale_to_max(smooth_noise_field(shape, v_sigma, _rng(seed + 1000)), max_v)
    psi = exp_svf(v, ss_steps)
    z, y, x = _grid(shape)
    pts = np.stack([z.ravel(), y.ravel(), x.ravel()], axis=1)
    lab_f = _voronoi_labels(pts, seeds).reshape(shape)
    wpts = np.stack([(z + psi[0]).ravel(), (y + psi[1]).ravel(), (x + psi[2]).ravel()], axis=1)
    lab_m = _voronoi_labels(wpts, seeds).reshape(shape)
    nrng = _rng(seed + 2000)
    fixed = means[lab_f] + nrng.normal(0.0, noise, size=shape)
    moving = means[lab_m] + nrng.normal(0.0, noise, size=shape)
    fixed = gaussian_filter(fixed, blur, mode="nearest")
    moving = gaussian_filter(moving, blur, mode="nearest")
    return fixed.astype(np.float32), moving.astype(np.float32), psi.astype(np.float32)


def microscopy_pair(shape=(512, 512, 256), density=1e-3, cell_sigma=1.5, field_sigma=16.0,
                    max_disp=12.0, seed=1000):
    """Returns (fixed, moving, w) with moving(x) = F(x + w(x)) (cells splatted
    analytically within 4 sigma of each centre)."""
    rng = _rng(seed)
    D, H, W = shape
    n = rng.poisson(density * D * H * W)
    centres = rng.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(shape, dtype=np.float64)
    amps = rng.lognormal(0.0, 0.5, size=n)
    w = _scale_to_max(smooth_noise_field(shape, field_sigma, _rng(seed + 1000)), max_disp)
    brng = _rng(seed + 2000)
    R = int(np.ceil(4 * cell_sigma))

    def render(disp):
        img = brng.normal(0.05, 0.01, size=shape)
        # voxel x sees F(x + disp(x)); a cell at c contributes where |x + disp - c| < R
        # (disp is smooth, so the voxels near c - disp(c) are the ones to visit)
        for c, a in zip(centres, amps):
            ci = np.clip(np.round(c).astype(int), 0, np.asarray(shape) - 1)
            off = disp[:, ci[0], ci[1], ci[2]] if disp is not None else np.zeros(3)
            base = np.round(c - off).astype(int)
            lo = np.maximum(base - R - 2, 0)
            hi = np.minimum(base + R + 3, np.asarray(shape))
            if np.any(hi <= lo):
                continue
            zz, yy, xx = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]),
                                     np.arange(lo[2], hi[2]), indexing="ij")
            pz, py, px = zz.astype(np.float64), yy.astype(np.float64), xx.astype(np.float64)
            if disp is not None:
                pz = pz + disp[0, lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
                py = py + disp[1, lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
                px = px + disp[2, lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
            r2 = (pz - c[0]) ** 2 + (py - c[1]) ** 2 + (px - c[2]) ** 2
            img[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += a * np.exp(-r2 / (2 * cell_sigma ** 2))
        return img

    fixed = render(None)
    moving = render(w)
    return fixed.astype(np.float32), moving.astype(np.float32), w.astype(np.float32)


def uneven_shapes(n=64, lo=(96, 112, 96), hi=(192, 224, 192), seed=3000):
    """n shapes, each axis an independent uniform integer in [lo_a, hi_a]."""
    rng = _rng(seed)
    return [tuple(int(rng.integers(lo[a], hi[a] + 1)) for a in range(3)) for _ in range(n)]


def random_field(shape, sigma, max_disp, seed):
    """Smooth displacement field [3, D, H, W] scaled to max |u| = max_disp."""
    return _scale_to_max(smooth_noise_field(shape, sigma, _rng(seed)), max_disp).astype(np.float32)
