"""Seeded synthetic inputs shaped like the paper's image workloads.

This module draws clean images and adds noise. It holds none of the denoiser's
arithmetic, so both the CUDA path's tests/benchmarks and the FP64 oracle can be
fed the same bytes from it.

Clean image recipe (one channel):
  * background 128;
  * 20 ellipses: centre U(0,W) x U(0,H), semi-axes U(0.05,0.4)*(W,H),
    angle U(0,pi), amplitude U(-80,80), soft edge 1/(1+exp(8(rho-1)));
  * 3 sinusoidal gratings: period U(4,16) px, angle U(0,pi), phase U(0,2pi),
    amplitude U(5,25);
  * clipped to [0,255].
RGB: channel k = 128 + sqrt(0.8)(B-128) + sqrt(0.2)(I_k-128) with B and I_k
independent single-channel draws (channel correlation 0.8), clipped.

Noise models (the paper's FM data are Poisson-Gaussian, Sec. IV-F):
  * gaussian:  y = clip(rint(x + sigma*n), 0, 255)
  * poisson_gaussian: y = clip(rint(a*Poisson(x/a) + sqrt(b)*n_k), 0, 255) with
    cross-channel correlated n_k = sqrt(0.5) n_shared + sqrt(0.5) n_k,ind.
Rounding is round-half-to-even (numpy rint).
"""
from __future__ import annotations

import numpy as np


def _gray_layer(rng: np.random.Generator, H: int, W: int) -> np.ndarray:
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.full((H, W), 128.0)
    for _ in range(20):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        ax, ay = rng.uniform(0.05, 0.4) * W, rng.uniform(0.05, 0.4) * H
        th = rng.uniform(0, np.pi)
        amp = rng.uniform(-80, 80)
        dx, dy = xx - cx, yy - cy
        u = (dx * np.cos(th) + dy * np.sin(th)) / ax
        v = (-dx * np.sin(th) + dy * np.cos(th)) / ay
        rho = np.sqrt(u * u + v * v)
        img += amp / (1.0 + np.exp(np.clip(8.0 * (rho - 1.0), -60, 60)))
    for _ in range(3):
        period = rng.uniform(4, 16)
        th = rng.uniform(0, np.pi)
        ph = rng.uniform(0, 2 * np.pi)
        amp = rng.uniform(5, 25)
        img += amp * np.sin(2 * np.pi * (xx * np.cos(th) + yy * np.sin(th)) / period + ph)
    return np.clip(img, 0, 255)


def clean_image(H: int, W: int, C: int, seed: int) -> np.ndarray:
    """Clean float64 image (H, W, C) in [0, 255]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if C == 1:
        return _gray_layer(rng, H, W)[:, :, None]
    base = _gray_layer(rng, H, W)
    chans = []
    for _ in range(C):
        ind = _gray_layer(rng, H, W)
        chans.append(128.0 + np.sqrt(0.8) * (base - 128.0) + np.sqrt(0.2) * (ind - 128.0))
    return np.clip(np.stack(chans, axis=-1), 0, 255)


def clean_cube(H: int, W: int, N: int, seed: int) -> np.ndarray:
    """Clean float64 hyperspectral cube (H, W, N) in [0, 255]: three smooth abundance maps (the
    image generator's layers, scaled to [0, 1]) mixing three smooth spectra over the N bands
    (Gaussian bumps at random centres and widths), plus a mild band-dependent offset; real
    reflectance cubes are likewise close to a few endmember spectra per pixel."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = np.arange(N, dtype=np.float64)
    cube = np.zeros((H, W, N))
    for _ in range(3):
        ab = _gray_layer(rng, H, W) / 255.0
        c, w, amp = rng.uniform(0, N), rng.uniform(0.15, 0.6) * N, rng.uniform(60, 140)
        spec = amp * np.exp(-0.5 * ((b - c) / w) ** 2)
        cube += ab[:, :, None] * spec[None, None, :]
    cube += 20.0 + 30.0 * b / max(N - 1, 1)
    return np.clip(cube, 0, 255)


def clean_volume(D: int, H: int, W: int, seed: int) -> np.ndarray:
    """Clean float64 volume (D, H, W) in [0, 255] shaped like a T1-weighted head scan: zero background,
    a soft head ellipsoid of intensity 90 holding 20 soft ellipsoids of amplitude U(-60, 80) (tissue
    compartments), plus 3 plane waves of period 6-20 voxels and amplitude 5-15 inside the head."""
    rng = np.random.Generator(np.random.PCG64(seed))
    zz, yy, xx = np.mgrid[0:D, 0:H, 0:W].astype(np.float64)

    def soft_ellipsoid(c, ax):
        rho = np.sqrt(((zz - c[0]) / ax[0]) ** 2 + ((yy - c[1]) / ax[1]) ** 2 + ((xx - c[2]) / ax[2]) ** 2)
        return 1.0 / (1.0 + np.exp(np.clip(8.0 * (rho - 1.0), -60, 60)))

    head = soft_ellipsoid((D / 2, H / 2, W / 2), (0.45 * D, 0.45 * H, 0.45 * W))
    vol = 90.0 * np.ones((D, H, W))
    for _ in range(20):
        c = (rng.uniform(0.2, 0.8) * D, rng.uniform(0.2, 0.8) * H, rng.uniform(0.2, 0.8) * W)
        ax = (rng.uniform(0.05, 0.3) * D, rng.uniform(0.05, 0.3) * H, rng.uniform(0.05, 0.3) * W)
        vol += rng.uniform(-60, 80) * soft_ellipsoid(c, ax)
    for _ in range(3):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        vol += rng.uniform(5, 15) * np.sin(2 * np.pi * (d[0] * zz + d[1] * yy + d[2] * xx) / rng.uniform(6, 20)
                                           + rng.uniform(0, 2 * np.pi))
    return np.clip(vol * head, 0, 255)


def quantize(x: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def add_gaussian(x: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return quantize(x + sigma * rng.standard_normal(x.shape))


def add_gaussian_float(x: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Unquantised float32 noisy image (for the differentiable workload)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return (x + sigma * rng.standard_normal(x.shape)).astype(np.float32)


def add_poisson_gaussian(x: np.ndarray, a: float, b: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    shot = a * rng.poisson(np.maximum(x, 0) / a)
    C = x.shape[2]
    shared = rng.standard_normal(x.shape[:2])[:, :, None]
    ind = rng.standard_normal(x.shape)
    n = np.sqrt(0.5) * shared + np.sqrt(0.5) * ind if C > 1 else ind
    return quantize(shot + np.sqrt(b) * n)


# ---- the workloads (sizes and parameters follow the configurations measured) ----

def workload_gray128(seed: int = 1001):
    """128x128 gray, Gaussian sigma=25; ps 8, stride 3, window 21, K 16, tau 2.7 sigma."""
    clean = clean_image(128, 128, 1, seed)
    noisy = add_gaussian(clean, 25.0, seed)
    params = dict(ps=8, stride=3, window=21, K=16, tau_mult=2.7)
    return quantize(clean), noisy, 25.0, params


def workload_rgb512(seed: int = 1002):
    """512x512 RGB, Poisson-Gaussian a=0.01 b=15^2; ps 8, stride 2, window 31, K 32; sigma estimated."""
    clean = clean_image(512, 512, 3, seed)
    noisy = add_poisson_gaussian(clean, 0.01, 15.0 ** 2, seed)
    params = dict(ps=8, stride=2, window=31, K=32, tau_mult=0.0)
    return quantize(clean), noisy, None, params


def workload_rgb4k(b: float = 25.0 ** 2, seed: int = 1003):
    """3840x2160 RGB, Poisson-Gaussian a=0.01, b in {10^2, 25^2, 50^2}; ps 8, stride 3, window 31, K 32."""
    clean = clean_image(2160, 3840, 3, seed)
    noisy = add_poisson_gaussian(clean, 0.01, b, seed)
    params = dict(ps=8, stride=3, window=31, K=32, tau_mult=0.0)
    return quantize(clean), noisy, float(np.sqrt(b)), params


def batch_shapes(n: int = 64, seed: int = 2000):
    """Uneven RGB sizes W~U{256..2048}, H~U{256..1536} and sigma~U(10,50)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws = rng.integers(256, 2049, size=n)
    Hs = rng.integers(256, 1537, size=n)
    sig = rng.uniform(10, 50, size=n)
    return [(int(h), int(w), float(s)) for h, w, s in zip(Hs, Ws, sig)]


def batch_image(j: int, H: int, W: int, sigma: float):
    clean = clean_image(H, W, 3, 2000 + j)
    return quantize(clean), add_gaussian(clean, sigma, 2000 + j)


def psnr(out: np.ndarray, clean_u8: np.ndarray) -> float:
    """PSNR (peak 255) of clip(out) against the clean uint8 image, all channels."""
    o = np.clip(np.asarray(out, dtype=np.float64), 0, 255)
    mse = np.mean((o - clean_u8.astype(np.float64)) ** 2)
    return float(10.0 * np.log10(255.0 ** 2 / mse))
