"""Lens-glare bloom (Sec. 3.4.3) in FP64 -- TEST INFRASTRUCTURE ONLY.

The plain, slow definition the CUDA bloom is checked against; only the tests
and the benchmark's CPU-baseline leg use it.  It restates the method step by
step, with no fusion:

  * point spread function: the photopic PSF of Spencer, Shirley, Zimmerman and
    Greenberg (SIGGRAPH 1995), P(theta) = 0.384 f0 + 0.478 f1 + 0.138 f2 with
    theta in degrees, f0 = 2.61e6 exp(-(theta/0.02)^2),
    f1 = 20.91/(theta+0.02)^3, f2 = 72.37/(theta+0.02)^2;
  * level weights: the PSF's energy (integral of P(theta) 2 pi theta) in the
    annulus of radii [2^(k-1/2), 2^(k+1/2)) pixels for level k >= 1 and below
    2^(1/2) pixels for level 0, over its energy below 2^(K+1/2) pixels, with the
    pixel angle fov_y / height -- integrated numerically here;
  * pyramid: D_0 = image, D_k = 2x2 box average of D_{k-1} (sizes rounded up,
    indices clamped), B_k = D_k filtered by the normalised 7-tap Gaussian of
    unit standard deviation along x then y (indices clamped);
  * output = w_0 image + sum_k w_k (B_k sampled bilinearly at the pixel
    centre, (x + 1/2)/2^k - 1/2 in level-k texels, indices clamped).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def spencer_psf(theta_deg):
    """Spencer et al.'s photopic point spread function (per square degree)."""
    t = np.asarray(theta_deg, dtype=np.float64)
    f0 = 2.61e6 * np.exp(-(t / 0.02) ** 2)
    f1 = 20.91 / (t + 0.02) ** 3
    f2 = 72.37 / (t + 0.02) ** 2
    return 0.384 * f0 + 0.478 * f1 + 0.138 * f2


def psf_energy(a_deg: float, b_deg: float) -> float:
    """Integral of P(theta) 2 pi theta dtheta from a to b degrees (adaptive
    quadrature, split where the narrow Gaussian core ends)."""
    f = lambda t: float(spencer_psf(t)) * 2.0 * math.pi * t
    pts = sorted({a_deg, b_deg} | {p for p in (0.02, 0.06, 0.2, 1.0) if a_deg < p < b_deg})
    tot = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        v, _ = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1e-12, limit=500)
        tot += v
    return tot


def bloom_weights(fov_y: float, height: int, levels: int) -> np.ndarray:
    a = math.degrees(fov_y) / height  # degrees per pixel
    edges = [0.0] + [a * 2.0 ** (k + 0.5) for k in range(levels + 1)]
    e = np.array([psf_energy(edges[k], edges[k + 1]) for k in range(levels + 1)])
    return e / e.sum()


def downsample(img: np.ndarray) -> np.ndarray:
    """2x2 box average; an odd last row/column averages with itself (clamped)."""
    h, w = img.shape[:2]
    H, W = (h + 1) // 2, (w + 1) // 2
    ys = np.minimum(np.arange(2 * H), h - 1)
    xs = np.minimum(np.arange(2 * W), w - 1)
    p = img[ys][:, xs]
    return 0.25 * (p[0::2, 0::2] + p[0::2, 1::2] + p[1::2, 0::2] + p[1::2, 1::2])


def gauss_taps() -> np.ndarray:
    t = np.exp(-0.5 * np.arange(-3, 4) ** 2)
    return t / t.sum()


def blur(img: np.ndarray) -> np.ndarray:
    """Separable 7-tap Gaussian (unit sigma) along x then y, indices clamped."""
    h, w = img.shape[:2]
    k = gauss_taps()
    out = np.zeros_like(img)
    for i, t in enumerate(range(-3, 4)):
        out += k[i] * img[:, np.clip(np.arange(w) + t, 0, w - 1)]
    res = np.zeros_like(img)
    for i, t in enumerate(range(-3, 4)):
        res += k[i] * out[np.clip(np.arange(h) + t, 0, h - 1)]
    return res


def upsample(lev: np.ndarray, k: int, H: int, W: int) -> np.ndarray:
    """Level-k image sampled bilinearly at the centres of the full-size pixels."""
    h, w = lev.shape[:2]
    s = 2.0 ** -k
    u = (np.arange(W) + 0.5) * s - 0.5
    v = (np.arange(H) + 0.5) * s - 0.5
    fu, fv = np.floor(u), np.floor(v)
    tu, tv = (u - fu)[None, :, None], (v - fv)[:, None, None]
    i0 = np.clip(fu.astype(int), 0, w - 1)
    i1 = np.clip(fu.astype(int) + 1, 0, w - 1)
    j0 = np.clip(fv.astype(int), 0, h - 1)
    j1 = np.clip(fv.astype(int) + 1, 0, h - 1)
    top = lev[j0][:, i0] * (1 - tu) + lev[j0][:, i1] * tu
    bot = lev[j1][:, i0] * (1 - tu) + lev[j1][:, i1] * tu
    return top * (1 - tv) + bot * tv


def bloom(img: np.ndarray, weights) -> np.ndarray:
    """Bloom of an (H, W, 3 or 4) linear-RGB image; returns RGB (H, W, 3)."""
    rgb = np.asarray(img, dtype=np.float64)[..., :3]
    H, W = rgb.shape[:2]
    out = weights[0] * rgb
    d = rgb
    for k in range(1, len(weights)):
        d = downsample(d)
        out = out + weights[k] * upsample(blur(d), k, H, W)
    return out
