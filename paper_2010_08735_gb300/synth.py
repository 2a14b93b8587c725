"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and fills plain dictionaries; it holds none
of the rendering arithmetic, so that both the CUDA library and the CPU oracle
can be fed the same inputs without sharing code.

Recipe (stands in for the Gaia DR2 / Tycho-2 catalogues and for the paper's
unspecified Fig. 1 views, which are not available):

* stars: directions uniform on the sphere (normalised Gaussian triples);
  luminosity L = X+Y+Z with density proportional to L^-1.5 on [1, 1e4]
  (inverse CDF); black-body temperature log-uniform on [3000, 30000] K;
  numpy PCG64 with the given seed.
* cameras: the five workloads below, with the default orientation looking at
  the hole, +z up (e_w, e_h, e_d) = (e'_phi, -e'_theta, e'_r).
"""
from __future__ import annotations

import math

import numpy as np

DEG = math.pi / 180.0
DEFAULT_ORIENT = ((0.0, 0.0, 1.0), (0.0, -1.0, 0.0), (1.0, 0.0, 0.0))


def stars(n: int, seed: int = 0) -> np.ndarray:
    """(n, 5) float32: unit direction x, y, z; luminosity; temperature (K)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    F = rng.random(n)
    lum = (1.0 - F * (1.0 - 1e-2)) ** -2.0  # pdf ~ L^-1.5 on [1, 1e4]
    temp = 3000.0 * 10.0 ** rng.random(n)   # log-uniform [3000, 30000] K
    out = np.empty((n, 5), dtype=np.float32)
    out[:, 0:3] = d
    out[:, 3] = lum
    out[:, 4] = temp
    return out


def camera(r, theta_deg, phi_deg=0.0, v=(0.0, 0.0, 0.0), width=256, height=256, fov_deg=60.0,
           orient=DEFAULT_ORIENT) -> dict:
    return {"r": float(r), "theta": theta_deg * DEG, "phi": phi_deg * DEG,
            "v": tuple(float(x) for x in v),
            "orient": tuple(tuple(float(x) for x in row) for row in orient),
            "fov_y": fov_deg * DEG, "width": int(width), "height": int(height)}


def disc(r_in=3.0, r_out=12.0, t_peak=1e4, density=0.5, enabled=True) -> dict:
    return {"r_in": float(r_in), "r_out": float(r_out), "t_peak": float(t_peak),
            "density": float(density), "enabled": bool(enabled)}


def disc_particles(n=16, seed=5, r_in=3.0, r_out=12.0) -> np.ndarray:
    """Linear particles of the animated disc (Appendix B), (n, 3) float64 rows
    (u1, u2, phi0): mean radius uniform on [r_in + 1/2, r_out - 1/2],
    eccentricity uniform on [0, 0.05] (u1, u2 = ubar (1 -+ ecc)), phase uniform
    on [0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rbar = rng.uniform(r_in + 0.5, r_out - 0.5, n)
    ecc = rng.uniform(0.0, 0.05, n)
    phi0 = rng.uniform(0.0, 2.0 * np.pi, n)
    ub = 1.0 / rbar
    return np.stack([ub * (1.0 - ecc), ub * (1.0 + ecc), phi0], axis=1)


# The five workloads: 256^2 static; 1080p orbiting at 0.5c; 4K infalling at
# 0.9c; a 64-camera batch; 256 served viewers.
WORKLOADS = {
    "static_256": dict(camera=camera(10.0, 80.0, width=256, height=256), disc=disc(3.0, 12.0),
                       n_stars=1000, star_seed=0, cube_n=2048, cube_dtype="f16"),
    "orbit_1080p": dict(camera=camera(6.0, 85.0, v=(0.0, 0.0, 0.5), width=1920, height=1080),
                        disc=disc(3.0, 12.0), n_stars=1_000_000, star_seed=0, cube_n=2048,
                        cube_dtype="f16"),
    "infall_4k": dict(camera=camera(3.2, 89.0, v=(-0.9, 0.0, 0.0), width=3840, height=2160),
                      disc=disc(3.0, 20.0), n_stars=4_000_000, star_seed=0, cube_n=4096,
                      cube_dtype="bf16"),
}

BATCH_RESOLUTIONS = ((320, 240), (640, 480), (1280, 720), (1920, 1080))


def random_rotation(rng) -> np.ndarray:
    """Uniform rotation (QR of a Gaussian matrix with the sign fixed)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def batch_cameras(n: int = 64, seed: int = 1, resolutions=BATCH_RESOLUTIONS) -> list[dict]:
    """Cameras of the batched workload: resolution uniform over the list,
    r ~ U[2.5, 50], position direction uniform on the sphere, speed
    ~ U[0, 0.9] with a uniform direction, orientation uniform on SO(3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cams = []
    for _ in range(n):
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        r = rng.uniform(2.5, 50.0)
        th = math.acos(1.0 - 2.0 * rng.random())
        ph = 2.0 * math.pi * rng.random()
        vd = rng.standard_normal(3)
        vd /= np.linalg.norm(vd)
        v = vd * rng.uniform(0.0, 0.9)
        o = random_rotation(rng)
        cams.append({"r": float(r), "theta": th, "phi": ph, "v": tuple(float(x) for x in v),
                     "orient": tuple(tuple(float(x) for x in row) for row in o),
                     "fov_y": 60.0 * DEG, "width": int(w), "height": int(h)})
    return cams


SERVE_RESOLUTIONS = ((1280, 720), (1920, 1080), (3840, 2160))


def viewer_traffic(n_viewers: int = 256, seed: int = 4, rate_hz: float = 60.0,
                   duration_s: float = 1.0, resolutions=SERVE_RESOLUTIONS) -> dict:
    """Served workload: per-viewer resolution, trajectory parameters and
    Poisson request times (exponential gaps at rate_hz)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    viewers = []
    for vid in range(n_viewers):
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        kind = "circular" if rng.random() < 0.5 else "radial"
        viewers.append({"id": vid, "width": int(w), "height": int(h), "kind": kind,
                        "r0": float(rng.uniform(4.0, 30.0)),
                        "theta": float(rng.uniform(60.0, 120.0) * DEG),
                        "phi0": float(rng.uniform(0.0, 2.0 * math.pi)),
                        "speed": float(rng.uniform(0.05, 0.6))})
    events = []
    for vid in range(n_viewers):
        t = rng.exponential(1.0 / rate_hz)
        while t < duration_s:
            events.append((t, vid))
            t += rng.exponential(1.0 / rate_hz)
    events.sort()
    return {"viewers": viewers, "events": events}
