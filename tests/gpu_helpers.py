"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
binding and the CPU oracle on the same seeded inputs, and compare them."""
from __future__ import annotations

import os

import numpy as np

# tolerances (linear RGB, star positions, hit radius, tables)
RGB_MEAN_REL = 1e-3
RGB_MAX_REL = 1e-2
HIT_U_REL = 1e-3
TABLE_REL = 1e-6


def image_error(gpu: np.ndarray, orc: np.ndarray, mask: np.ndarray):
    """Per-pixel relative error of linear RGB (reading C19): the denominator is
    max(|ref|, 1e-4 * max over the image of |ref|).  Returns (mean, max, per-pixel)."""
    g = gpu[..., :3].astype(np.float64)
    o = orc[..., :3]
    floor = 1e-4 * max(np.abs(o).max(), 1e-30)
    rel = (np.abs(g - o) / np.maximum(np.abs(o), floor)).max(axis=-1)
    sel = rel[~mask]
    if sel.size == 0:
        return 0.0, 0.0, rel
    return float(sel.mean()), float(sel.max()), rel


def dilate(m: np.ndarray, r: int = 1) -> np.ndarray:
    out = m.copy()
    H, W = m.shape
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            sh = np.zeros_like(m)
            ys, yd = (slice(max(dy, 0), H), slice(0, H - max(dy, 0))) if dy >= 0 else (
                slice(0, H + dy), slice(-dy, H))
            xs, xd = (slice(max(dx, 0), W), slice(0, W - max(dx, 0))) if dx >= 0 else (
                slice(0, W + dx), slice(-dx, W))
            sh[yd, xd] = m[ys, xs]
            out |= sh
    return out


def mask_parts(dbg: np.ndarray, level_margin=0.02, face_margin=2e-3) -> dict:
    """The groups of pixels excluded from the comparison, from the oracle's
    values only: within 1 px of a change of disc-hit count or of the capture
    state (disc edges, shadow silhouette: the mask the tolerance names), and
    pixels whose mip-level or cube-face decision lies within a small margin of
    its threshold, or whose footprint Jacobian is degenerate (discontinuities
    of the method, where FP32 and FP64 may take either side)."""
    cap = ~np.isfinite(dbg[..., 2])
    hits = dbg[..., 3]
    edge = np.zeros(cap.shape, dtype=bool)
    for a in (cap, hits):
        e = np.zeros(cap.shape, dtype=bool)
        e[:, 1:] |= a[:, 1:] != a[:, :-1]
        e[:, :-1] |= a[:, 1:] != a[:, :-1]
        e[1:, :] |= a[1:, :] != a[:-1, :]
        e[:-1, :] |= a[1:, :] != a[:-1, :]
        edge |= e
    lvl = dbg[..., 6]
    hm = dbg[..., 16]
    has = lvl >= 0
    ratio = np.where(has, 2 * hm / (8 * 2.0 ** np.maximum(lvl, 0)), 0.0)
    near_up = has & (ratio > 1 - level_margin) & (ratio <= 1)
    prev = np.where(has & (lvl > 0), 2 * hm / (8 * 2.0 ** np.maximum(lvl - 1, 0)), 0.0)
    near_dn = has & (lvl > 0) & (prev < 1 + level_margin)
    return {"edge": dilate(edge, 1), "level_margin": near_up | near_dn,
            "face_margin": has & (dbg[..., 17] < face_margin),
            "degenerate": has & (dbg[..., 18] < 1e-5)}


def oracle_mask(dbg: np.ndarray, level_margin=0.02, face_margin=2e-3) -> np.ndarray:
    """Union of mask_parts: the pixels excluded from the comparison."""
    m = np.zeros(dbg.shape[:2], dtype=bool)
    for v in mask_parts(dbg, level_margin, face_margin).values():
        m |= v
    return m


# Bounds on the share of an image each excluded group may take: the mask
# must stay a thin set (edges and decision thresholds), never a region.  A
# +-2 % band around every mip-level threshold covers 2 x log2(1.02) = 5.7 %
# of the pixels when log2 of the footprint is spread evenly over the image.
MASK_BOUNDS = {"edge": 0.30, "level_margin": 0.08, "face_margin": 0.01, "degenerate": 0.01,
               "ill_conditioned": 0.10}


def mask_report(name: str, dbg: np.ndarray, orc: np.ndarray, cam: dict) -> dict:
    """Share of the image in each excluded group (printed, and bounded by
    MASK_BOUNDS)."""
    parts = mask_parts(dbg)
    rep = {k: float(v.mean()) for k, v in parts.items()}
    rep["ill_conditioned"] = float((star_ill_conditioned(dbg, orc, cam) & ~oracle_mask(dbg)).mean())
    print(f"MASK {name} {cam['width']}x{cam['height']}: " +
          " ".join(f"{k}={v:.4f}" for k, v in rep.items()))
    if cam["width"] * cam["height"] >= 4096:  # tiny test images are mostly edge
        for k, v in rep.items():
            assert v <= MASK_BOUNDS[k], (name, k, v)
    return rep


# FP32 places a beam's escape direction to a few float ulps of the angle,
# about 1e-6 rad.  In screen pixels of footprint shift that is
# 1e-6 * sqrt(Omega/Omega') / (pixel angle): about 1e-3 px for a 4K pixel,
# far less for a coarse image.  A pixel whose linear RGB can change by more
# than 1 % for that shift (a bright star near the edge of its tent filter,
# amplified where the XYZ -> RGB matrix cancels) is ill-conditioned for a
# per-pixel relative comparison.  The oracle reports, per channel, a bound on
# the change per pixel of shift (channels 20..22) and Omega/Omega' (8).
POS_EPS_RAD = 1e-6


def pos_eps_px(dbg: np.ndarray, cam: dict) -> np.ndarray:
    pix = cam["fov_y"] / cam["height"]
    return POS_EPS_RAD * np.sqrt(np.maximum(dbg[..., 8], 0.0)) / pix


def rgb_sensitivity(dbg: np.ndarray, orc: np.ndarray) -> np.ndarray:
    o = orc[..., :3]
    floor = 1e-4 * max(np.abs(o).max(), 1e-30)
    return (dbg[..., 20:23] / np.maximum(np.abs(o), floor)).max(axis=-1)


def star_ill_conditioned(dbg: np.ndarray, orc: np.ndarray, cam: dict) -> np.ndarray:
    return rgb_sensitivity(dbg, orc) * pos_eps_px(dbg, cam) > RGB_MAX_REL


def ill_conditioned_ok(rel: np.ndarray, dbg: np.ndarray, orc: np.ndarray, cam: dict,
                       mask_other: np.ndarray) -> bool:
    """Validity of the pixels masked only for conditioning: their error stays
    within what three times that shift explains, plus the base tolerance."""
    sel = star_ill_conditioned(dbg, orc, cam) & ~mask_other
    if not sel.any():
        return True
    bound = RGB_MAX_REL + 3 * (pos_eps_px(dbg, cam) * rgb_sensitivity(dbg, orc))[sel]
    return bool(np.all(rel[sel] <= bound))


def maybe_dump(name: str, **arrays) -> None:
    """Save arrays for offline inspection when BH_DUMP_DIR is set."""
    d = os.environ.get("BH_DUMP_DIR")
    if not d:
        return
    os.makedirs(d, exist_ok=True)
    np.savez_compressed(os.path.join(d, name + ".npz"),
                        **{k: (v.astype(np.float32) if v.dtype == np.float64 else v)
                           for k, v in arrays.items()})
