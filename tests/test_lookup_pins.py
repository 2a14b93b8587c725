"""Pins of the oracle's table lookups that the render path shares in
definition (not in code) with the CUDA kernel: the disc black-body table
(Sec. 3.4.2, exact black-body shift read through a 1D table in log2 T) and the
mip-level rule of the star gather (Sec. 3.3.2, "at most 9x9 texels", reading
C17).  Each is checked against an independent computation: direct Planck x
colour-matching integration, and the hand-derived footprint of a pinhole
camera in flat space.  No GPU.
"""
import math

import numpy as np
import pytest

from paper_2010_08735_gb300 import synth


# ----------------------------------------------------------------------------
# disc black-body table: ln Y, X/Y, Z/Y linear in log2 T (1024 texel centres
# over log2 T in [8, 20])
# ----------------------------------------------------------------------------

def test_disc_table_lookup_matches_planck_integral(orc):
    """The table read equals XYZ(B_T) of the direct 5 nm Planck x CMF sum within
    the linear-interpolation bound h^2/8 max|f''| (h = 12/1024 in log2 T): below
    1e-3 relative from 300 K (where ln Y curves most, Wien regime) and below
    1e-4 from 3000 K to 1e5 K.  A half-texel shift of the axis (dropping the
    texel-centre 1/2) would move the read by h/2 |d ln Y / d log2 T|, about
    1e-2 at 6000 K, and fail."""
    tab = orc.disc_colour_table(1024)
    Ts = np.exp(np.linspace(math.log(300.0), math.log(1e5), 1201))
    worst_lo = worst_hi = 0.0
    for T in Ts:
        got = orc.disc_xyz(tab, T)
        ref = orc.blackbody_xyz(T)
        rel = float(np.max(np.abs(got / ref - 1.0)))
        if T >= 3000.0:
            worst_hi = max(worst_hi, rel)
        worst_lo = max(worst_lo, rel)
    assert worst_lo < 1e-3, worst_lo
    assert worst_hi < 1e-4, worst_hi
    # the bound itself, from second differences of the exact ln Y on the table's
    # spacing, at 300 K: h^2/8 |f''| with f = ln Y(2^s)
    h = 12.0 / 1024
    s0 = math.log2(300.0)
    f = [math.log(orc.blackbody_xyz(2.0 ** (s0 + k * h))[1]) for k in (-1, 0, 1)]
    bound = h * h / 8 * abs(f[0] - 2 * f[1] + f[2]) / (h * h)
    assert 1e-4 < bound < 1e-3


def test_disc_table_lookup_clamps(orc):
    """Below 256 K the disc emits nothing; at and below the first texel centre
    the read is that texel; above the last centre, the last texel."""
    tab = orc.disc_colour_table(1024)
    assert np.all(orc.disc_xyz(tab, 255.9) == 0.0)
    assert np.all(orc.disc_xyz(tab, 0.0) == 0.0)
    first = 2.0 ** (8 + 12 * 0.5 / 1024)
    for T in (256.0, first):
        got = orc.disc_xyz(tab, T)
        Y = math.exp(tab[0, 0])
        assert got == pytest.approx([Y * tab[0, 1], Y, Y * tab[0, 2]], rel=1e-13)
    last = 2.0 ** (8 + 12 * 1023.5 / 1024)
    for T in (last, 2e6, 1e9):
        got = orc.disc_xyz(tab, T)
        Y = math.exp(tab[-1, 0])
        assert got == pytest.approx([Y * tab[-1, 1], Y, Y * tab[-1, 2]], rel=1e-13)


# ----------------------------------------------------------------------------
# mip level of the star gather (reading C17): L = smallest level with
# 2 max(h_s, h_t) <= 8 2^L, h = |J_w| + |J_h| in level-0 texels
# ----------------------------------------------------------------------------

def _flat_scene(orc, N):
    Ct, dl = orc.colour_table(8, 8, 8), orc.disc_colour_table(64)
    star = np.array([[-1.0, 0.0, 0.0, 1.0, 5000.0]], dtype=np.float32)
    rec = orc.build_cubemap(star, N, 1)
    return orc.SceneTables(np.zeros((64, 64)), np.ones((8, 8)), Ct, dl, rec, N, 1)


@pytest.mark.parametrize("k,level", [(0.7, 0), (0.98, 0), (1.02, 1), (1.5, 1), (1.98, 1),
                                     (2.02, 2), (3.0, 2), (6.0, 3)])
def test_mip_level_rule_pinhole_flat_space(orc, k, level):
    """A far static camera in flat space (zero deflection tables, r = 1e6)
    looking along -x sees face -x through a pinhole: with focal length f the
    cube coordinates are S = (q_h/f + 1) N/2, T = (-q_w/f + 1) N/2, so the quad
    derivatives (fine semantics, reading C16) give, exactly,
        J_sw = J_th = 0,  J_sh = (N/2f) n_P/n_Q(h),  J_tw = -(N/2f) n_P/n_Q(w),
    n = |(q_w, q_h, -f)| of the pixel P and of its quad neighbour Q.  With
    N/(8f) = k the half-extent is h = 4k (1 + O(1e-3)) level-0 texels; the
    expected level is the smallest L with 2h <= 8 2^L, and the visited texel
    range is [floor(c - h/2^L), floor(c + h/2^L)] in each axis, clipped."""
    N, W, H = 2048, 32, 32
    f = N / (8.0 * k)  # focal length in pixels for N/(8f) = k
    fov = 2.0 * math.atan(0.5 * H / f)
    cam = synth.camera(1e6, 90.0, width=W, height=H, fov_deg=fov / synth.DEG)
    _, dbg, _ = orc.render(cam, synth.disc(enabled=False), _flat_scene(orc, N), debug=True,
                           nthreads=2)
    # the oracle's own f; the static frame's radial axis carries sqrt(1 - u) in
    # the pseudo-Cartesian frame, which scales the view axis by sqrt(1 - 1e-6)
    f = 0.5 * H / math.tan(0.5 * cam["fov_y"]) * math.sqrt(1.0 - 1.0 / cam["r"])
    jj, ii = np.mgrid[0:H, 0:W]
    qw, qh = ii + 0.5 - W / 2, H / 2 - jj - 0.5
    n = np.sqrt(qw * qw + qh * qh + f * f)
    nq_w = np.sqrt((qw + np.where(ii % 2 == 0, 1.0, -1.0)) ** 2 + qh * qh + f * f)
    nq_h = np.sqrt(qw * qw + (qh + np.where(jj % 2 == 0, -1.0, 1.0)) ** 2 + f * f)
    hs = N / (2 * f) * n / nq_h
    ht = N / (2 * f) * n / nq_w
    hm = np.maximum(hs, ht)
    assert np.all(dbg[..., 7] == 1)                        # face -x
    assert np.allclose(dbg[..., 16], hm, rtol=1e-9)        # half-extent, level-0 texels
    exp_level = np.zeros_like(hm, dtype=int)
    for L in range(12):
        exp_level = np.where((exp_level == L) & (2 * hm > 8 * 2.0 ** L), L + 1, exp_level)
    assert np.all(exp_level == level)                      # the chosen k is unambiguous
    assert np.all(dbg[..., 6] == level)
    # visited texel range at that level
    NL = N >> level
    cS = (qh / f + 1) * N / 2 / 2 ** level
    cT = (-qw / f + 1) * N / 2 / 2 ** level
    hsL, htL = hs / 2 ** level, ht / 2 ** level
    ends = [cS - hsL, cS + hsL, cT - htL, cT + htL]
    safe = np.ones_like(hm, dtype=bool)
    for e in ends:
        safe &= np.abs(e - np.round(e)) > 1e-7
    i0 = np.clip(np.floor(cS - hsL), 0, NL - 1)
    i1 = np.clip(np.floor(cS + hsL), 0, NL - 1)
    j0 = np.clip(np.floor(cT - htL), 0, NL - 1)
    j1 = np.clip(np.floor(cT + htL), 0, NL - 1)
    cnt = (i1 - i0 + 1) * (j1 - j0 + 1)
    assert safe.sum() > 0.9 * W * H
    assert np.all(dbg[..., 15][safe] == cnt[safe])
    assert cnt.max() <= 81
