"""Pins of the oracle's lens-glare bloom (Sec. 3.4.3; oracle/bloom.py) against
library routines, closed forms and the point spread function it approximates.
No GPU."""
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle import bloom as ob


def test_psf_weights_sum_to_one_and_follow_the_wings():
    """The weights are energy shares (sum 1).  Far from the core (theta >> 0.02
    deg) the PSF is 0.478 x 20.91/theta^3 + 0.138 x 72.37/theta^2, whose energy
    between theta_a and theta_b is 2 pi (0.478 x 20.91 (1/theta_a - 1/theta_b)
    + 0.138 x 72.37 ln(theta_b/theta_a)): an octave of radius takes a constant
    share from the 1/theta^2 wing plus a halving one from the 1/theta^3 wing."""
    w = ob.bloom_weights(math.radians(60), 1080, 10)
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    a = 60.0 / 1080
    tot = ob.psf_energy(0.0, a * 2 ** 10.5)
    c = 0.02
    F1 = lambda t: -1 / (t + c) + c / (2 * (t + c) ** 2)  # antiderivative of theta/(theta+c)^3
    F2 = lambda t: math.log(t + c) + c / (t + c)          # antiderivative of theta/(theta+c)^2
    for k in (5, 6, 7, 8, 9, 10):  # theta >= 1.2 deg: the Gaussian core adds nothing
        ta, tb = a * 2 ** (k - 0.5), a * 2 ** (k + 0.5)
        wing = 2 * math.pi * (0.478 * 20.91 * (F1(tb) - F1(ta)) + 0.138 * 72.37 * (F2(tb) - F2(ta)))
        assert w[k] == pytest.approx(wing / tot, rel=1e-8), k
    # and the share per octave tends to the 1/theta^2 wing's constant
    assert w[10] == pytest.approx(2 * math.pi * 0.138 * 72.37 * math.log(2) / tot, rel=2e-2)


def test_psf_energy_closed_form_pieces():
    """The Gaussian core alone integrates to 2.61e6 pi 0.02^2 and the 1/theta^3
    term to 2 pi 20.91 / (2 x 0.02) over (0, inf): the two published terms carry
    the same energy to 0.2 %."""
    e0 = 2.61e6 * math.pi * 0.02 ** 2
    e1 = 2 * math.pi * 20.91 / (2 * 0.02)
    assert abs(e0 / e1 - 1) < 2e-3
    # the quadrature reproduces them (the 1/theta^2 term integrated separately)
    e2 = 2 * math.pi * 72.37 * (math.log(10.02 / 0.02) + 0.02 / 10.02 - 1.0)
    ref = 0.384 * e0 + 0.478 * e1 * (1 - (1 / 10.02 - 0.02 / (2 * 10.02 ** 2)) / (1 / 0.02 - 1 / 0.04)) + 0.138 * e2
    assert ob.psf_energy(0.0, 10.0) == pytest.approx(ref, rel=1e-9)


def test_steps_match_library_routines():
    rng = np.random.default_rng(3)
    img = rng.random((37, 53, 3))
    # separable blur with clamped edges = scipy's correlate1d, mode 'nearest'
    k = ob.gauss_taps()
    ref = ndimage.correlate1d(ndimage.correlate1d(img, k, axis=1, mode="nearest"), k, axis=0, mode="nearest")
    assert np.allclose(ob.blur(img), ref, rtol=0, atol=1e-14)
    # box downsample: odd edges replicate the last row/column
    pad = np.pad(img, ((0, 1), (0, 1), (0, 0)), mode="edge")
    ref = pad.reshape(19, 2, 27, 2, 3).mean(axis=(1, 3))
    assert np.allclose(ob.downsample(img), ref, rtol=0, atol=1e-15)
    # bilinear upsampling at the pixel centres, clamped = map_coordinates, order 1
    lev = rng.random((5, 7, 3))
    k = 3
    H, W = 37, 53
    yy, xx = np.mgrid[0:H, 0:W]
    coords = [(yy + 0.5) / 2 ** k - 0.5, (xx + 0.5) / 2 ** k - 0.5]
    ref = np.stack([ndimage.map_coordinates(lev[..., c], coords, order=1, mode="nearest") for c in range(3)], -1)
    assert np.allclose(ob.upsample(lev, k, H, W), ref, rtol=0, atol=1e-14)


def test_bloom_conserves_energy_and_is_linear():
    w = ob.bloom_weights(math.radians(60), 1080, 5)
    H = W = 384
    img = np.zeros((H, W, 3))
    img[191, 192] = [1.0, 2.0, 3.0]
    img[200, 180] = [0.5, 0.0, 4.0]
    out = ob.bloom(img, w)
    assert np.allclose(out.sum(axis=(0, 1)), img.sum(axis=(0, 1)), rtol=1e-12)
    rng = np.random.default_rng(2)
    a, b = rng.random((H, W, 3)), rng.random((H, W, 3))
    assert np.allclose(ob.bloom(2 * a - 3 * b, w), 2 * ob.bloom(a, w) - 3 * ob.bloom(b, w), atol=1e-12)
    # no bloom levels: the identity
    assert np.array_equal(ob.bloom(a, np.array([1.0])), a)


def test_point_source_follows_the_psf():
    """The bloom of one pixel holds, within every radius from 2^(1/2) to 64
    pixels, the PSF's encircled energy to within 0.04 -- the error of handing
    each octave of radius to one Gaussian level (the 1080p camera's pixel
    angle, six levels)."""
    K, fov, height = 6, math.radians(60), 1080
    w = ob.bloom_weights(fov, height, K)
    H = W = 512
    img = np.zeros((H, W, 3))
    img[256, 256] = 1.0
    out = ob.bloom(img, w)[..., 1]
    yy, xx = np.mgrid[0:H, 0:W]
    r = np.hypot(xx - 256, yy - 256)
    a = math.degrees(fov) / height
    tot = ob.psf_energy(0.0, a * 2 ** (K + 0.5))
    for R in 2.0 ** np.arange(0.5, 6.01, 0.5):
        ee = out[r <= R].sum()
        assert abs(ee - ob.psf_energy(0.0, a * R) / tot) < 0.04, R
