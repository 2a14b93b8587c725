"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(Carlson's elliptic integral R_F for the Binet quadrature, the weak- and
strong-field deflection series, Synge's shadow radius, special-relativistic
aberration and Doppler, the point-lens magnification, Wien's law, the
published sRGB matrix), invariants (first integral, apsis symmetry, flux and
mip sums) and special cases that reduce to a textbook routine (pinhole
projection with tent splatting).  No GPU.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest
from scipy import integrate
from scipy.special import elliprf

from paper_2010_08735_gb300 import synth

MU = 4.0 / 27.0
GOLDEN = json.loads((Path(__file__).parent / "golden" / "paper_constants.json").read_text())


# ----------------------------------------------------------------------------
# closed forms of the ray equation (Sec. 3.3.1, Eq. rayequation)
# ----------------------------------------------------------------------------

def phi_carlson(e2, u):
    """phi(u) = int_0^u du'/sqrt(u'^3 - u'^2 + e^2) for e^2 < mu, by DLMF 19.29.4
    with the three real roots r1 < 0 < r2 = u_a < r3."""
    r1, r2, r3 = np.sort(np.roots([1.0, -1.0, 0.0, e2]).real)
    if abs(u - r2) < 1e-12 * r2:
        u = r2  # at the apsis use the root itself: phi ~ sqrt(r2 - u) there
    X = [math.sqrt(u - r1), math.sqrt(max(r2 - u, 0.0)), math.sqrt(r3 - u)]
    Y = [math.sqrt(-r1), math.sqrt(r2), math.sqrt(r3)]
    U12 = (X[0] * X[1] * Y[2] + Y[0] * Y[1] * X[2]) / u
    U13 = (X[0] * X[2] * Y[1] + Y[0] * Y[2] * X[1]) / u
    U23 = (X[1] * X[2] * Y[0] + Y[1] * Y[2] * X[0]) / u
    return 2.0 * float(elliprf(U12 ** 2, U13 ** 2, U23 ** 2))


def phi_quad(e2, u):
    """Same integral by adaptive quadrature (e^2 > mu: no real root in [0,1])."""
    f = lambda x: 1.0 / math.sqrt(x ** 3 - x ** 2 + e2)
    pts = [2.0 / 3.0] if u > 2.0 / 3.0 else None
    v, _ = integrate.quad(f, 0.0, u, points=pts, epsabs=1e-14, epsrel=1e-13, limit=2000)
    return v


def test_golden_constants(orc):
    assert GOLDEN["mu"]["value"] == pytest.approx(MU, rel=1e-15)
    # mu is the maximum of u^2 (1-u) on [0,1], reached at u = 2/3
    u = np.linspace(0, 1, 200001)
    g = u * u * (1 - u)
    assert g.max() == pytest.approx(GOLDEN["mu"]["value"], rel=1e-9)
    assert u[g.argmax()] == pytest.approx(GOLDEN["photon_sphere_u"]["value"], abs=1e-5)
    assert orc.apsis(MU * (1 - 1e-14)) == pytest.approx(2.0 / 3.0, abs=1e-6)


@pytest.mark.parametrize("e2", [1e-6, 0.01, 0.1, 0.14, MU * (1 - 1e-6)])
def test_apsis_is_root_of_ray_equation(orc, e2):
    """Eq. uapsis is the smallest positive root of e^2 - u^2 (1-u)."""
    roots = np.sort(np.roots([1.0, -1.0, 0.0, e2]).real)
    assert orc.apsis(e2) == pytest.approx(roots[1], rel=1e-9)


def test_D_table_matches_carlson(orc, exact_tables):
    """D(e,u) = phi(u) - atan2(u, du/dphi) with phi from Carlson's R_F."""
    D, _ = exact_tables
    n = D.shape[0]
    worst = 0.0
    for i in [0, 1, 3, 10, 60, 128, 200, 250, 254, 255]:
        e2 = orc.d_e2_of_x(i / (n - 1))
        assert e2 < MU
        for j in [1, 50, 200, 400, 500, 510, 511]:
            u = orc.d_u_of_y(e2, j / (n - 1))
            P = u ** 3 - u ** 2 + e2
            if j == n - 1:  # y = 1 is the apsis, where du/dphi = 0
                P = 0.0
            ref = phi_carlson(e2, u) - math.atan2(u, math.sqrt(max(P, 0.0)))
            worst = max(worst, abs(D[j, i] - ref) / max(abs(ref), 1e-3))
    assert worst < 2e-8


def test_D_table_matches_quadrature_above_critical(orc, exact_tables):
    """Plunging rays (e^2 > mu): D against adaptive quadrature of the same integral."""
    D, _ = exact_tables
    n = D.shape[0]
    worst = 0.0
    for i in [256, 257, 300, 400, 480, 505, 510, 511]:
        e2 = orc.d_e2_of_x(i / (n - 1))
        assert e2 > MU
        for j in [1, 100, 250, 300, 400, 511]:
            u = orc.d_u_of_y(e2, j / (n - 1))
            P = u ** 3 - u ** 2 + e2
            ref = phi_quad(e2, u) - math.atan2(u, math.sqrt(P))
            worst = max(worst, abs(D[j, i] - ref) / max(abs(ref), 1e-3))
    assert worst < 2e-8


@pytest.mark.parametrize("e", [1e-3, 3e-3, 1e-2, 3e-2])
def test_weak_field_deflection(orc, e):
    """Total deflection 2 Delta_a = 2/b + (15 pi/16)/b^2 + (16/3)/b^3 + O(b^-4),
    e = 1/b, r_s = 1 (Schwarzschild light bending series)."""
    tot = 2.0 * orc.apsis_deflection(e * e, 1e-4)
    series = 2 * e + 15 * math.pi / 16 * e ** 2 + 16.0 / 3.0 * e ** 3
    assert abs(tot - series) < 20 * e ** 4 + 1e-12


@pytest.mark.parametrize("eta", [1e-4, 1e-6, 1e-8])
def test_strong_field_deflection(orc, eta):
    """Near b_c = 3 sqrt(3)/2: 2 Delta_a = -ln(b/b_c - 1) + ln(216 (7 - 4 sqrt 3)) - pi
    + o(1) (Bozza 2002, strong deflection limit)."""
    e2 = MU * (1 - eta)
    b = 1 / math.sqrt(e2)
    bc = 1.5 * math.sqrt(3.0)
    tot = 2.0 * orc.apsis_deflection(e2, 1e-4)
    ref = -math.log(b / bc - 1) + math.log(216 * (7 - 4 * math.sqrt(3))) - math.pi
    assert abs(tot - ref) < 50 * eta ** 0.5 + 1e-6


@pytest.mark.parametrize("e2,phi", [(0.01, 1.0), (0.1, 2.5), (0.147, 5.0), (0.2, 1.2), (2.0, 0.3)])
def test_first_integral(orc, e2, phi):
    """(du/dphi)^2 = e^2 - u^2 (1-u) holds along the integrated ray (Eq. rayequation)."""
    u, ud = orc.state_at_phi(e2, phi, 1e-3)
    assert ud * ud == pytest.approx(e2 - u * u * (1 - u), abs=1e-12)


@pytest.mark.parametrize("e2", [0.01, 0.1, 0.14])
def test_apsis_symmetry(orc, e2):
    """phi -> 2 phi_a - phi leaves the ray unchanged (Sec. 3.3.1)."""
    phia = orc.apsis_deflection(e2, 1e-4) + math.pi / 2
    for x in [0.1, 0.5, 1.0]:
        a = orc.u_of_phi(e2, phia - x, 1e-4)
        b = orc.u_of_phi(e2, phia + x, 1e-4)
        assert a == pytest.approx(b, abs=1e-10)


def test_U_table_inverts_phi(orc, exact_tables):
    """U(e,phi) = u with phi(u) = phi before the apsis, 2 phi_a - phi(u) after it,
    and u = 1 once the ray is captured (reading C7)."""
    _, U = exact_tables
    nphi, ne = U.shape
    checked = 0
    for i in range(1, ne, 3):
        e2 = orc.u_e2_of_x(i / (ne - 1))
        for j in range(1, nphi, 2):
            phi = orc.u_phi_of_y(e2, j / (nphi - 1))
            u = U[j, i]
            if e2 < MU:
                ua = orc.apsis(e2)
                phia = phi_carlson(e2, ua)
                pu = phi_carlson(e2, u)
                ref = pu if phi <= phia else 2 * phia - pu
                assert ref == pytest.approx(phi, abs=2e-7 / max(1e-3, math.sqrt(max(ua - u, 1e-12))))
            else:
                total = phi_quad(e2, 1.0)
                if phi >= total:
                    assert u == 1.0
                else:
                    assert phi_quad(e2, u) == pytest.approx(phi, abs=1e-8)
            checked += 1
    assert checked > 100


def test_plunging_rays_reach_horizon(orc, exact_tables):
    """Every D column with e^2 > mu (b < b_c) reaches u = 1: its last texel centre
    is u = 1, and u(phi) reaches 1 at a finite angle."""
    D, _ = exact_tables
    n = D.shape[0]
    for i in [256, 300, 511]:
        e2 = orc.d_e2_of_x(i / (n - 1))
        assert orc.d_u_of_y(e2, 1.0) == pytest.approx(1.0, abs=1e-15)
        assert orc.u_of_phi(e2, 50.0, 1e-3) == 1.0


# ----------------------------------------------------------------------------
# camera, aberration and Doppler (Eq. d, Sec. 3.4.2)
# ----------------------------------------------------------------------------

def test_shadow_radius_synge(orc, exact_tables):
    """For a static camera the capture boundary is at the angle psi from the hole
    with sin psi = (b_c / r) sqrt(1 - 1/r) (Synge 1966): there e^2 = mu."""
    D, U = exact_tables
    for r in [3.0, 10.0, 50.0]:
        cam = synth.camera(r, 80.0, width=64, height=64)
        f = 0.5 * 64 / math.tan(0.5 * cam["fov_y"])
        psi = math.asin(1.5 * math.sqrt(3) / r * math.sqrt(1 - 1 / r))
        b = orc.beam(cam, f * math.tan(psi), 0.0)
        e2 = orc.trace_ray(D, U, r, b["delta"], 0.0, 1 / 3, 1 / 12)["e2"]
        assert e2 == pytest.approx(MU, rel=1e-9)
        inside = orc.beam(cam, f * math.tan(psi * (1 - 1e-4)), 0.0)
        outside = orc.beam(cam, f * math.tan(psi * (1 + 1e-4)), 0.0)
        assert math.isinf(orc.trace_ray(D, U, r, inside["delta"], 0, 1 / 3, 1 / 12)["delta_p"])
        assert not math.isinf(orc.trace_ray(D, U, r, outside["delta"], 0, 1 / 3, 1 / 12)["delta_p"])


def test_static_camera_identity(orc):
    """v = 0: the beam direction is the screen direction in the static frame, and
    the camera-to-static energy ratio is 1."""
    cam = synth.camera(1e9, 60.0, phi_deg=30.0, width=100, height=80)
    rng = np.random.default_rng(0)
    for _ in range(20):
        qw, qh = rng.uniform(-50, 50), rng.uniform(-40, 40)
        b = orc.beam(cam, qw, qh)
        assert b["dcam"] == pytest.approx(1.0, abs=1e-12)
        # camera axes (e_w, e_h, e_d) = (e_phi, -e_theta, e_r); direction = q in that frame
        th, ph = cam["theta"], cam["phi"]
        er = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        et = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
        ep = np.array([-math.sin(ph), math.cos(ph), 0.0])
        q = b["q"]
        d = q[0] * ep - q[1] * et + q[2] * er
        dc = b["dcart"] / np.linalg.norm(b["dcart"])
        assert np.allclose(dc, d, atol=1e-9)


def test_aberration_and_doppler_far_from_hole(orc):
    """v != 0 at u -> 0: the static-frame direction and energy ratio follow the
    special-relativistic boost of the null vector (aberration, Doppler)."""
    rng = np.random.default_rng(1)
    for _ in range(10):
        v = rng.standard_normal(3)
        v *= rng.uniform(0.1, 0.95) / np.linalg.norm(v)
        cam = synth.camera(1e12, 70.0, v=tuple(v), width=64, height=64)
        for _ in range(5):
            qw, qh = rng.uniform(-40, 40), rng.uniform(-40, 40)
            b = orc.beam(cam, qw, qh)
            # independent boost: camera-frame photon momentum P_c = (1, -n) with n the
            # backward direction; n in the boosted (r', theta', phi') axes = O^T q
            O = np.array(cam["orient"])
            n_boost = O.T @ b["q"]
            g = 1 / math.sqrt(1 - v @ v)
            Pt, Psp = 1.0, -n_boost
            vv = v / np.linalg.norm(v)
            Ps_t = g * (Pt + v @ Psp)
            Ps_sp = Psp + ((g - 1) * (vv @ Psp) + g * Pt * np.linalg.norm(v)) * vv
            back = -Ps_sp / np.linalg.norm(Ps_sp)  # backward direction, static (r, theta, phi)
            th, ph = cam["theta"], cam["phi"]
            er = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            et = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
            ep = np.array([-math.sin(ph), math.cos(ph), 0.0])
            ref = back[0] * er + back[1] * et + back[2] * ep
            dc = b["dcart"] / np.linalg.norm(b["dcart"])
            assert np.allclose(dc, ref, atol=1e-9)
            assert b["dcam"] == pytest.approx(Pt / Ps_t, rel=1e-9)


def test_local_doppler_equals_paper_g_ratio(orc):
    """The local-frame disc Doppler factor (reading C12) equals the paper's
    g(k,l)/g(k',l') with k' the circular-orbit 4-velocity (Eq. k_prime) and a
    static camera: nu/nu' = (|e|/sqrt(1-u)) / (|e| sqrt(2/(2-3u')) +
    sqrt(u'^3/(2-3u')) e_z.e_z')."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        up = rng.uniform(1 / 20, 1 / 3)
        ucam = rng.uniform(0.0, 0.5)
        emin = up * math.sqrt(1 - up)
        e = rng.uniform(emin, 3.0)
        ezz = rng.uniform(-1, 1)
        ref = (e / math.sqrt(1 - ucam)) / (e * math.sqrt(2 / (2 - 3 * up)) +
                                          math.sqrt(up ** 3 / (2 - 3 * up)) * ezz)
        assert orc.disc_doppler(1.0, ucam, e, up, ezz) == pytest.approx(ref, rel=1e-12)


def test_disc_temperature_profile(orc):
    """T^4 ~ u^3 (1 - sqrt(3u)): zero at r = 3, maximum t_peak at r = 49/12 (Sec. 3.3.3)."""
    assert orc.disc_temperature(1e4, 1 / 3) == 0.0
    assert orc.disc_temperature(1e4, 12 / 49) == pytest.approx(1e4, rel=1e-12)
    for du in [1e-3, -1e-3]:
        assert orc.disc_temperature(1e4, 12 / 49 + du) < 1e4
    u = 0.1
    ratio = (orc.disc_temperature(1.0, u) / orc.disc_temperature(1.0, 0.2)) ** 4
    assert ratio == pytest.approx(u ** 3 * (1 - math.sqrt(3 * u)) / (0.008 * (1 - math.sqrt(0.6))),
                                  rel=1e-12)


# ----------------------------------------------------------------------------
# colour (Sec. 3.4.2)
# ----------------------------------------------------------------------------

def test_planck_wien_and_liouville(orc):
    """Wien's displacement law lambda_max T = 2.897771955e6 nm K, and the beaming
    identity D^5 B_T(D lambda) = B_{DT}(lambda) behind the black-body shift."""
    for T in [3000.0, 5800.0, 20000.0]:
        lam = np.linspace(50, 3000, 295001)
        B = np.array([orc.planck(l, T) for l in lam[::50]])
        lmax = lam[::50][B.argmax()]
        assert lmax * T == pytest.approx(2.897771955e6, rel=2e-3)
    rng = np.random.default_rng(3)
    for _ in range(50):
        l, T, D = rng.uniform(360, 830), rng.uniform(1e3, 4e4), 2 ** rng.uniform(-4, 4)
        assert D ** 5 * orc.planck(D * l, T) == pytest.approx(orc.planck(l, D * T), rel=1e-12)


def test_srgb_matrix_matches_published(orc):
    """XYZ -> linear sRGB from the Rec.709 primaries and D65 (IEC 61966-2-1 values)."""
    M = orc.xyz_to_rgb_matrix()
    ref = np.array([[3.2406, -1.5372, -0.4986], [-0.9689, 1.8758, 0.0415],
                    [0.0557, -0.2040, 1.0570]])
    assert np.allclose(M, ref, atol=2e-3)


def test_colour_table_is_blackbody_shift(orc, colour_tables):
    """C(xy, D) = XYZ(B_{DT}) / (X+Y+Z)(B_T) with T the nearest Planckian-locus
    temperature of the cell's xy in CIE 1960 uv (reading C14), found here by an
    independent brute-force search."""
    C, _ = colour_tables
    nd, ny, nx, _ = C.shape
    temps = 1000.0 * 40.0 ** (np.arange(4096) / 4095.0)
    locus = np.array([orc.blackbody_xyz(t) for t in temps])
    den = locus[:, 0] + 15 * locus[:, 1] + 3 * locus[:, 2]
    lu, lv = 4 * locus[:, 0] / den, 6 * locus[:, 1] / den
    rng = np.random.default_rng(8)
    for _ in range(12):
        i, j, k = rng.integers(nx), rng.integers(ny), rng.integers(nd)
        x, y = 0.15 + 0.60 * (i + 0.5) / nx, 0.15 + 0.35 * (j + 0.5) / ny
        X, Z = x / y, (1 - x - y) / y
        d = X + 15 + 3 * Z
        m = np.argmin((4 * X / d - lu) ** 2 + (6 / d - lv) ** 2)
        T = temps[m]
        D = 2.0 ** (-4 + 8 * (k + 0.5) / nd)
        ref = orc.blackbody_xyz(D * T) / orc.blackbody_xyz(T).sum()
        assert np.allclose(C[k, j, i], ref, rtol=1e-9, atol=0)


def test_blackbody_xyz_integral(orc):
    """The 5 nm trapezoid XYZ of a black body agrees with the adaptive integral of
    Planck times the colour matching functions over 360-830 nm."""
    for T in [2500.0, 6500.0, 25000.0]:
        tr = orc.blackbody_xyz(T)
        for c in range(3):
            ref, _ = integrate.quad(lambda l: orc.planck(l, T) * orc.cmf(l)[c], 360, 830,
                                    limit=400, epsrel=1e-10)
            assert tr[c] == pytest.approx(ref, rel=2e-3)


def kim_planckian_locus(T):
    """CIE 1931 chromaticity of a black body at T kelvin (1667-25000 K) from the
    published cubic-spline fit of the Planckian locus of Kim, Lee, Kim et al.,
    "Design of advanced color temperature control system for HDTV
    applications", J. Korean Phys. Soc. 41 (2002) -- independent of the
    oracle's colour-matching functions and spectral integration."""
    if T <= 4000.0:
        x = -0.2661239e9 / T ** 3 - 0.2343589e6 / T ** 2 + 0.8776956e3 / T + 0.179910
    else:
        x = -3.0258469e9 / T ** 3 + 2.1070379e6 / T ** 2 + 0.2226347e3 / T + 0.240390
    if T <= 2222.0:
        y = -1.1063814 * x ** 3 - 1.34811020 * x ** 2 + 2.18555832 * x - 0.20219683
    elif T <= 4000.0:
        y = -0.9549476 * x ** 3 - 1.37418593 * x ** 2 + 2.09137015 * x - 0.16748867
    else:
        y = 3.0817580 * x ** 3 - 5.87338670 * x ** 2 + 3.75112997 * x - 0.37001483
    return x, y


# oracle black body vs the published locus: the project's piecewise-Gaussian
# observer is an approximation of CIE 1931, least exact in the deep red
LOCUS_TOL = [(2600.0, 4e-3), (4500.0, 1.5e-3), (25000.0, 5e-4)]


def locus_tolerance(T):
    return next(tol for top, tol in LOCUS_TOL if T <= top)


def test_blackbody_chromaticity_on_published_planckian_locus(orc):
    """Absolute colorimetry (reading C14): the chromaticity of the oracle's
    black body, XYZ(B_T) through its colour-matching functions, lies on the
    published Planckian locus from 1700 K to 25000 K within the accuracy of a
    Gaussian-lobe fit of the CIE observer.  The pin discriminates: the same
    integration with the second radiation constant 2 % off misses the locus."""
    temps = [1700, 2000, 2500, 3000, 3500, 4000, 5000, 6500, 8000, 10000, 15000, 20000, 25000]

    def xy(xyz):
        return xyz[0] / xyz.sum(), xyz[1] / xyz.sum()

    for T in temps:
        x, y = xy(orc.blackbody_xyz(T))
        kx, ky = kim_planckian_locus(T)
        tol = locus_tolerance(T)
        assert abs(x - kx) <= tol and abs(y - ky) <= tol, (T, x, y, kx, ky)
    # planted mistake: the oracle's spectral sum redone here with c2 2 % high
    lam = 360.0 + 5.0 * np.arange(95)
    w = np.full(lam.shape, 5.0)
    w[0] = w[-1] = 2.5
    cmf = np.array([orc.cmf(float(l)) for l in lam])

    def planted_xy(T, c2):
        b = w / (lam ** 5 * np.expm1(c2 / (lam * T)))
        return xy(b @ cmf)

    for T in (3000, 6500):  # the re-done sum reproduces the oracle with the true constant
        assert np.allclose(planted_xy(T, 1.4387769e7), xy(orc.blackbody_xyz(T)), rtol=0, atol=1e-12)
    off = [max(abs(a - b) for a, b in zip(planted_xy(T, 1.02 * 1.4387769e7), kim_planckian_locus(T)))
           > locus_tolerance(T) for T in temps]
    assert any(off)


def test_blackbody_xyz_positive_and_ordered(orc):
    """Hotter black bodies are bluer: z/(x+y+z) grows with T."""
    zs = []
    for T in [2000, 4000, 6500, 10000, 30000]:
        xyz = orc.blackbody_xyz(T)
        assert np.all(xyz > 0)
        zs.append(xyz[2] / xyz.sum())
    assert np.all(np.diff(zs) > 0)


# ----------------------------------------------------------------------------
# star cube map (Sec. 3.3.2) and its encodings
# ----------------------------------------------------------------------------

def test_half_and_bf16_encoders(orc):
    rng = np.random.default_rng(4)
    vals = np.concatenate([10 ** rng.uniform(-9, 4.8, 2000), [0.0, 65504.0, 70000.0, 6e-8]])
    for v in vals:
        h = orc.encode16(float(v), 1)
        ref = np.array([min(v, 65504.0)], dtype=np.float64).astype(np.float16).view(np.uint16)[0]
        assert h == ref, v
    # bfloat16: compare with RNE of the float64 value computed on the bit level
    for v in 10 ** rng.uniform(-30, 30, 2000):
        b = orc.encode16(float(v), 2)
        m, e = math.frexp(v)
        q = round(m * 256) / 256  # RNE (Python rounds half to even)
        ref = np.float32(math.ldexp(q, e)).view(np.uint32) >> 16
        assert b == ref, v
        assert orc.decode16(b, 2) == pytest.approx(v, rel=2 ** -8)


def test_cubemap_sums_and_positions(orc):
    """Mip levels keep the total colour (colour sum, not average), and a lone
    star's texel stores the star's in-texel position."""
    st = synth.stars(3000, seed=5)
    N = 64
    rec = orc.build_cubemap(st, N, 1)
    tot = np.array([orc.star_xyz(float(s[3]), float(s[4])) for s in st], dtype=np.float64).sum(0)
    for L in range(orc.cube_levels(N)):
        off = orc.cube_level_offset(N, L)
        nl = N >> L
        r = rec[off:off + 6 * nl * nl].astype(np.uint16)
        xyz = r[:, :3].view(np.float16).astype(np.float64) * 4.0 ** L
        assert np.allclose(xyz.sum(0), tot, rtol=2e-3), L
    # a lone star
    one = np.array([[0.3, -0.2, 0.9, 5.0, 6000.0]], dtype=np.float32)
    one[0, :3] /= np.linalg.norm(one[0, :3])
    rec = orc.build_cubemap(one, N, 1)
    d = one[0, :3].astype(np.float64)
    # +z face: s = (x/|z| + 1)/2, t = (-y/|z| + 1)/2
    S = (d[0] / d[2] + 1) / 2 * N
    T = (-d[1] / d[2] + 1) / 2 * N
    i, j = int(S), int(T)
    r = rec[(4 * N + j) * N + i]
    assert (r[3] & 255) == int((S - i) * 256) and (r[3] >> 8) == int((T - j) * 256)
    assert r[:3].view(np.float16).astype(np.float64).sum() == pytest.approx(5.0, rel=2e-3)
    nz = np.flatnonzero(rec[: 6 * N * N, 1])
    assert list(nz) == [(4 * N + j) * N + i]


# ----------------------------------------------------------------------------
# star gather and lensing
# ----------------------------------------------------------------------------

def flat_tables(orc):
    Ct, dl = orc.colour_table(8, 8, 8), orc.disc_colour_table(64)
    return np.zeros((64, 64)), np.ones((8, 8)), Ct, dl


def test_flat_space_star_gather_is_pinhole_tent_splat(orc):
    """With zero deflection tables and a far static camera the star term is a
    pinhole projection of each star splatted with the tent f(w) f(h), summing
    to the star's colour (flux conservation)."""
    D, U, Ct, dl = flat_tables(orc)
    N = 2048
    W = H = 32
    cam = synth.camera(1e6, 90.0, width=W, height=H, fov_deg=2.0)
    f = 0.5 * H / math.tan(0.5 * cam["fov_y"])
    rng = np.random.default_rng(6)
    for _ in range(4):
        qw, qh = rng.uniform(-8, 8), rng.uniform(-8, 8)
        # star direction seen at screen point (qw, qh): camera looks along -x, e_w = +y, e_h = +z
        s = np.array([-f, qw, qh])
        s /= np.linalg.norm(s)
        star = np.array([[s[0], s[1], s[2], 7.0, 5000.0]], dtype=np.float32)
        rec = orc.build_cubemap(star, N, 1)
        T = orc.SceneTables(D, U, Ct, dl, rec, N, 1)
        _, dbg, _ = orc.render(cam, synth.disc(enabled=False), T, force_level=0, debug=True,
                               nthreads=2)
        Y = dbg[..., 11]
        ystar = float(orc.star_xyz(7.0, 5000.0)[1])
        assert Y.sum() == pytest.approx(ystar, rel=3e-3)
        # expected tent weights around the star's pixel coordinates
        ic = qw + W / 2 - 0.5
        jc = H / 2 - 0.5 - qh
        jj, ii = np.mgrid[0:H, 0:W]
        ref = np.maximum(1 - np.abs(ii - ic), 0) * np.maximum(1 - np.abs(jj - jc), 0) * ystar
        assert np.abs(Y - ref).max() < 0.02 * ystar
        cy = (Y * jj).sum() / Y.sum()
        cx = (Y * ii).sum() / Y.sum()
        assert abs(cx - ic) < 0.02 and abs(cy - jc) < 0.02


def test_lensing_amplification_point_lens(orc, exact_tables):
    """Omega/Omega' for a far static camera follows the point-lens image
    magnification 1 / (1 - (theta_E/theta)^4), theta_E = sqrt(2 r_s / r)."""
    D, U = exact_tables
    Ct, dl = orc.colour_table(8, 8, 8), orc.disc_colour_table(64)
    r = 1e4
    thE = math.sqrt(2.0 / r)
    W = H = 160
    fov = 8 * thE
    cam = synth.camera(r, 90.0, width=W, height=H, fov_deg=fov / synth.DEG)
    # a single dim star so that the star path runs everywhere
    star = np.array([[1.0, 0.0, 0.0, 1.0, 5000.0]], dtype=np.float32)
    T = orc.SceneTables(D, U, Ct, dl, orc.build_cubemap(star, 64, 1), 64, 1)
    _, dbg, _ = orc.render(cam, synth.disc(enabled=False), T, debug=True, nthreads=2)
    f = 0.5 * H / math.tan(0.5 * cam["fov_y"])
    jj, ii = np.mgrid[0:H, 0:W]
    qw, qh = ii + 0.5 - W / 2, H / 2 - jj - 0.5
    theta = np.arctan(np.hypot(qw, qh) / f)
    amp = dbg[..., 8]
    # beyond ~2.6 theta_E the beams have e below the first D column (e = 2.66e-3),
    # where the table clamps; one-pixel quad differences limit the accuracy to ~1 %
    sel = (theta > 1.5 * thE) & (theta < 2.5 * thE)
    ref = 1.0 / (1.0 - (thE / theta[sel]) ** 4)
    rel = np.abs(amp[sel] - ref) / ref
    assert sel.sum() > 500
    assert np.median(rel) < 0.01 and rel.max() < 0.06


# ----------------------------------------------------------------------------
# TRACERAY vs the table-free integrator (Sec. 4, 1e-3)
# ----------------------------------------------------------------------------

def test_bruteforce_weak_field_and_capture(orc):
    """The table-free integrator: deflection 2/b at large b, capture iff b < b_c."""
    b = 2000.0
    out = orc.bruteforce_ray([1e7, b, 0.0], [-1.0, 0.0, 0.0])
    defl = math.atan2(-out["dir"][1], -out["dir"][0])
    assert abs(defl) == pytest.approx(2 / b + 15 * math.pi / 16 / b ** 2, rel=1e-4)
    bc = 1.5 * math.sqrt(3)
    assert orc.bruteforce_ray([1e5, bc * 0.999, 0.0], [-1.0, 0.0, 0.0])["captured"]
    assert not orc.bruteforce_ray([1e5, bc * 1.001, 0.0], [-1.0, 0.0, 0.0])["captured"]


@pytest.mark.parametrize("workload", ["static_256", "orbit_1080p"])
def test_traceray_within_paper_error_of_bruteforce(orc, exact_tables, workload):
    """delta', u0 and u1 of TRACERAY (512x512 D and 64x32 U tables, bilinear)
    against the table-free integrator of the 3D photon orbit, for 500 random
    beams of the view: every beam within 1e-3 (Sec. 4; read as an absolute
    bound on the dimensionless delta' in radians and u = r_s/r).  Capture must
    agree on every beam; a disc-hit count may differ only where a hit of
    either method lies within that 1e-3 of a disc edge (1/r_in, 1/r_out)."""
    D, U = exact_tables
    wk = synth.WORKLOADS[workload]
    cam, disc = wk["camera"], wk["disc"]
    W, H = cam["width"], cam["height"]
    th, ph = cam["theta"], cam["phi"]
    er = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    u_edges = np.array([1 / disc["r_in"], 1 / disc["r_out"]])
    rng = np.random.default_rng(7)
    derr, uerr, nmis = [], [], 0
    for _ in range(500):
        i, j = rng.integers(0, W), rng.integers(0, H)
        b = orc.beam(cam, i + 0.5 - W / 2, H / 2 - j - 0.5)
        tr = orc.trace_ray(D, U, cam["r"], b["delta"], b["alpha"], 1 / disc["r_in"],
                           1 / disc["r_out"], b["alpha_valid"])
        bf = orc.bruteforce_ray(cam["r"] * er, b["dcart"], disc["r_in"], disc["r_out"])
        assert bf["captured"] == math.isinf(tr["delta_p"])
        if not bf["captured"]:
            dp = math.cos(tr["delta_p"]) * er + math.sin(tr["delta_p"]) * b["ey"]
            derr.append(math.acos(min(1.0, float(dp @ bf["dir"]))))
        hits = [h[0] for h in tr["hits"]]
        bfh = bf["hits_u"][:2]
        if len(hits) == len(bfh):
            uerr += [abs(a - c) for a, c in zip(hits, bfh)]
        else:
            nmis += 1
            near = [min(abs(x - u_edges)) < 1e-3 for x in hits + bfh]
            assert any(near), (hits, bfh)
    derr, uerr = np.array(derr), np.array(uerr)
    print(f"{workload}: delta' error p50 {np.median(derr):.2e} p99 {np.percentile(derr, 99):.2e} "
          f"max {derr.max():.2e} rad ({derr.size} beams); hit u error p50 {np.median(uerr):.2e} "
          f"p99 {np.percentile(uerr, 99):.2e} max {uerr.max():.2e} ({uerr.size} hits); "
          f"{nmis} hit-count differences at disc edges")
    assert derr.size > 300 and uerr.size > 100
    assert derr.max() < 1e-3
    assert uerr.max() < 1e-3
