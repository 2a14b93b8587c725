"""Pins of the oracle's animated disc (Appendix B) and of the hit geometry and
retarded times it reads, against closed forms, library routines and the
table-free photon integrator.  No GPU."""
import math

import numpy as np
import pytest

from paper_2010_08735_gb300 import synth

MU = 4.0 / 27.0
special = pytest.importorskip("scipy.special")


@pytest.mark.parametrize("k", [0.0, 0.1, 0.5, 0.9, 0.99])
def test_ellipk_matches_library(orc, k):
    # scipy's ellipk takes the parameter m = k^2
    assert orc.ellipk(k) == pytest.approx(special.ellipk(k * k), rel=1e-14)


def exact_orbit_u(u1, u2, phi):
    """Darwin's massive-particle orbit u = u1 + (u2 - u1) sn^2(phi/2 sqrt(u3 - u1), kappa)."""
    u3 = 1.0 - u1 - u2
    m = (u2 - u1) / (u3 - u1)
    sn, _, _, _ = special.ellipj(0.5 * phi * math.sqrt(u3 - u1), m)
    return u1 + (u2 - u1) * sn * sn


@pytest.mark.parametrize("u1,u2", [(0.1, 0.12), (0.2, 0.21), (0.08, 0.15)])
def test_exact_orbit_solves_geodesic_equation(u1, u2):
    """The closed form satisfies (du/dphi)^2 = (u - u1)(u2 - u)(u3 - u), the
    Schwarzschild (r_s = 1) orbit equation whose roots sum to 1."""
    u3 = 1.0 - u1 - u2
    h = 1e-6
    for phi in [0.3, 1.1, 2.5, 4.0]:
        du = (exact_orbit_u(u1, u2, phi + h) - exact_orbit_u(u1, u2, phi - h)) / (2 * h)
        u = exact_orbit_u(u1, u2, phi)
        assert du * du == pytest.approx((u - u1) * (u2 - u) * (u3 - u), rel=1e-6, abs=1e-14)


@pytest.mark.parametrize("u1,u2", [(0.1, 0.105), (0.2, 0.21), (0.08, 0.088)])
def test_quasi_circular_approximation_of_the_orbit(orc, u1, u2):
    """The oracle's sin^2 form agrees with the exact sn^2 orbit to O(kappa^2)
    of its amplitude, and both reach u1 and u2 at the same angles."""
    u3 = 1.0 - u1 - u2
    kappa2 = (u2 - u1) / (u3 - u1)
    worst = 0.0
    for phi in np.linspace(0.0, 12.0, 61):
        u, ph = orc.particle_point([u1, u2, 0.0], 0.0, phi)
        assert ph == pytest.approx(phi)
        worst = max(worst, abs(u - exact_orbit_u(u1, u2, phi)))
    assert worst <= (u2 - u1) * kappa2
    half = 2.0 * special.ellipk(kappa2) / math.sqrt(u3 - u1)  # half a radial period
    assert orc.particle_point([u1, u2, 0.0], 0.0, half)[0] == pytest.approx(u2, rel=1e-12)
    assert orc.particle_point([u1, u2, 0.0], 0.0, 2 * half)[0] == pytest.approx(u1, rel=1e-12)


@pytest.mark.parametrize("r", [4.0, 6.0, 12.0])
def test_circular_angular_velocity(orc, r):
    """d phi/dt of a circular orbit equals L u^2 (1 - u) / E with the
    circular-orbit constants L^2 = M r^2/(r - 3M), E = (1 - 2M/r)/sqrt(1 - 3M/r)."""
    M = 0.5
    L = math.sqrt(M * r * r / (r - 3 * M))
    E = (1 - 2 * M / r) / math.sqrt(1 - 3 * M / r)
    omega = (L / r ** 2) * (1 - 2 * M / r) / E
    u = 1.0 / r
    t = 37.0
    ph0 = orc.particle_point([u, u, 0.4], 0.0, 0.0)[1]
    ph1 = orc.particle_point([u, u, 0.4], t, 0.0)[1]
    assert (ph1 - ph0) / t == pytest.approx(omega, rel=1e-12)


def test_density_closed_forms(orc):
    """One circular particle at r = 8: its centre (a = pi) has density rho, its
    ends (a = 0, 2 pi) none; a radial or angular offset of half the support
    gives (1 - 1/4)^2 rho; the centre moves with the orbit; sums clamp at 1."""
    p = np.array([[1 / 8, 1 / 8, 0.0]])
    rho = 0.5
    assert orc.disc_density(p, rho, 0.0, 8.0, math.pi) == pytest.approx(rho)
    assert orc.disc_density(p, rho, 0.0, 8.5, math.pi) == pytest.approx(0.5625 * rho)
    assert orc.disc_density(p, rho, 0.0, 8.0, math.pi / 2) == pytest.approx(0.5625 * rho)
    assert orc.disc_density(p, rho, 0.0, 8.0, 1e-9) == pytest.approx(0.0, abs=1e-8)
    assert orc.disc_density(p, rho, 0.0, 9.5, math.pi) == 0.0
    omega = math.sqrt(0.5 / 8 ** 3)
    t = 100.0
    assert orc.disc_density(p, rho, t, 8.0, math.pi + omega * t - 2 * math.pi) == pytest.approx(rho)
    assert orc.disc_density(np.vstack([p, p]), 0.8, 0.0, 8.0, math.pi) == 1.0


def test_particle_recipe_is_valid():
    p = synth.disc_particles(16, 5, 3.0, 12.0)
    assert p.shape == (16, 3)
    assert (p[:, 0] <= p[:, 1]).all() and (p[:, 1] <= 1 / 3).all() and (p[:, 0] > 0).all()


def test_hit_delays_and_azimuths_match_bruteforce(orc):
    """Disc hits of TRACERAY with the time channels: the radius, the retarded
    time (coordinate time from the hit to the camera) and the azimuth of the
    hit point (at angle psi from e_x' towards e_y') against the table-free
    photon orbit, which integrates dt/dlambda = E/(1 - 1/r) along the way."""
    D, U, DT, UT = orc.tables_exact_t(512, 64, 32, 1e-3)
    wk = synth.WORKLOADS["static_256"]
    cam, disc = wk["camera"], wk["disc"]
    W, H = cam["width"], cam["height"]
    th, ph = cam["theta"], cam["phi"]
    er = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    rng = np.random.default_rng(11)
    terr, perr, n = [], [], 0
    for _ in range(80):
        i, j = rng.integers(0, W), rng.integers(0, H)
        b = orc.beam(cam, i + 0.5 - W / 2, H / 2 - j - 0.5)
        tr = orc.trace_ray_t(D, DT, U, UT, cam["r"], b["delta"], b["alpha"], 1 / disc["r_in"],
                             1 / disc["r_out"], b["alpha_valid"])
        if not tr["hits"] or abs(tr["e2"] / MU - 1) < 0.05:
            continue
        bf = orc.bruteforce_ray(cam["r"] * er, b["dcart"], disc["r_in"], disc["r_out"])
        for u, psi, delay in tr["hits"]:
            k = int(np.argmin([abs(u - c) for c in bf["hits_u"]]))
            if abs(u - bf["hits_u"][k]) > 1e-2 * u:
                continue
            n += 1
            hd = math.cos(psi) * er + math.sin(psi) * b["ey"]
            assert abs(hd[2]) < 1e-9  # the hit point lies in the disc plane
            terr.append(abs(delay - bf["hits_t"][k]) / bf["hits_t"][k])
            dphi = math.atan2(hd[1], hd[0]) - bf["hits_phi"][k]
            perr.append(abs(math.remainder(dphi, 2 * math.pi)))
    assert n > 20
    assert np.median(terr) < 1e-3 and max(terr) < 1e-2, (np.median(terr), max(terr))
    assert np.median(perr) < 1e-3 and max(perr) < 1e-2, (np.median(perr), max(perr))


def test_render_density_channels_consistent(orc, exact_tables, colour_tables):
    """The animated render's per-hit densities equal the density function at
    the hit's retarded time, radius and azimuth, and the constant disc is the
    n_particles = 0 case."""
    D, U, DT, UT = orc.tables_exact_t(512, 64, 32, 1e-3)
    Ct, dl = colour_tables
    scene = orc.SceneTables(D, U, Ct, dl, DT=DT, UT=UT)
    cam = synth.camera(10.0, 80.0, width=48, height=48)
    parts = synth.disc_particles(16, 5, 3.0, 12.0)
    disc = dict(synth.disc(3.0, 12.0), particles=parts, time=250.0)
    _, dbg, _ = orc.render(cam, disc, scene, debug=True, nthreads=4)
    _, dbg0, _ = orc.render(cam, synth.disc(3.0, 12.0), scene, debug=True, nthreads=4)
    checked = 0
    for y in range(48):
        for x in range(48):
            d = dbg[y, x]
            for h in range(int(d[3])):
                want = orc.disc_density(parts, 0.5, 250.0 - d[23 + h], 1.0 / d[4 + h], d[27 + h])
                assert d[25 + h] == pytest.approx(want, rel=1e-12, abs=1e-15)
                assert dbg0[y, x, 25 + h] == 0.5
                checked += 1
    assert checked > 100
    assert (dbg[..., 25:27] > 0).any() and (dbg[..., 25:27] < 0.5).any()
