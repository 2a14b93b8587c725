"""Pins of the oracle's free-fall camera orbit (Appendix C) against closed
forms: circular geodesics, the radial drop from rest (cycloid), the energy
first integral, and the geometry of the orbital plane.  No GPU."""
import math

import numpy as np
import pytest


def test_circular_orbit_stays_circular(orc):
    r0 = 6.0
    u = 1 / r0
    vcirc = math.sqrt(u / (2 * (1 - u)))
    o = orc.orbit_init(r0, math.pi / 2, vcirc, 0.4)
    assert o.l == pytest.approx(math.sqrt(1 / (u * (2 - 3 * u))), rel=1e-12)
    orc.orbit_advance(o, 200.0, 4000)
    assert o.r == pytest.approx(r0, abs=1e-9)
    assert o.psi == pytest.approx(o.l * u * u * 200.0, rel=1e-10)
    cam = orc.orbit_camera(o)
    speed = math.sqrt(sum(x * x for x in cam["v"]))
    assert speed == pytest.approx(vcirc, rel=1e-12)


def test_radial_drop_from_rest_is_a_cycloid(orc):
    """r = r0 (1 + cos eta)/2, tau = sqrt(r0^3/4) (eta + sin eta) (r_s = 1)."""
    r0 = 10.0
    o = orc.orbit_init(r0, math.pi, 0.0, 0.0)
    assert o.l == pytest.approx(0.0, abs=1e-12)
    tau = 0.0
    h = 1e-3
    while o.r > 2.0:
        orc.orbit_advance(o, h, 1)
        tau += h
    eta = math.acos(2 * o.r / r0 - 1)
    ref = math.sqrt(r0 ** 3 / 4) * (eta + math.sin(eta))
    assert tau == pytest.approx(ref, abs=2e-3)


@pytest.mark.parametrize("r0,delta0,v0", [(8.0, 1.2, 0.3), (20.0, 2.2, 0.25), (5.0, 1.6, 0.45)])
def test_energy_first_integral(orc, r0, delta0, v0):
    o = orc.orbit_init(r0, delta0, v0, 0.2)
    for _ in range(20):
        orc.orbit_advance(o, 2.0, 200)
        if o.r < 1.5:
            break
        u = 1 / o.r
        rhs = o.e ** 2 + o.l ** 2 * u ** 3 - o.l ** 2 * u ** 2 + u - 1
        assert o.rdot ** 2 == pytest.approx(rhs, abs=1e-10)


def test_initial_speed_and_direction(orc):
    """The camera's speed wrt the static observer at the start is v0, and its
    direction makes the coordinate angle delta0 with the radius: tan delta =
    r dpsi/dr = tan(static-frame angle) / sqrt(1 - u)."""
    for r0, d0, v0 in [(8.0, 1.2, 0.3), (12.0, 2.5, 0.6)]:
        o = orc.orbit_init(r0, d0, v0, 0.7)
        cam = orc.orbit_camera(o)
        v = np.array(cam["v"])
        assert np.linalg.norm(v) == pytest.approx(v0, rel=1e-12)
        u = 1 / r0
        assert math.atan2(math.hypot(v[1], v[2]), v[0] * math.sqrt(1 - u)) == pytest.approx(d0, abs=1e-12)


def test_orbit_plane_geometry(orc):
    """Position on r (cos chi cos psi, sin psi, sin chi cos psi), and the
    tangential velocity along the derivative of that position in psi (this
    fixes the sign of e_chi . e_phi, reading C22)."""
    chi = 0.6
    o = orc.orbit_init(9.0, 1.3, 0.35, chi)
    orc.orbit_advance(o, 7.0, 300)
    cam = orc.orbit_camera(o)
    th, ph, psi = cam["theta"], cam["phi"], o.psi
    pos = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    ref = np.array([math.cos(chi) * math.cos(psi), math.sin(psi), math.sin(chi) * math.cos(psi)])
    assert np.allclose(pos, ref, atol=1e-12)
    et = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    ep = np.array([-math.sin(ph), math.cos(ph), 0.0])
    vt = cam["v"][1] * et + cam["v"][2] * ep
    dpos = np.array([-math.cos(chi) * math.sin(psi), math.cos(psi), -math.sin(chi) * math.sin(psi)])
    assert np.allclose(vt / np.linalg.norm(vt), dpos, atol=1e-12)
    # the orientation rows stay orthonormal
    O = np.array(cam["orient"])
    assert np.allclose(O @ O.T, np.eye(3), atol=1e-12)
