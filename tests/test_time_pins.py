"""Pins of the oracle's retarded-time channel (Algorithm 1 stores t in D and
U; reading C5 regularises it as R = t + 1/u - ln(u/(1-u)), finite from u = 0
to the horizon).  No GPU."""
import math

import numpy as np
import pytest

MU = 4.0 / 27.0


def R_quad(e2, u):
    """R(u) = int_0^u du' / (sqrt(P) (e + sqrt(P))), P = e^2 - u'^2 (1 - u'),
    by 30-digit adaptive quadrature (substituting u' = u_a - w^2 near an apsis,
    where P = w^2 q(w) with q the quadratic cofactor of the cubic)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    e2m = mp.mpf(e2)
    e = mp.sqrt(e2m)
    if e2 < MU:
        r1, ua, r3 = sorted(r.real for r in mp.polyroots([1, -1, 0, e2m]))

        def g(w):
            up = ua - w * w
            q = (up - r1) * (r3 - up)
            return 2 / (mp.sqrt(q) * (e + w * mp.sqrt(q)))
        w0 = mp.sqrt(max(ua - mp.mpf(u), 0))
        wa = mp.sqrt(ua)
        pts = [w0] + [x for x in (wa * 1e-3, wa * 0.1) if x > w0] + [wa]
        return float(mp.quad(g, pts))

    def f(x):
        P = e2m - x * x * (1 - x)
        return 1 / (mp.sqrt(P) * (e + mp.sqrt(P)))
    um = mp.mpf(u)
    pts = [0] + ([mp.mpf(2) / 3] if um > mp.mpf(2) / 3 else []) + [um]
    return float(mp.quad(f, pts))


def test_time_channel_of_D_matches_quadrature(orc):
    D, U, DT, UT = orc.tables_exact_t(128, 16, 16, 1e-3)
    n = 128
    worst = 0.0
    for i in [0, 5, 40, 63, 64, 70, 100, 127]:
        e2 = orc.d_e2_of_x(i / (n - 1))
        for j in [1, 30, 64, 100, 126, 127]:
            u = orc.d_u_of_y(e2, j / (n - 1))
            if u >= 1.0:
                continue
            ref = R_quad(e2, u)
            worst = max(worst, abs(DT[j, i] - ref) / max(abs(ref), 1e-3))
    assert worst < 1e-7


@pytest.mark.parametrize("e2,phi", [(0.01, 0.7), (0.1, 1.5), (0.14, 2.2), (0.3, 0.4)])
def test_time_derivative_is_dt_dphi(orc, e2, phi):
    """t = R - 1/u + ln(u/(1-u)) satisfies dt/dphi = e/(u^2 (1-u)) (Eq. motionconstants)."""
    h = 1e-4
    ta = orc.time_at_phi(e2, phi - h)[3]
    tb = orc.time_at_phi(e2, phi + h)[3]
    u = orc.time_at_phi(e2, phi)[0]
    ref = math.sqrt(e2) / (u * u * (1 - u))
    assert (tb - ta) / (2 * h) == pytest.approx(ref, rel=1e-6)


@pytest.mark.parametrize("e2", [0.02, 0.1, 0.14])
def test_time_symmetric_about_apsis(orc, e2):
    """The ray is symmetric about its apsis in time as in angle."""
    phia = orc.apsis_deflection(e2, 1e-4) + math.pi / 2
    ta = orc.time_at_phi(e2, phia)[3]
    for x in [0.1, 0.4]:
        before = orc.time_at_phi(e2, phia - x)[3]
        after = orc.time_at_phi(e2, phia + x)[3]
        assert after - ta == pytest.approx(ta - before, rel=1e-8)


def test_U_time_channel_consistent_with_ray(orc):
    D, U, DT, UT = orc.tables_exact_t(64, 16, 16, 1e-3)
    ne, nphi = 16, 16
    for i in range(1, ne - 1, 3):
        e2 = orc.u_e2_of_x(i / (ne - 1))
        for j in range(1, nphi, 4):
            if U[j, i] >= 1.0:
                continue
            phi = orc.u_phi_of_y(e2, j / (nphi - 1))
            u, _, R, _ = orc.time_at_phi(e2, phi, 1e-3)
            assert UT[j, i] == pytest.approx(R, rel=1e-9, abs=1e-12)
            assert U[j, i] == pytest.approx(u, rel=1e-9, abs=1e-12)
