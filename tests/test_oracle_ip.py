"""Pins of the oracle's track impact parameters (the paper's output table of
Sec. 2.5: d0, z0 and their errors for charged particles).

The oracle takes the point of closest approach from the circle geometry.
These tests pin it to something else:

* an RK4 integration of the Lorentz force dp/dl = 0.299792458 q (p/|p|) x B
  in Cartesian coordinates, stepped forward and backward from the vertex, with
  the transverse distance to the beam axis minimised along the path (golden
  section on the integrated trajectory); d0 is that distance signed by the
  angular momentum about the axis, z0 the z of that point;
* the vertex on the axis (d0 = 0, z0 = vz), the straight line for B = 0
  (hand-worked numbers), and mirror symmetries;
* the errors sqrt(a^2 + (b/pT)^2) with hand-worked numbers, and the smeared
  values' counter contract and moments.
"""
import math

import numpy as np
import pytest

import oracle

K = 0.299792458


@pytest.fixture(scope="module")
def cms():
    return oracle.load_card("cms_like")


def _card_with_B(B):
    c = oracle.load_card("cms_like")
    c.B = B
    return c


def _rk4_pca(B, pt, eta, phi, q, x0, y0, z0, span, h=2e-4):
    """(d0, z0) of the trajectory integrated over path lengths [-span, span]
    (3D path l; transverse distance minimised)."""
    p = np.array([pt * math.cos(phi), pt * math.sin(phi), pt * math.sinh(eta)])
    pmag = float(np.linalg.norm(p))
    bvec = np.array([0.0, 0.0, B])

    def deriv(s):
        d = s[3:] / pmag
        return np.concatenate([d, K * q * np.cross(d, bvec)])

    def step(s, dl):
        k1 = deriv(s)
        k2 = deriv(s + 0.5 * dl * k1)
        k3 = deriv(s + 0.5 * dl * k2)
        k4 = deriv(s + dl * k3)
        return s + dl / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)

    start = np.array([x0, y0, z0, p[0], p[1], p[2]])
    best = (math.hypot(x0, y0), start, 0.0)
    for sign in (1.0, -1.0):
        s, l = start.copy(), 0.0
        while l < span:
            s = step(s, sign * h)
            l += h
            rho = math.hypot(s[0], s[1])
            if rho < best[0]:
                best = (rho, s.copy(), sign * l)
    # golden-section refinement around the best grid point
    _, s_best, l_best = best

    def at(l):
        return step(s_best, l - l_best) if l != l_best else s_best

    lo, hi = l_best - h, l_best + h
    gr = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        a = hi - gr * (hi - lo)
        b = lo + gr * (hi - lo)
        if math.hypot(*at(a)[:2]) < math.hypot(*at(b)[:2]):
            hi = b
        else:
            lo = a
    st = at(0.5 * (lo + hi))
    d = st[3:5] / np.linalg.norm(st[3:5])
    d0 = st[1] * d[0] - st[0] * d[1]   # (p_hat x pca)_z
    return d0, st[2]


@pytest.mark.parametrize("q,B", [(1, 3.8), (-1, 3.8), (1, -2.0), (2, 1.5)])
@pytest.mark.parametrize("pt,eta,phi,x0,y0,z0", [
    (0.8, 0.4, 0.3, 0.004, -0.002, 0.01),
    (2.0, -1.2, -2.5, -0.01, 0.006, -0.03),
    (0.4, 2.0, 1.9, 0.02, 0.015, 0.0),
    (15.0, 0.1, 3.0, -0.003, -0.004, 0.05),
])
def test_against_lorentz_force_integration(pt, eta, phi, x0, y0, z0, q, B):
    c = _card_with_B(B)
    d0, zz0, s = oracle.track_ip(c, pt, eta, phi, q, x0, y0, z0)
    span = 3 * math.hypot(x0, y0) * math.cosh(eta) + 0.01
    rd0, rz0 = _rk4_pca(B, pt, eta, phi, q, x0, y0, z0, span)
    assert d0 == pytest.approx(rd0, abs=2e-9)
    assert zz0 == pytest.approx(rz0, abs=2e-8)


def test_vertex_on_the_axis(cms):
    for q in (1, -1):
        d0, z0, s = oracle.track_ip(cms, 3.0, 0.7, -1.1, q, 0.0, 0.0, 0.042)
        assert d0 == 0.0 and z0 == 0.042 and s == 0.0


def test_straight_line_hand_worked():
    """B = 0: vertex (3, 4) mm, phi = 0: the line y = 4 mm passes the axis at
    x = 0, 3 mm behind the vertex: d0 = +4 mm (p_hat x pca = (1,0) x (0,4mm)),
    s = -3 mm, z0 = z_v - 3 mm sinh(eta)."""
    c = _card_with_B(0.0)
    d0, z0, s = oracle.track_ip(c, 5.0, 0.5, 0.0, 1, 0.003, 0.004, 0.02)
    assert d0 == pytest.approx(0.004, abs=1e-15)
    assert s == pytest.approx(-0.003, abs=1e-15)
    assert z0 == pytest.approx(0.02 - 0.003 * math.sinh(0.5), abs=1e-15)


def test_high_momentum_tends_to_the_straight_line(cms):
    c0 = _card_with_B(0.0)
    args = (0.6, 2.2, 1, 0.005, -0.007, 0.01)
    d_line, z_line, _ = oracle.track_ip(c0, 1.0, *args)
    d_hi, z_hi, _ = oracle.track_ip(cms, 1e5, *args)
    assert d_hi == pytest.approx(d_line, abs=1e-9)
    assert z_hi == pytest.approx(z_line, abs=1e-9)


def test_mirror_symmetry(cms):
    """Reflecting the event in the y = 0 plane (y -> -y, phi -> -phi) and
    flipping the charge (the field's sense of rotation is mirrored) gives
    d0 -> -d0 and the same z0."""
    d0, z0, _ = oracle.track_ip(cms, 1.3, -0.4, 0.8, 1, 0.006, 0.009, -0.02)
    m0, mz, _ = oracle.track_ip(cms, 1.3, -0.4, -0.8, -1, 0.006, -0.009, -0.02)
    assert m0 == pytest.approx(-d0, abs=1e-15) and mz == pytest.approx(z0, abs=1e-15)


def test_errors_and_smearing_contract(cms):
    ip = oracle.IPParams(10e-6, 50e-6, 30e-6, 80e-6)
    # pT = 5 GeV: sigma_d0 = sqrt(1e-10 + 1e-10) = 14.142 um, sigma_z0 = sqrt(9e-10 + 2.56e-10) = 34.0 um
    o = oracle.track_ip_smeared(cms, ip, 5.0, 0.3, 0.2, 1, 0.001, 0.0, 0.0, 7, 3, 11)
    assert o[2] == pytest.approx(math.sqrt(2e-10), rel=1e-12)
    assert o[3] == pytest.approx(math.sqrt(1.156e-9), rel=1e-12)
    d0, z0, _ = oracle.track_ip(cms, 5.0, 0.3, 0.2, 1, 0.001, 0.0, 0.0)
    w = oracle.philox([11, 3, 9, 0], [7, 0])
    assert o[0] == pytest.approx(d0 + o[2] * oracle.normal(int(w[0]), int(w[1])), abs=1e-18)
    assert o[1] == pytest.approx(z0 + o[3] * oracle.normal(int(w[2]), int(w[3])), abs=1e-18)


def test_smearing_moments(cms):
    ip = oracle.IPParams(10e-6, 50e-6, 30e-6, 80e-6)
    n = 20000
    res = np.array([oracle.track_ip_smeared(cms, ip, 2.0, 0.0, 0.0, 1, 0.0, 0.0, 0.0, 5, 1, i) for i in range(n)])
    sd, sz = res[0, 2], res[0, 3]
    for col, sig in ((0, sd), (1, sz)):
        x = res[:, col] / sig
        assert abs(x.mean()) < 5 / math.sqrt(n)
        assert abs(x.var() - 1.0) < 0.05
    assert abs(np.corrcoef(res[:, 0], res[:, 1])[0, 1]) < 5 / math.sqrt(n)
