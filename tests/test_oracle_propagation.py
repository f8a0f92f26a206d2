"""Pins for the oracle's propagation step (App. D.2, PropagatedParticle).

The oracle uses the closed-form helix/cylinder intersection.  These tests pin
it to things other than that formula:

* an RK4 integration of the Lorentz force dp/dl = 0.299792458 q (p/|p|) x B in
  Cartesian coordinates, stepped until the track leaves the cylinder (no
  helix formula, no asin/asinh of the closed form), for barrel and endcap hits,
  both charges and both field signs, with displaced vertices;
* the straight-line limit (neutral particles, B -> 0);
* the textbook chord geometry at R / 2r = 1/2 (azimuth shift pi/6, arc R pi/3);
* the minimum pT to reach the barrel, 0.299792458 B R / 2;
* particles produced outside the detector and loopers are not propagated.
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


def _rk4_exit(R, L, B, pt, eta, phi, q, vz, h=2e-3, max_len=60.0):
    """Integrate from (0, 0, vz) until max(rho/R, |z|/L) reaches 1.

    Returns (eta_pos, phi_pos, turning_angle) at the exit point.
    """
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

    def g(s):
        return max(math.hypot(s[0], s[1]) / R, abs(s[2]) / L) - 1.0

    s = np.array([0.0, 0.0, vz, p[0], p[1], p[2]])
    turn = 0.0
    length = 0.0
    while length < max_len:
        nxt = step(s, h)
        if g(nxt) >= 0.0:
            lo, hi = 0.0, h
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if g(step(s, mid)) >= 0.0:
                    hi = mid
                else:
                    lo = mid
            ex = step(s, hi)
            turn += _dangle(s, ex)
            rho = math.hypot(ex[0], ex[1])
            return math.asinh(ex[2] / rho), math.atan2(ex[1], ex[0]), turn
        turn += _dangle(s, nxt)
        s = nxt
        length += h
    raise RuntimeError("did not leave the detector")


def _dangle(a, b):
    d = math.atan2(b[4], b[3]) - math.atan2(a[4], a[3])
    return abs((d + math.pi) % (2 * math.pi) - math.pi)


def _dphi(a, b):
    return abs((a - b + math.pi) % (2 * math.pi) - math.pi)


def test_straight_line_from_axis_keeps_direction_exactly(cms):
    rng = np.random.default_rng(1)
    for _ in range(200):
        eta = float(np.float32(rng.uniform(-4.9, 4.9)))
        phi = float(np.float32(rng.uniform(-math.pi, math.pi)))
        reach, _b, ep, pp = oracle.propagate(cms, 5.0, eta, phi, 0, 0.0)
        assert reach == 1 and ep == eta and pp == phi


@pytest.mark.parametrize("B", [3.8, -2.0])
def test_helix_matches_lorentz_force_integration(B):
    card = _card_with_B(B)
    R, L = card.R, card.L
    rng = np.random.default_rng(17 if B > 0 else 18)
    n_barrel = n_endcap = n_loop = 0
    cases = 0
    while cases < 40:
        q = int(rng.choice([-1, 1]))
        pt = float(np.float32(np.exp(rng.uniform(math.log(0.3), math.log(60.0)))))
        eta = float(np.float32(rng.uniform(-3.0, 3.0)))
        phi = float(np.float32(rng.uniform(-math.pi, math.pi)))
        vz = float(np.float32(rng.uniform(-0.2, 0.2)))
        reach, barrel, ep, pp = oracle.propagate(card, pt, eta, phi, q, vz)
        r = pt / (K * abs(B))
        if reach == 0:
            # dropped: the turning angle before the endcap is at least 2 pi
            # (the integrator runs until it exits anyway)
            e2, p2, turn = _rk4_exit(R, L, B, pt, eta, phi, q, vz, h=min(2e-3, r / 50))
            assert turn >= 2 * math.pi - 1e-6
            n_loop += 1
            cases += 1
            continue
        e2, p2, turn = _rk4_exit(R, L, B, pt, eta, phi, q, vz, h=min(2e-3, r / 50))
        assert abs(ep - e2) < 2e-8 * max(1.0, abs(e2)), (pt, eta, phi, q, vz, ep, e2)
        assert _dphi(pp, p2) < 2e-8, (pt, eta, phi, q, vz, pp, p2)
        if barrel:
            n_barrel += 1
        else:
            n_endcap += 1
        cases += 1
    assert n_barrel >= 5 and n_endcap >= 5


def test_neutral_displaced_vertex_matches_integration(cms):
    rng = np.random.default_rng(5)
    for _ in range(30):
        eta = float(np.float32(rng.uniform(-3.5, 3.5)))
        phi = float(np.float32(rng.uniform(-math.pi, math.pi)))
        vz = float(np.float32(rng.uniform(-0.25, 0.25)))
        reach, barrel, ep, pp = oracle.propagate(cms, 3.0, eta, phi, 0, vz)
        e2, p2, _ = _rk4_exit(cms.R, cms.L, 0.0, 3.0, eta, phi, 0, vz, h=5e-3)
        assert reach == 1
        assert abs(ep - e2) < 1e-9 * max(1.0, abs(e2))
        assert pp == phi


def test_small_field_limit_is_straight_line():
    tiny = _card_with_B(1e-9)
    cms = _card_with_B(3.8)
    rng = np.random.default_rng(3)
    for _ in range(100):
        eta = float(np.float32(rng.uniform(-3.0, 3.0)))
        phi = float(np.float32(rng.uniform(-3.1, 3.1)))
        vz = float(np.float32(rng.uniform(-0.2, 0.2)))
        q = int(rng.choice([-1, 1]))
        r1 = oracle.propagate(tiny, 10.0, eta, phi, q, vz)
        r0 = oracle.propagate(cms, 10.0, eta, phi, 0, vz)
        assert r1[0] == r0[0] == 1
        # deviation O(R / r): r = 10 / (0.3 * 1e-9) m
        assert abs(r1[2] - r0[2]) < 1e-9 and _dphi(r1[3], r0[3]) < 1e-9


@pytest.mark.parametrize("q,B,sign", [(1, 3.8, -1), (-1, 3.8, 1), (1, -3.8, 1), (-1, -3.8, -1)])
def test_chord_geometry_at_half(q, B, sign):
    """R / 2r = 1/2: the chord R subtends 60 degrees of the circle of radius r = R,
    so the position azimuth moves by pi/6 (against the turning sense for qB > 0)
    and the transverse arc is R pi/3."""
    card = _card_with_B(B)
    pt = K * abs(B) * card.R  # r = R
    eta, phi = 0.4, 0.3
    reach, barrel, ep, pp = oracle.propagate(card, pt, eta, phi, q, 0.0)
    assert reach == 1 and barrel == 1
    assert abs(pp - (phi + sign * math.pi / 6)) < 1e-14
    assert abs(math.sinh(ep) - (math.pi / 3) * math.sinh(eta)) < 1e-13


def test_minimum_pt_to_reach_barrel(cms):
    pt_min = K * 3.8 * 1.29 / 2  # = 0.7348 GeV: 2r = R
    assert abs(pt_min - 0.734791) < 1e-6
    above = oracle.propagate(cms, pt_min * (1 + 1e-6), 0.1, 0.0, 1, 0.0)
    below = oracle.propagate(cms, pt_min * (1 - 1e-6), 0.1, 0.0, 1, 0.0)
    assert above[0] == 1 and above[1] == 1
    # just above threshold the track meets the cylinder tangentially: pi/2 turn
    assert abs(above[3] - (-math.pi / 2)) < 2e-3
    # below threshold at small |eta| it spirals more than a full turn before the endcap
    assert below[0] == 0
    # below threshold but forward it reaches the endcap within one turn
    fwd = oracle.propagate(cms, pt_min * 0.9, 2.0, 0.0, 1, 0.0)
    assert fwd[0] == 1 and fwd[1] == 0


def test_not_propagated_cases(cms):
    assert oracle.propagate(cms, 5.0, 0.5, 0.0, 1, 3.5)[0] == 0   # vertex beyond L
    assert oracle.propagate(cms, 5.0, 0.5, 0.0, 0, -3.5)[0] == 0
    assert oracle.propagate(cms, 0.0, 1.0, 0.0, 1, 0.0)[0] == 0    # pT = 0 charged: no transverse motion
    assert oracle.propagate(cms, 0.5, 0.0, 0.0, -1, 0.0)[0] == 0   # pz = 0 below barrel threshold
    r = oracle.propagate(cms, 0.5, 0.0, 0.0, 0, 0.0)                 # neutral at eta = 0: barrel
    assert r[0] == 1 and r[1] == 1 and r[2] == 0.0


def test_classification():
    assert oracle.classify(11, -1) == oracle.CLS_E
    assert oracle.classify(-11, 1) == oracle.CLS_E
    assert oracle.classify(13, -1) == oracle.CLS_MU
    assert oracle.classify(22, 0) == oracle.CLS_GAMMA
    for p in (211, -211, 321, 2212, -2212):
        assert oracle.classify(p, 1 if p > 0 else -1) == oracle.CLS_CHAD
    for p in (130, 2112):
        assert oracle.classify(p, 0) == oracle.CLS_NHAD
    for p in (12, -14, 16):
        assert oracle.classify(p, 0) == oracle.CLS_INVIS
