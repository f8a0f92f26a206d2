"""Pins for the resolution model sigma(x)/x = a/sqrt(x) (+) b/x (+) c (+) d x and
for the smearing as it is applied inside an event.

* each coefficient alone reduces to its textbook term (stochastic a/sqrt(E),
  noise b/E, constant c, the tracker's d pT);
* the four terms add in quadrature (squares add);
* the |eta| bin picks the row of coefficients;
* inside events, smeared track pT and photon energies have mean x and standard
  deviation sigma(x) for the card's coefficients (z-tests over many particles).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle

P_MIN = 1e-3


def _card_with_res(comp, rows, edges):
    c = oracle.load_card("cms_like")
    c.res_n[comp] = len(edges)
    for k, e in enumerate(edges):
        c.res_edges[comp][k] = e
    for k, abcd in enumerate(rows):
        for j in range(4):
            c.res_abcd[comp][k][j] = abcd[j]
    return c


def test_single_terms_reduce_to_textbook_forms():
    comp = oracle.RES_ECAL
    c = _card_with_res(comp, [(0.5, 0, 0, 0)], [0.0])
    assert oracle.rel_resolution(c, comp, 0.3, 4.0) == pytest.approx(0.25, rel=1e-15)   # a / sqrt(E)
    c = _card_with_res(comp, [(0, 0.3, 0, 0)], [0.0])
    assert oracle.rel_resolution(c, comp, 0.3, 6.0) == pytest.approx(0.05, rel=1e-15)   # b / E
    c = _card_with_res(comp, [(0, 0, 0.02, 0)], [0.0])
    assert oracle.rel_resolution(c, comp, 0.3, 123.0) == pytest.approx(0.02, rel=1e-15)  # c
    c = _card_with_res(comp, [(0, 0, 0, 1e-3)], [0.0])
    assert oracle.rel_resolution(c, comp, 0.3, 50.0) == pytest.approx(0.05, rel=1e-15)  # d pT


def test_terms_add_in_quadrature():
    comp = oracle.RES_HCAL
    full = (0.7, 0.4, 0.03, 2e-4)
    for x in (0.3, 2.0, 17.0, 400.0):
        tot = oracle.rel_resolution(_card_with_res(comp, [full], [0.0]), comp, 1.0, x) ** 2
        parts = 0.0
        for j in range(4):
            one = [0.0] * 4
            one[j] = full[j]
            parts += oracle.rel_resolution(_card_with_res(comp, [one], [0.0]), comp, 1.0, x) ** 2
        assert tot == pytest.approx(parts, rel=1e-13)


def test_eta_bin_selects_coefficients():
    comp = oracle.RES_TRACK
    c = _card_with_res(comp, [(0, 0, 0.01, 0), (0, 0, 0.03, 0), (0, 0, 0.05, 0)], [0.0, 1.5, 2.5])
    assert oracle.rel_resolution(c, comp, 1.49, 10.0) == pytest.approx(0.01)
    assert oracle.rel_resolution(c, comp, 1.5, 10.0) == pytest.approx(0.03)   # bins are [lo, hi)
    assert oracle.rel_resolution(c, comp, 2.6, 10.0) == pytest.approx(0.05)   # last bin is open


def _sigma(abcd, x):
    a, b, c, d = abcd
    return x * math.sqrt(a * a / x + b * b / (x * x) + c * c + d * d * x * x)


def _moment_z(xs, x, sig):
    n = xs.size
    q = 1.0 + (sig / x) ** 2
    m2, m4 = x * x * q, x**4 * q**6
    z1 = abs(xs.mean() - x) / math.sqrt((m2 - x * x) / n)
    z2 = abs((xs * xs).mean() - m2) / math.sqrt((m4 - m2 * m2) / n)
    return z1, z2


@pytest.mark.parametrize("pt,eta,abcd", [(20.0, 0.5, (0, 0, 0.01, 1e-4)), (150.0, 2.0, (0, 0, 0.02, 2e-4))])
def test_track_smearing_in_events(pt, eta, abcd):
    card = oracle.load_card("cms_like")
    rows = {k: np.full(500, v, dtype=dt) for k, v, dt in
            (("pt", pt, np.float32), ("eta", eta, np.float32), ("phi", 0.1, np.float32),
             ("mass", 0.13957039, np.float32), ("pdg", 211, np.int32), ("charge", 1, np.int8))}
    vals = []
    for e in range(200):
        r = oracle.run_event(card, rows, seed=21, event=e, g=0.0)
        vals.append(r.tracks["pt"])
    xs = np.concatenate(vals)
    assert xs.size > 50_000
    zcrit = stats.norm.isf(P_MIN / 2)
    z1, z2 = _moment_z(xs, float(np.float32(pt)), _sigma(abcd, float(np.float32(pt))))
    assert z1 < zcrit and z2 < zcrit


@pytest.mark.parametrize("eta,abcd", [(0.8, (0.03, 0.12, 0.005, 0)), (2.1, (0.06, 0.25, 0.01, 0))])
def test_photon_energy_smearing_in_events(eta, abcd):
    card = oracle.load_card("cms_like")
    pt = 40.0
    rows = {k: np.full(400, v, dtype=dt) for k, v, dt in
            (("pt", pt, np.float32), ("eta", eta, np.float32), ("phi", -1.0, np.float32),
             ("mass", 0.0, np.float32), ("pdg", 22, np.int32), ("charge", 0, np.int8))}
    e_true = pt * math.cosh(float(np.float32(eta)))
    vals = []
    for e in range(200):
        r = oracle.run_event(card, rows, seed=22, event=e, g=0.0)
        vals.append(r.cands["pt"] * math.cosh(float(np.float32(eta))))
    xs = np.concatenate(vals)
    assert xs.size > 50_000
    zcrit = stats.norm.isf(P_MIN / 2)
    z1, z2 = _moment_z(xs, e_true, _sigma(abcd, e_true))
    assert z1 < zcrit and z2 < zcrit
