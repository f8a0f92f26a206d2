"""Pins for the oracle's per-event stages: towers (S5, S6), energy flow (S7),
efficiencies (S2, S4) and isolation (S8, Sec. 2.4 Eq. 1).

Hand-built events with a known answer, counting identities that hold for any
event, and binomial tests of the acceptance against the card's efficiencies.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2606_26089_b300 import synth

P_MIN = 1e-3
M_PI0 = 0.13957039
M_KL = 0.497611


def ev(rows):
    cols = list(zip(*rows))
    d = dict(pt=np.array(cols[0], np.float32), eta=np.array(cols[1], np.float32),
             phi=np.array(cols[2], np.float32), mass=np.array(cols[3], np.float32),
             pdg=np.array(cols[4], np.int32), charge=np.array(cols[5], np.int8))
    if any(len(r) > 6 for r in rows):
        d["vz"] = np.array([r[6] if len(r) > 6 else 0.0 for r in rows], np.float32)
    return d


@pytest.fixture(scope="module")
def cms():
    return oracle.load_card("cms_like")


# ---------------------------------------------------------------- tower grid
def test_tower_counts_per_card():
    c, a, e = (oracle.load_card(n) for n in ("cms_like", "atlas_like", "ee_like"))
    # CMS-like ECAL: 2 x 86 rings x 360 + 2 x 30 rings x 180; HCAL 114 x 72
    assert oracle.n_towers(c, oracle.ECAL) == 172 * 360 + 60 * 180 == 72720
    assert oracle.n_towers(c, oracle.HCAL) == 114 * 72 == 8208
    assert oracle.n_towers(a, oracle.ECAL) == 200 * 256 + 14 * 64
    assert oracle.n_towers(a, oracle.HCAL) == 98 * 64
    assert oracle.n_towers(e, oracle.ECAL) == oracle.n_towers(e, oracle.HCAL) == 100 * 126


def test_tower_ids_known_values(cms):
    E, H = oracle.ECAL, oracle.HCAL
    # eta 0.01: first positive barrel ring, after 30 endcap rings (180 phi) and
    # 86 barrel rings (360 phi) on the negative side; phi 0.001 is bin 180 of 360.
    assert oracle.tower_key(cms, E, 0.01, 0.001) == 30 * 180 + 86 * 360 + 180
    assert oracle.tower_key(cms, E, -0.01, -0.001) == 30 * 180 + 85 * 360 + 179
    # eta 2.0: endcap ring 10 of 30 (width (3 - 1.4964)/30), phi 0.5 -> bin 104 of 180
    assert oracle.tower_key(cms, E, 2.0, 0.5) == 30 * 180 + 172 * 360 + 10 * 180 + 104
    # HCAL eta 0.5 -> ring 57 + 5, phi -3.0 -> bin 1 of 72
    assert oracle.tower_key(cms, H, 0.5, -3.0) == (1 << 24) | (62 * 72 + 1)
    # outside coverage
    assert oracle.tower_key(cms, E, 3.5, 0.0) == oracle.NO_KEY
    assert oracle.tower_key(cms, H, 5.0, 0.0) == oracle.NO_KEY
    assert oracle.tower_key(cms, H, -4.96, 0.0) == oracle.NO_KEY
    # the phi seam: -pi is the first bin, just below +pi the last
    assert oracle.tower_key(cms, E, 0.01, -math.pi) == 30 * 180 + 86 * 360
    assert oracle.tower_key(cms, E, 0.01, 3.14159) == 30 * 180 + 86 * 360 + 359


def test_tower_centres(cms):
    eta_c, phi_c, ring, iphi = oracle.tower_centre(cms, 30 * 180 + 86 * 360 + 180)
    assert ring == 116 and iphi == 180
    assert abs(eta_c - 1.4964 / 86 / 2) < 1e-15
    assert abs(phi_c - math.pi / 360) < 1e-15
    eta_c, phi_c, ring, iphi = oracle.tower_centre(cms, (1 << 24) | (62 * 72 + 1))
    assert abs(eta_c - 5.5 * 0.087) < 1e-14
    assert abs(phi_c - (-math.pi + 1.5 * 2 * math.pi / 72)) < 1e-14


# ------------------------------------------------------------ hand events
def test_single_neutral_hadron_makes_one_tower(cms):
    r = oracle.run_event(cms, ev([(10.0, 0.3, 1.0, M_KL, 130, 0)]), seed=5, event=0)
    e_true = math.sqrt((10.0 * math.cosh(float(np.float32(0.3)))) ** 2 + float(np.float32(M_KL)) ** 2)
    assert len(r.towers) == 1 and len(r.tracks) == 0 and len(r.cands) == 0
    t = r.towers[0]
    assert t["key"] == oracle.tower_key(cms, oracle.HCAL, float(np.float32(0.3)), float(np.float32(1.0)))
    assert t["key"] == r.particles[0]["key"]
    assert abs(t["esum"] - e_true) < 1e-12 * e_true
    assert t["etrk"] == 0.0 and t["owner"] == 0
    assert t["eflow_e"] == t["e"]  # no track to subtract


def test_two_photons_in_one_tower_add(cms):
    rows = [(3.0, 0.500, 0.200, 0.0, 22, 0), (1.0, -2.0, 1.0, 0.0, 22, 0), (4.0, 0.503, 0.203, 0.0, 22, 0)]
    r = oracle.run_event(cms, ev(rows), seed=1, event=7)
    k0, k2 = r.particles[0]["key"], r.particles[2]["key"]
    assert k0 == k2 != oracle.NO_KEY and (k0 >> 24) == oracle.ECAL
    t = r.towers[r.towers["key"] == k0][0]
    e0 = 3.0 * math.cosh(float(np.float32(0.5)))
    e2 = 4.0 * math.cosh(float(np.float32(0.503)))
    assert abs(t["esum"] - (e0 + e2)) < 1e-12 * (e0 + e2)
    assert t["owner"] == 0
    assert len(r.towers) == 2


def test_forward_photon_goes_to_hcal_and_muon_neutrino_deposit_nothing(cms):
    rows = [(5.0, 3.5, 0.0, 0.0, 22, 0), (20.0, 0.4, 0.0, 0.1056583755, 13, -1),
            (20.0, 0.4, 1.0, 0.0, 12, 0)]
    r = oracle.run_event(cms, ev(rows), seed=0, event=0)
    assert (r.particles[0]["key"] >> 24) == oracle.HCAL
    assert r.particles[0]["flags"] & oracle.F_HCAL
    assert r.particles[1]["key"] == oracle.NO_KEY and r.particles[2]["key"] == oracle.NO_KEY
    assert r.particles[2]["flags"] == 0  # invisible: not propagated
    assert len(r.towers) == 1


def test_tower_smearing_is_keyed_by_tower_not_particle(cms):
    photon = (12.0, -0.7, 2.2, 0.0, 22, 0)
    filler = [(2.0, 1.9, -1.0, M_PI0, 211, 1), (2.0, -1.9, 1.0, M_KL, 130, 0), (1.0, 4.0, 0.0, 0.0, 12, 0)]
    a = oracle.run_event(cms, ev([photon]), seed=9, event=3)
    b = oracle.run_event(cms, ev(filler + [photon]), seed=9, event=3)
    c = oracle.run_event(cms, ev([photon]), seed=9, event=4)
    key = a.particles[0]["key"]
    ta = a.towers[a.towers["key"] == key][0]
    tb = b.towers[b.towers["key"] == key][0]
    tc = c.towers[c.towers["key"] == key][0]
    assert tb["owner"] == 3
    assert ta["e"] == tb["e"]          # same tower, same sum, same event -> same draw
    assert ta["e"] != tc["e"]          # another event number -> another draw


def test_eflow_subtracts_track_energy(cms):
    for event in range(50):
        r = oracle.run_event(cms, ev([(8.0, 0.9, -0.4, M_PI0, 211, 1)]), seed=2, event=event)
        if len(r.tracks) == 1:
            break
    else:
        pytest.fail("pion never tracked")
    tr, t = r.tracks[0], r.towers[0]
    ch = math.cosh(float(np.float32(0.9)))
    assert abs(tr["e"] - math.sqrt((tr["pt"] * ch) ** 2 + float(np.float32(M_PI0)) ** 2)) < 1e-12 * tr["e"]
    assert t["etrk"] == tr["e"]
    assert abs(t["eflow_e"] - (t["e"] - tr["e"])) < 1e-12 * t["e"]
    assert abs(t["eflow_et"] - t["eflow_e"] / math.cosh(t["eta_c"])) < 1e-12 * abs(t["eflow_e"])


def test_event_identities_on_tiny_workload(cms):
    """Conservation and bookkeeping identities on every event of a workload."""
    b = synth.make("tiny")
    for e in range(b.n_events):
        r = oracle.run_event(cms, b.event(e), seed=0, event=e)
        p = r.particles
        dep = p["key"] != oracle.NO_KEY
        # S5: deposited energy is conserved in the tower sums
        assert abs(r.towers["esum"].sum() - p["e"][dep].sum()) <= 1e-12 * p["e"][dep].sum()
        # one tower per distinct key, owner = lowest depositing index
        assert len(np.unique(p["key"][dep])) == len(r.towers)
        for t in r.towers:
            assert t["owner"] == np.flatnonzero(p["key"] == t["key"])[0]
        # track energies of tracked e/hadrons are the towers' subtracted energy
        tracked_dep = dep & ((p["flags"] & oracle.F_TRACKED) != 0)
        assert abs(r.towers["etrk"].sum() - r.tracks["e"][np.isin(r.tracks["idx"], np.flatnonzero(tracked_dep))].sum()) < 1e-9
        # thresholds: kept iff E' > E_min and E'/sigma > S_min (float32 decisions, strict)
        for t in r.towers:
            calo = t["key"] >> 24
            emin, smin = cms.e_min[calo], cms.s_min[calo]
            keep = (np.float32(t["e"]) > np.float32(emin)) and (np.float32(t["e"] / t["sigma"]) > np.float32(smin))
            assert bool(t["kept"]) == keep
        assert r.counts.n_twr_kept == int(r.towers["kept"].sum())
        # tracked particles reached the calorimeter and are charged
        tr = (p["flags"] & oracle.F_TRACKED) != 0
        assert np.all(p["flags"][tr] & oracle.F_REACH) and np.all(b.event(e)["charge"][tr] != 0)
        assert len(r.tracks) == int(tr.sum())
        assert np.all(np.diff(r.tracks["idx"].astype(np.int64)) > 0)


# ---------------------------------------------------------------- efficiencies
def _acceptance_events(rows_per_config, n_events, seed, card):
    """Run events built from the configs; return per-config (eligible, accepted) counts."""
    res = {}
    for e in range(n_events):
        rows, tags = [], []
        for tag, row in rows_per_config:
            rows.append(row)
            tags.append(tag)
        r = oracle.run_event(card, ev(rows), seed=seed, event=e, g=0.0)
        for i, tag in enumerate(tags):
            res.setdefault(tag, []).append(r.particles[i]["flags"])
    return {k: np.array(v) for k, v in res.items()}


def test_tracking_efficiency_per_bin(cms):
    # (class, pT, |eta|) -> card efficiency (CMS-like): hadron 0.70/0.60 (0.1-1 GeV), 0.95/0.85 (>1)
    configs = []
    expected = {}
    for cls_name, pdg, m, effs in (("h", 211, M_PI0, {(0.5, 1.2): 0.70, (0.5, 2.0): 0.60, (5.0, 1.2): 0.95,
                                                      (5.0, 2.0): 0.85, (5.0, 3.0): 0.0}),
                                   ("e", 11, 0.000511, {(5.0, 1.2): 0.969, (0.5, 2.0): 0.612}),
                                   ("mu", 13, 0.10566, {(5.0, 0.3): 0.9975, (5.0, 2.2): 0.8925})):
        for (pt, aeta), eff in effs.items():
            for sgn in (1, -1):
                tag = (cls_name, pt, aeta, sgn)
                q = 1 if pdg == 211 else -1
                configs.extend([(tag, (pt, sgn * aeta, 0.3 * sgn, m, pdg, q))] * 20)
                expected[tag] = eff
    flags = _acceptance_events(configs, 250, seed=11, card=cms)
    for tag, eff in expected.items():
        f = flags[tag].reshape(-1)
        reached = (f & oracle.F_REACH) != 0
        acc = (f & oracle.F_TRACKED) != 0
        n = int(reached.sum())
        assert n > 1000, tag
        k = int(acc.sum())
        if eff == 0.0:
            assert k == 0, tag
            continue
        assert stats.binomtest(k, n, eff).pvalue > P_MIN, (tag, k / n, eff)


def test_tracking_efficiency_zero_below_0p1_gev():
    # in a 0.2 T field a 0.09 GeV pion reaches the barrel (2r = 1.5 m > R) but
    # the card's first pT bin [0, 0.1) has efficiency 0
    low = oracle.load_card("cms_like")
    low.B = 0.2
    flags = _acceptance_events([("h", (0.09, 1.0, 0.5, M_PI0, 211, 1))] * 50, 40, seed=3, card=low)
    f = flags["h"].reshape(-1)
    assert np.all(f & oracle.F_REACH)
    assert not np.any(f & oracle.F_TRACKED)


def test_identification_efficiency_and_candidate_cut(cms):
    configs = []
    expected = {}
    for aeta, eff in ((0.7, 0.95), (2.0, 0.85), (2.7, 0.0)):
        tag = ("gamma", aeta)
        configs.extend([(tag, (20.0, aeta, 0.1, 0.0, 22, 0))] * 40)
        expected[tag] = eff
    configs.extend([(("gamma_low", 0.7), (9.99, 0.7, 0.1, 0.0, 22, 0))] * 40)
    flags = _acceptance_events(configs, 200, seed=13, card=cms)
    for tag, eff in expected.items():
        f = flags[tag].reshape(-1)
        eligible = (f & oracle.F_ECAL) != 0
        n, k = int(eligible.sum()), int(((f & oracle.F_CAND) != 0).sum())
        assert n == f.size
        if eff == 0.0:
            assert k == 0
        else:
            assert stats.binomtest(k, n, eff).pvalue > P_MIN, (tag, k / n, eff)
    low = flags[("gamma_low", 0.7)].reshape(-1)
    assert not np.any(low & oracle.F_CAND)  # truth pT below cand_ptmin


# ---------------------------------------------------------------- isolation
def _cone_sum_brute_force(r, cand, cand_key, card):
    """Eq. 1 written out over the oracle's own output objects."""
    total = 0.0
    for t in r.tracks:
        if t["idx"] == cand["idx"] or not t["pt"] > card.iso_ptmin:
            continue
        dphi = (t["phi"] - cand["phi"] + math.pi) % (2 * math.pi) - math.pi
        dr = math.hypot(t["eta"] - cand["eta"], dphi)
        if card.iso_drmin <= dr < card.iso_dr:
            total += t["pt"]
    for t in r.eflow:
        if t["key"] == cand_key or not t["eflow_et"] > card.iso_ptmin:
            continue
        dphi = (t["phi_c"] - cand["phi"] + math.pi) % (2 * math.pi) - math.pi
        dr = math.hypot(t["eta_c"] - cand["eta"], dphi)
        if card.iso_drmin <= dr < card.iso_dr:
            total += t["eflow_et"]
    return total


def test_isolation_hand_event(cms):
    # muon at (0, 0); pions at dR = 0.1, 0.2, 0.29 (in), 0.31 (out), 0.005 (below dR_min)
    rows = [(50.0, 0.0, 0.0, 0.1056583755, 13, -1),
            (5.0, 0.1, 0.0, M_PI0, 211, 1), (5.0, 0.0, 0.2, M_PI0, 211, 1),
            (5.0, -0.29, 0.0, M_PI0, -211, -1), (5.0, 0.0, -0.31, M_PI0, 211, 1),
            (5.0, 0.005, 0.0, M_PI0, -211, -1)]
    for event in range(400):
        r = oracle.run_event(cms, ev(rows), seed=4, event=event)
        tracked = {int(t["idx"]) for t in r.tracks}
        if len(r.cands) == 1 and tracked >= {0, 1, 2, 3, 4, 5} and len(r.eflow) == 0:
            break
    else:
        pytest.fail("no event with every particle tracked and no neutral")
    c = r.cands[0]
    assert c["idx"] == 0 and c["cls"] == 1
    pt = {int(t["idx"]): t["pt"] for t in r.tracks}
    assert abs(c["iso_sum"] - (pt[1] + pt[2] + pt[3])) < 1e-12
    assert abs(c["iso_rel"] - c["iso_sum"] / c["pt"]) < 1e-15
    assert c["isolated"] == int(c["iso_rel"] < 0.1)


def test_isolation_matches_brute_force_on_batched_events(cms):
    b = synth.make("batched", n_events=30)
    n_c = 0
    for e in range(b.n_events):
        r = oracle.run_event(cms, b.event(e), seed=1, event=e)
        for c in r.cands:
            key = r.particles[c["idx"]]["key"]
            ref = _cone_sum_brute_force(r, c, key, cms)
            assert abs(c["iso_sum"] - ref) <= 1e-9 * max(1.0, ref)
            n_c += 1
    assert n_c > 50


# ---------------------------------------------------------------- marginal decisions
def test_marginal_ring_decision_and_flip(cms):
    # a photon exactly on a float32 ring edge of the ECAL barrel (edge 0.0174 * 10)
    edge = np.float32(1.4964 / 86 * 10)
    r = oracle.run_event(cms, ev([(5.0, float(edge), 0.1, 0.0, 22, 0)]), seed=0, event=0)
    m = [x for x in r.marginal if x["kind"] == oracle.K_ETA]
    assert len(m) == 1 and m[0]["id"] == 0
    key = r.particles[0]["key"]
    f = oracle.run_event(cms, ev([(5.0, float(edge), 0.1, 0.0, 22, 0)]), seed=0, event=0,
                         flips=[(oracle.K_ETA, 0, oracle.ECAL, 0)])
    assert f.particles[0]["key"] == key - 360  # the ring below, same phi bin
    with pytest.raises(RuntimeError):
        oracle.run_event(cms, ev([(5.0, 0.123, 0.1, 0.0, 22, 0)]), seed=0, event=0,
                         flips=[(oracle.K_ETA, 0, oracle.ECAL, 0)])
