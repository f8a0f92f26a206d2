"""Pins of the oracle's filter pipeline and event features (Sec. 2.4: the
filter drops entries of a collection by per-field conditions combined with
all/any; H_T and missing E_T are recomputed from the survivors).

Expected values are worked by hand for a hand-built event, or follow from
identities that do not restate the oracle's sums: partition of a collection
by complementary cuts, rotation covariance, set algebra of the operators,
float32 rounding of thresholds, and the kinematic identities of the object
fields.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import features as F
from paper_2606_26089_b300 import synth


def _hand_event():
    """Three tracks, an ECAL and an HCAL EFlow neutral, one more kept tower,
    one candidate (generated particles 0..3)."""
    trk = np.zeros(3, oracle.TRACK)
    trk["pt"] = [10.0, 20.0, 5.0]
    trk["eta"] = [0.0, 1.0, -2.4]
    trk["phi"] = [0.0, math.pi, math.pi / 2]
    trk["idx"] = [0, 1, 2]
    trk["e"] = [10.0, 20.0 * math.cosh(1.0), 5.0 * math.cosh(2.4)]
    twr = np.zeros(3, oracle.TOWER)
    twr["key"] = [0x000010, 0x01000020, 0x000030]      # ECAL, HCAL, ECAL
    twr["owner"] = [3, 1, 2]
    twr["kept"] = [1, 1, 1]
    twr["eflow_kept"] = [1, 1, 0]
    twr["eflow_et"] = [3.0, 4.0, 0.0]
    twr["eflow_e"] = [3.0 * math.cosh(0.5), 4.0, 0.0]
    twr["e"] = [5.0, 6.0, 7.0]
    twr["et"] = [4.5, 6.0, 7.0]
    twr["eta_c"] = [0.5, 0.0, 1.2]
    twr["phi_c"] = [-math.pi / 2, 0.0, 1.0]
    cand = np.zeros(1, oracle.CAND)
    cand["pt"], cand["eta"], cand["phi"], cand["idx"] = 50.0, 0.7, 2.0, 3
    ev = {"pdg": np.array([211, -211, 321, 11], np.int32), "charge": np.array([1, -1, 1, -1], np.int8),
          "mass": np.array([0.1396, 0.1396, 0.4937, 0.000511], np.float32)}
    ref = oracle.EventResult(np.zeros(4, oracle.PARTICLE), trk, twr, cand, np.zeros(0, oracle.MARGINAL), None)
    return ref, ev


def test_hand_event_features():
    ref, ev = _hand_event()
    f = F.event_features(ref, ev)
    # H_T = 10 + 20 + 5 (tracks) + 3 + 4 (EFlow neutrals; the third tower is not one)
    assert f["ht"] == pytest.approx(42.0, abs=1e-12)
    # missing E_T = -(10 (1, 0) + 20 (-1, 0) + 5 (0, 1) + 3 (0, -1) + 4 (1, 0)) = (6, -2)
    assert f["met_x"] == pytest.approx(6.0, abs=1e-12)
    assert f["met_y"] == pytest.approx(-2.0, abs=1e-12)
    assert f["met"] == pytest.approx(math.sqrt(40.0), abs=1e-12)


def test_hand_event_filters():
    ref, ev = _hand_event()
    f = F.event_features(ref, ev, {"collection": "pflow", "combine": "all",
                                   "conditions": [{"field": "pt", "op": ">", "value": 4.5}]})
    assert list(f["keep"]["track"]) == [True, True, True] and list(f["keep"]["neutral"]) == [False, False]
    assert f["ht"] == pytest.approx(35.0) and f["met_x"] == pytest.approx(10.0) and f["met_y"] == pytest.approx(-5.0)
    # |eta| > 2 or a photon-like neutral: the third track and the ECAL neutral
    f = F.event_features(ref, ev, {"collection": "pflow", "combine": "any", "conditions": [
        {"field": "eta", "op": ">", "value": 2.0, "abs": True}, {"field": "pdg", "op": "==", "value": 22}]})
    # (neutrals in the order of their lowest depositing particle: HCAL, then ECAL)
    assert list(f["keep"]["track"]) == [False, False, True] and list(f["keep"]["neutral"]) == [False, True]
    assert f["ht"] == pytest.approx(8.0) and f["met_x"] == pytest.approx(0.0, abs=1e-12)
    assert f["met_y"] == pytest.approx(-2.0)
    # charged pions only, on the track collection: neutrals untouched
    f = F.event_features(ref, ev, {"collection": "track", "conditions": [
        {"field": "pdg", "op": "in", "value": [211, -211]}]})
    assert list(f["keep"]["track"]) == [True, True, False] and f["ht"] == pytest.approx(37.0)
    # towers and candidates are not PFlow objects: the features do not move
    base = F.event_features(ref, ev)
    for coll in ("tower", "cand"):
        f = F.event_features(ref, ev, {"collection": coll, "conditions": [{"field": "pt", "op": ">", "value": 100}]})
        assert not f["keep"][coll].any() and f["ht"] == base["ht"] and f["met_x"] == base["met_x"]
    # features from the unfiltered collection when asked
    f = F.event_features(ref, ev, {"collection": "pflow", "update_event_features": False,
                                   "conditions": [{"field": "pt", "op": ">", "value": 1000}]})
    assert not f["keep"]["track"].any() and f["ht"] == base["ht"]


def test_object_fields():
    ref, ev = _hand_event()
    o = F.objects(ref, ev)
    assert list(o["neutral"]["pdg"]) == [130, 22] and list(o["neutral"]["charge"]) == [0, 0]
    assert list(o["track"]["pdg"]) == [211, -211, 321] and list(o["track"]["charge"]) == [1, -1, 1]
    assert list(o["cand"]["pdg"]) == [11]
    assert o["cand"]["e"][0] == pytest.approx(50.0 * math.cosh(0.7))
    # towers in the order of their lowest depositing particle
    assert list(o["tower"]["key"]) == [0x01000020, 0x000030, 0x000010]


def test_float32_thresholds():
    """Both the field and the threshold are rounded to float32 before the
    comparison: a field equal to float32(1.1) passes >= 1.1 and fails > 1.1."""
    obj = {"pt": np.array([np.float32(1.1), 1.1000001, 1.0999999], np.float64)}
    gt, _ = F.condition(obj, {"field": "pt", "op": ">", "value": 1.1}, 1e-5)
    ge, marg = F.condition(obj, {"field": "pt", "op": ">=", "value": 1.1}, 1e-5)
    f32 = np.float32(1.1)
    assert list(gt) == [bool(np.float32(v) > f32) for v in obj["pt"]]
    assert list(ge) == [bool(np.float32(v) >= f32) for v in obj["pt"]]
    assert gt[0] == False and ge[0] == True and marg.all()  # noqa: E712


def test_operator_set_algebra():
    rng = np.random.default_rng(4)
    obj = {"pdg": rng.choice([22, 130, 211, -211, 11, -11, 13], 500).astype(np.int64),
           "eta": rng.uniform(-5, 5, 500), "pt": rng.exponential(3.0, 500)}
    k_in, _ = F.keep_mask(obj, [{"field": "pdg", "op": "in", "value": [211, -211, 22]}])
    k_or, _ = F.keep_mask(obj, [{"field": "pdg", "op": "==", "value": v} for v in (211, -211, 22)], "any")
    k_not, _ = F.keep_mask(obj, [{"field": "pdg", "op": "not in", "value": [211, -211, 22]}])
    assert np.array_equal(k_in, k_or) and np.array_equal(k_not, ~k_in)
    k_abs, _ = F.keep_mask(obj, [{"field": "pdg", "op": "==", "value": 211, "abs": True}])
    assert np.array_equal(k_abs, np.abs(obj["pdg"]) == 211)
    # |eta| < 2.5 is eta < 2.5 and eta > -2.5 (no value sits on a bound here)
    a, _ = F.keep_mask(obj, [{"field": "eta", "op": "<", "value": 2.5, "abs": True}])
    b, _ = F.keep_mask(obj, [{"field": "eta", "op": "<", "value": 2.5}, {"field": "eta", "op": ">", "value": -2.5}])
    assert np.array_equal(a, b)
    # De Morgan: not(any(A, B)) == all(not A, not B)
    A = {"field": "pt", "op": ">", "value": 2.0}
    Bc = {"field": "eta", "op": ">", "value": 1.0}
    nA = {"field": "pt", "op": "<=", "value": 2.0}
    nB = {"field": "eta", "op": "<=", "value": 1.0}
    assert np.array_equal(~F.keep_mask(obj, [A, Bc], "any")[0], F.keep_mask(obj, [nA, nB], "all")[0])
    assert F.keep_mask(obj, [])[0].all()


@pytest.fixture(scope="module")
def real_event():
    card = oracle.load_card("cms_like")
    b = synth.make_batched(3, seed=11)
    ev = b.event(1)
    return oracle.run_event(card, ev, 5, 1), ev


def test_partition_by_complementary_cuts(real_event):
    ref, ev = real_event
    full = F.event_features(ref, ev)
    hi = F.event_features(ref, ev, {"collection": "pflow", "conditions": [{"field": "pt", "op": ">", "value": 1.0}]})
    lo = F.event_features(ref, ev, {"collection": "pflow", "conditions": [{"field": "pt", "op": "<=", "value": 1.0}]})
    assert hi["ht"] + lo["ht"] == pytest.approx(full["ht"], rel=1e-12)
    assert hi["met_x"] + lo["met_x"] == pytest.approx(full["met_x"], abs=1e-9 * full["ht"])
    assert hi["met_y"] + lo["met_y"] == pytest.approx(full["met_y"], abs=1e-9 * full["ht"])
    n = len(ref.tracks) + int((ref.towers["eflow_kept"] != 0).sum())
    assert hi["keep"]["track"].sum() + lo["keep"]["track"].sum() + hi["keep"]["neutral"].sum() + \
        lo["keep"]["neutral"].sum() == n


def test_rotation_covariance(real_event):
    """Rotating every object by alpha in phi keeps H_T and |MET| and rotates
    the MET vector by alpha."""
    ref, ev = real_event
    f0 = F.event_features(ref, ev)
    alpha = 0.7
    trk = ref.tracks.copy()
    twr = ref.towers.copy()
    trk["phi"] += alpha
    twr["phi_c"] += alpha
    rot = oracle.EventResult(ref.particles, trk, twr, ref.cands, ref.marginal, ref.counts)
    f1 = F.event_features(rot, ev)
    assert f1["ht"] == pytest.approx(f0["ht"], rel=1e-12)
    assert f1["met"] == pytest.approx(f0["met"], rel=1e-9, abs=1e-9)
    c, s = math.cos(alpha), math.sin(alpha)
    assert f1["met_x"] == pytest.approx(c * f0["met_x"] - s * f0["met_y"], abs=1e-9 * f0["ht"])
    assert f1["met_y"] == pytest.approx(s * f0["met_x"] + c * f0["met_y"], abs=1e-9 * f0["ht"])


def test_track_energy_is_the_mass_shell(real_event):
    ref, ev = real_event
    o = F.objects(ref, ev)["track"]
    m = np.asarray(ev["mass"], np.float64)[ref.tracks["idx"].astype(np.int64)]
    p = o["pt"] * np.cosh(o["eta"])
    assert np.allclose(o["e"] ** 2 - p ** 2, m ** 2, rtol=0, atol=1e-9 * np.max(o["e"] ** 2))
    n = F.objects(ref, ev)["neutral"]
    assert np.array_equal(n["pdg"] == 22, (n["key"] >> 24) == 0)
    assert np.allclose(n["pt"] * np.cosh(n["eta"]), n["e"], rtol=1e-12)


def test_marginal_filter_decisions_flip_and_others_refuse():
    """A threshold within the band g of a track's pT makes that decision
    marginal; taking it the other way drops (or keeps) exactly that track and
    moves H_T and the missing E_T by its own terms.  Flipping a decision that
    is not marginal, or one on a collection the filter does not target, is
    refused, as for the response's decisions."""
    ref, ev = _hand_event()
    spec = {"collection": "track", "conditions": [{"field": "pt", "op": ">", "value": 20.0 * (1 - 1e-6)}]}
    f = F.event_features(ref, ev, spec)
    # the 20 GeV track passes (20 > 19.99998) but sits within 1e-5 of the threshold
    assert list(f["keep"]["track"]) == [False, True, False] and list(f["marginal_at"]["track"]) == [1]
    assert f["ht"] == pytest.approx(20.0 + 3.0 + 4.0)
    g = F.event_features(ref, ev, spec, flips={"track": [1]})
    assert list(g["keep"]["track"]) == [False, False, False]
    assert g["ht"] == pytest.approx(f["ht"] - 20.0)
    # the 20 GeV track at phi = pi contributed +20 to the missing E_x
    assert g["met_x"] == pytest.approx(f["met_x"] - 20.0) and g["met_y"] == pytest.approx(f["met_y"])
    with pytest.raises(ValueError):
        F.event_features(ref, ev, spec, flips={"track": [0]})
    with pytest.raises(ValueError):
        F.event_features(ref, ev, spec, flips={"neutral": [0]})
