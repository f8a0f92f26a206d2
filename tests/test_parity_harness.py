"""CPU check of the parity harness itself (tests/parity.py).

Records built from the oracle's own output, rounded to float32 and laid out the
way the CUDA library writes them, must pass the comparison; planted mistakes
(a wrong tower, a perturbed energy, a dropped track, a non-marginal decision
taken the other way) must fail it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_26089_b300 import synth
from tests import parity as P


def records_from_oracle(ref, n):
    """The oracle's event as float32 records in the library's output order."""
    f32 = lambda x: np.asarray(x, np.float32)
    t = ref.towers
    kt = t[t["kept"] != 0]
    kt = kt[np.argsort(kt["owner"], kind="stable")]
    ef = t[t["eflow_kept"] != 0]
    ef = ef[np.argsort(ef["owner"], kind="stable")]
    p = ref.particles
    return dict(
        tracks=dict(pt=f32(ref.tracks["pt"]), eta=f32(ref.tracks["eta"]), phi=f32(ref.tracks["phi"]),
                    idx=ref.tracks["idx"].astype(np.uint32)),
        towers=dict(key=kt["key"].astype(np.uint32), e=f32(kt["e"]), et=f32(kt["et"])),
        eflow=dict(key=ef["key"].astype(np.uint32), e=f32(ef["eflow_e"]), et=f32(ef["eflow_et"])),
        cands=dict(pt=f32(ref.cands["pt"]), eta=f32(ref.cands["eta"]), phi=f32(ref.cands["phi"]),
                   info=(ref.cands["idx"] | (ref.cands["cls"] << 28) | (ref.cands["isolated"] << 31)).astype(np.uint32),
                   iso_sum=f32(ref.cands["iso_sum"]), iso_rel=f32(ref.cands["iso_rel"])),
        debug=dict(key=p["key"].astype(np.uint32), eta_pos=f32(p["eta_pos"]), phi_pos=f32(p["phi_pos"]),
                   flags=p["flags"].astype(np.uint32)),
    )


@pytest.fixture(scope="module")
def events():
    card = oracle.load_card("cms_like")
    b = synth.make("batched", n_events=6)
    return card, b


def test_oracle_records_pass(events):
    card, b = events
    st = P.Stats()
    for e in range(b.n_events):
        ref = oracle.run_event(card, b.event(e), 1, e)
        P.compare_event(card, b.event(e), records_from_oracle(ref, len(ref.particles)), 1, e, st)
    assert st.events == b.n_events


def _mutated(events, fn):
    card, b = events
    e = 2
    ref = oracle.run_event(card, b.event(e), 1, e)
    g = records_from_oracle(ref, len(ref.particles))
    fn(g, ref)
    with pytest.raises(AssertionError):
        P.compare_event(card, b.event(e), g, 1, e, P.Stats())


def test_perturbed_tower_energy_fails(events):
    def f(g, ref):
        g["towers"]["e"][3] *= np.float32(1 + 1e-5)
    _mutated(events, f)


def test_wrong_particle_tower_fails(events):
    def f(g, ref):
        i = int(np.flatnonzero(g["debug"]["key"] != oracle.NO_KEY)[5])
        g["debug"]["key"][i] += 1  # neighbouring phi bin, far from any edge
    _mutated(events, f)


def test_dropped_track_fails(events):
    def f(g, ref):
        for k in g["tracks"]:
            g["tracks"][k] = g["tracks"][k][1:]
    _mutated(events, f)


def test_wrong_isolation_sum_fails(events):
    def f(g, ref):
        g["cands"]["iso_sum"][0] += np.float32(0.5)
    _mutated(events, f)


def test_tower_order_matters(events):
    def f(g, ref):
        for k in g["towers"]:
            g["towers"][k] = g["towers"][k][::-1].copy()
    _mutated(events, f)


def test_marginal_flip_is_accepted():
    """A photon exactly on a ring edge: the other ring is accepted, with the
    downstream tower re-derived by the oracle on that branch."""
    card = oracle.load_card("cms_like")
    edge = float(np.float32(1.4964 / 86 * 10))
    ev = dict(pt=np.array([5.0, 2.0], np.float32), eta=np.array([edge, -1.0], np.float32),
              phi=np.array([0.1, 2.0], np.float32), mass=np.zeros(2, np.float32),
              pdg=np.array([22, 22], np.int32), charge=np.zeros(2, np.int8))
    flipped = oracle.run_event(card, ev, 3, 0, flips=[(oracle.K_ETA, 0, oracle.ECAL, 0)])
    g = records_from_oracle(flipped, 2)
    P.compare_event(card, ev, g, 3, 0, P.Stats())
