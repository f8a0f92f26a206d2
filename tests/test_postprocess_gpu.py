"""Filter pipeline and event features on the GPU (pdr_postprocess) against
the oracle (Sec. 2.4: a filter drops a collection's failing entries in place;
H_T and missing E_T of the PFlow collection are recomputed from the
survivors).

Each event's detector response is first checked against the oracle as in the
response parity tests; the oracle's records of that event (after any
marginal-decision flips) then go through the oracle's filter and features.
Surviving records must be the same records in the same order (track
indices, tower keys, candidate indices bit for bit); H_T and the missing E_T
components must agree within 3e-6 of the sum of the terms' magnitudes plus
the fixed-point quantum per term: each term carries the response's 2e-6
relative error, the hardware sine/cosine's 4e-7 absolute error on |phi| <=
pi, 2e-7 from a tower centre's float32 azimuth and a rounding of the
product.  A filter decision whose value lies within the band g of its
threshold is marginal: where the GPU took one the other way (seen in the
surviving records), the oracle is re-run with that decision flipped, and it
refuses to flip one that is not marginal; without compaction, where the
survivors are not visible, the features must match the oracle's with some
combination of the event's marginal decisions flipped.  No event is skipped;
the marginal and flip counts are printed.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import features as OF
from tests import parity as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED = 41


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26089_b300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def setup(B, ctx):
    from paper_2606_26089_b300 import synth
    batch = synth.make_batched(120, seed=23)
    cid = ctx.card_load("cms_like")
    card = oracle.load_card("cms_like")
    dev = B.batch_to_device(batch)
    # the oracle's records of every event, checked against the GPU's response
    host = P.run_gpu(ctx, cid, batch, SEED, dev=dev)
    stats = P.Stats()
    refs = [P.compare_event(card, batch.event(e), P.gpu_event(host, batch, e), SEED, e, stats)
            for e in range(batch.n_events)]
    return batch, cid, dev, refs


def _run(B, ctx, setup, spec, compact=True):
    batch, cid, dev, refs = setup
    outs = B.alloc_outputs(batch.n_events, batch.n_particles, debug=True)
    b = B.make_batch(dev, cid, SEED, debug=True)
    ctx.run(b, B.make_outputs(outs))
    feats = torch.zeros((batch.n_events, 4), dtype=torch.float32, device="cuda")
    filt = None if spec is None else B.make_filter(spec, compact=compact)
    ctx.postprocess(b, B.make_outputs(outs), filt, feats)
    torch.cuda.synchronize()
    ctx.check()
    host = {k: (v.cpu().numpy() if v is not None else None) for k, v in outs.items()}
    host["counts"] = host["counts"].view(np.uint32)[:batch.n_events]
    return host, feats.cpu().numpy()


def _gpu_keep(o, ref, g):
    """The GPU's filter decisions on the oracle's objects, from its surviving records."""
    return {"track": np.isin(ref.tracks["idx"], g["tracks"]["idx"]),
            "neutral": np.isin(o["objects"]["neutral"]["key"], g["eflow"]["key"]),
            "tower": np.isin(o["objects"]["tower"]["key"], g["towers"]["key"]),
            "cand": np.isin(ref.cands["idx"], g["cands"]["info"] & 0x0FFFFFFF)}


def _features_ok(o, f):
    tol = 3e-6 * o["scale"] + o["n_terms"] * 2.0**-25 + 1e-6
    return (abs(f[0] - o["ht"]) <= tol + 6e-8 * o["ht"] and abs(f[1] - o["met_x"]) <= tol + 6e-8 * abs(o["met_x"])
            and abs(f[2] - o["met_y"]) <= tol + 6e-8 * abs(o["met_y"])
            and abs(f[3] - o["met"]) <= 1.5 * tol + 6e-8 * o["met"])


def _check(B, ctx, setup, spec, compact=True):
    batch, cid, dev, refs = setup
    host, feats = _run(B, ctx, setup, spec, compact)
    n_marg = n_flip = 0
    for e in range(batch.n_events):
        ev = batch.event(e)
        o = OF.event_features(refs[e], ev, spec)
        g = B.event_records(host, host["counts"], batch.offsets, e)
        n_marg += o["marginal"]
        if o["marginal"] and spec is not None:
            if compact:
                # the decisions the GPU took the other way (the oracle refuses non-marginal ones)
                gk = _gpu_keep(o, refs[e], g)
                flips = {k: np.flatnonzero(gk[k] != o["keep"][k]) for k in o["marginal_at"]}
                flips = {k: v for k, v in flips.items() if len(v)}
                if flips:
                    o = OF.event_features(refs[e], ev, spec, flips=flips)
                    n_flip += sum(len(v) for v in flips.values())
            elif spec.get("update_event_features", True):
                # survivors not visible: some combination of marginal flips must give the GPU's features
                at = [(k, int(j)) for k, v in o["marginal_at"].items() for j in v]
                assert len(at) <= 10, (e, len(at))
                for r in range(len(at) + 1):
                    for sub in itertools.combinations(at, r):
                        fl = {}
                        for k, j in sub:
                            fl.setdefault(k, []).append(j)
                        oc = OF.event_features(refs[e], ev, spec, flips=fl) if fl else o
                        if _features_ok(oc, feats[e]):
                            o = oc
                            n_flip += r
                            break
                    else:
                        continue
                    break
        keep = o["keep"] if compact or spec is None else {k: np.ones_like(v) for k, v in o["keep"].items()}
        assert np.array_equal(g["tracks"]["idx"], refs[e].tracks["idx"][keep["track"]]), (e, "tracks")
        assert np.array_equal(g["eflow"]["key"], o["objects"]["neutral"]["key"][keep["neutral"]]), (e, "neutrals")
        assert np.array_equal(g["towers"]["key"], o["objects"]["tower"]["key"][keep["tower"]]), (e, "towers")
        assert np.array_equal(g["cands"]["info"] & 0x0FFFFFFF, refs[e].cands["idx"][keep["cand"]]), (e, "cands")
        if len(g["cands"]["pt"]):
            # isolation records move with their candidates
            r = np.abs(g["cands"]["iso_sum"] - refs[e].cands["iso_sum"][keep["cand"]])
            assert np.all(r <= 2e-6 * np.maximum(np.abs(refs[e].cands["iso_sum"][keep["cand"]]), 1e-3)), e
        tol = 3e-6 * o["scale"] + o["n_terms"] * 2.0**-25 + 1e-6
        assert abs(feats[e, 0] - o["ht"]) <= tol + 6e-8 * o["ht"], (e, feats[e, 0], o["ht"])
        assert abs(feats[e, 1] - o["met_x"]) <= tol + 6e-8 * abs(o["met_x"]), (e, feats[e, 1], o["met_x"])
        assert abs(feats[e, 2] - o["met_y"]) <= tol + 6e-8 * abs(o["met_y"]), (e, feats[e, 2], o["met_y"])
        assert abs(feats[e, 3] - o["met"]) <= 1.5 * tol + 6e-8 * o["met"], (e, feats[e, 3], o["met"])
    print(f"filter {spec and spec.get('collection')}: {batch.n_events} events, marginal filter decisions "
          f"{n_marg}, flipped {n_flip}")
    return host, feats


def test_features_without_filter(B, ctx, setup):
    host, feats = _check(B, ctx, setup, None)
    assert np.all(feats[:, 0] > 0)


def test_pflow_kinematic_cuts_compacted(B, ctx, setup):
    spec = {"collection": "pflow", "combine": "all", "conditions": [
        {"field": "pt", "op": ">", "value": 1.0}, {"field": "eta", "op": "<", "value": 2.5, "abs": True}]}
    host, feats = _check(B, ctx, setup, spec)
    assert host["counts"][:, 0].sum() > 0


def test_species_sets_and_any(B, ctx, setup):
    _check(B, ctx, setup, {"collection": "track", "combine": "any", "conditions": [
        {"field": "pdg", "op": "in", "value": [211, -211, 11]}, {"field": "e", "op": ">=", "value": 20.0}]})
    _check(B, ctx, setup, {"collection": "pflow", "conditions": [
        {"field": "pdg", "op": "not in", "value": [22]}, {"field": "charge", "op": "!=", "value": 0}]})


def test_neutral_energy_cut(B, ctx, setup):
    _check(B, ctx, setup, {"collection": "neutral", "conditions": [{"field": "e", "op": ">", "value": 2.0}]})


def test_towers_and_candidates_leave_the_features(B, ctx, setup):
    h0, f0 = _run(B, ctx, setup, None)
    host, feats = _check(B, ctx, setup, {"collection": "tower", "conditions": [
        {"field": "et", "op": ">", "value": 1.0}]})
    assert np.array_equal(feats, f0)
    host, feats = _check(B, ctx, setup, {"collection": "cand", "conditions": [
        {"field": "pt", "op": ">", "value": 40.0}, {"field": "pdg", "op": "==", "value": 22, "abs": True}],
        "combine": "any"})
    assert np.array_equal(feats, f0)


def test_features_from_all_and_no_compaction(B, ctx, setup):
    batch = setup[0]
    h0, f0 = _run(B, ctx, setup, None)
    spec = {"collection": "pflow", "conditions": [{"field": "pt", "op": ">", "value": 2.0}],
            "update_event_features": False}
    host, feats = _check(B, ctx, setup, spec)
    assert np.array_equal(feats, f0)
    host, feats = _check(B, ctx, setup, {"collection": "pflow", "conditions": [
        {"field": "pt", "op": ">", "value": 2.0}]}, compact=False)
    assert np.array_equal(host["counts"], h0["counts"])   # records untouched
    assert np.all(feats[:, 0] <= f0[:, 0])


def test_bad_filters_are_rejected(B, ctx, setup):
    batch, cid, dev, refs = setup
    outs = B.alloc_outputs(batch.n_events, batch.n_particles)
    b = B.make_batch(dev, cid, SEED)
    f = B.make_filter({"conditions": [{"field": "pt", "op": ">", "value": 1.0}]})
    f.cond[0].op = 99
    with pytest.raises(B.PdrError):
        ctx.postprocess(b, B.make_outputs(outs), f, None)
    f = B.make_filter({"conditions": [{"field": "pdg", "op": "==", "value": 1.0}]})
    f.cond[0].values[0] = 211.5
    with pytest.raises(B.PdrError):
        ctx.postprocess(b, B.make_outputs(outs), f, None)
    f = B.make_filter({"conditions": [{"field": "pt", "op": ">", "value": 1.0}]})
    f.n_conditions = 9
    with pytest.raises(B.PdrError):
        ctx.postprocess(b, B.make_outputs(outs), f, None)


def test_decisions_at_the_threshold_go_through_the_flip_protocol(B, ctx, setup):
    """Thresholds equal to the oracle's own float32 pT of chosen tracks: those
    decisions are marginal by construction, the GPU's smeared pT (within 2e-6)
    may fall on either side, and every decision it takes the other way must be
    one the oracle accepts flipped; compacted and not."""
    batch, cid, dev, refs = setup
    picks = [(e, j) for e in range(0, batch.n_events, 17) for j in (0, 3) if len(refs[e].tracks) > j][:8]
    conds = [{"field": "pt", "op": "==", "value": float(np.float32(refs[e].tracks["pt"][j]))} for e, j in picks]
    spec = {"collection": "track", "combine": "any", "conditions": conds}
    for compact in (True, False):
        host, feats = _check(B, ctx, setup, spec, compact=compact)
    n_marg = sum(OF.event_features(refs[e], batch.event(e), spec)["marginal"] for e in range(batch.n_events))
    assert n_marg >= len(picks)
