"""FP64 oracle (TEST INFRASTRUCTURE) of the filter pipeline and the event
features H_T and missing E_T (Sec. 2.4, event post-processing; the filter
pipeline's parameters table).  Only tests/, the smoke entry point and the
benchmark's CPU baseline may use it.

The paper describes the filter as dropping entries of a target collection in
place by declarative per-field conditions (field, op, value, abs) combined
with "all" (AND) or "any" (OR), applied before any later stage, and says the
cached event features H_T and E_T^miss are recomputed from the survivors.  It
defines neither feature; the readings coded here (and in the CUDA path) are:

* the PFlow collection is the energy-flow tracks plus the energy-flow
  neutrals of the detector response;
* H_T = sum of pT over the PFlow objects, missing E_T = minus the vector sum
  of their transverse momenta (pT cos phi, pT sin phi), and its magnitude;
* an object's fields: tracks pt = smeared pT, eta/phi = momentum direction,
  e = the track energy sqrt(pT^2 cosh^2 eta + m^2), et = pt, pdg and charge of
  the generated particle; EFlow neutrals pt = et = dE / cosh(eta_c), e = dE,
  eta/phi = the tower centre, pdg 22 from ECAL and 130 from HCAL, charge 0;
  towers pt = et = E' / cosh(eta_c), e = E', tower centre, pdg 0, charge 0;
  candidates pt, eta, phi as reconstructed, e = pt cosh(eta), et = pt, pdg
  and charge of the generated particle;
* a float field is compared in float32 (field value and threshold each
  rounded to float32), an integer field as an integer; "abs" takes the
  magnitude first; "in" / "not in" test membership in a value list; no
  conditions keep everything;
* with the features taken from the survivors, a filter on the PFlow, track
  or neutral collection changes H_T and E_T^miss; a filter on towers or
  candidates does not (they are not PFlow objects).

A float decision whose value lies within g max(|v|, |t|, 1, scale) of its
threshold is counted as marginal: the CUDA path may take it the other way.
The scale is that of the value's own rounding: for an EFlow neutral's energy
dE = E' - E_trk (a cancellation) it is max(E', E_trk), over cosh(eta_c) for
its pt and et; else 0.
"""
from typing import Optional, Sequence

import numpy as np

FIELDS = ("pt", "eta", "phi", "e", "et", "pdg", "charge")
INT_FIELDS = ("pdg", "charge")
OPS = (">", ">=", "<", "<=", "==", "!=", "in", "not in")
COLLECTIONS = ("pflow", "track", "neutral", "tower", "cand")
ECAL = 0


def _objects_tracks(ref, ev) -> dict:
    t = ref.tracks
    idx = t["idx"].astype(np.int64)
    return {"pt": t["pt"], "eta": t["eta"], "phi": t["phi"], "e": t["e"], "et": t["pt"],
            "pdg": np.asarray(ev["pdg"], np.int64)[idx], "charge": np.asarray(ev["charge"], np.int64)[idx]}


def _sorted_towers(ref, flag: str):
    t = ref.towers
    k = t[t[flag] != 0]
    return k[np.argsort(k["owner"], kind="stable")]


def _objects_neutrals(ref) -> dict:
    n = _sorted_towers(ref, "eflow_kept")
    calo = (n["key"] >> 24).astype(np.int64)
    scale = np.maximum(n["e"], n["etrk"])
    return {"pt": n["eflow_et"], "eta": n["eta_c"], "phi": n["phi_c"], "e": n["eflow_e"], "et": n["eflow_et"],
            "pdg": np.where(calo == ECAL, 22, 130).astype(np.int64), "charge": np.zeros(len(n), np.int64),
            "key": n["key"], "scale_e": scale, "scale_pt": scale / np.cosh(n["eta_c"])}


def _objects_towers(ref) -> dict:
    w = _sorted_towers(ref, "kept")
    return {"pt": w["et"], "eta": w["eta_c"], "phi": w["phi_c"], "e": w["e"], "et": w["et"],
            "pdg": np.zeros(len(w), np.int64), "charge": np.zeros(len(w), np.int64), "key": w["key"]}


def _objects_cands(ref, ev) -> dict:
    c = ref.cands
    idx = c["idx"].astype(np.int64)
    return {"pt": c["pt"], "eta": c["eta"], "phi": c["phi"], "e": c["pt"] * np.cosh(c["eta"]), "et": c["pt"],
            "pdg": np.asarray(ev["pdg"], np.int64)[idx], "charge": np.asarray(ev["charge"], np.int64)[idx]}


def objects(ref, ev) -> dict:
    """The four record collections of one event (output order) as field arrays."""
    return {"track": _objects_tracks(ref, ev), "neutral": _objects_neutrals(ref),
            "tower": _objects_towers(ref), "cand": _objects_cands(ref, ev)}


def condition(obj: dict, cond: dict, g: float):
    """(pass mask, marginal mask) of one condition {field, op, value, abs}."""
    field, op, value = cond["field"], cond["op"], cond["value"]
    use_abs = bool(cond.get("abs", False))
    if field not in FIELDS or op not in OPS:
        raise ValueError(f"bad condition {cond}")
    values = list(value) if op in ("in", "not in") else [value]
    v = np.asarray(obj[field])
    n = v.shape[0]
    marg = np.zeros(n, bool)
    if field in INT_FIELDS:
        v = np.abs(v) if use_abs else v
        ts = [int(x) for x in values]
        cmp_v = v.astype(np.int64)
    else:
        v64 = np.abs(v.astype(np.float64)) if use_abs else v.astype(np.float64)
        cmp_v = v64.astype(np.float32)
        ts = [np.float32(x) for x in values]
        scale = obj.get("scale_e" if field == "e" else "scale_pt" if field in ("pt", "et") else "", None)
        floor = np.maximum(1.0, scale) if scale is not None else 1.0
        for t in ts:
            marg |= np.abs(v64 - float(t)) <= g * np.maximum(np.maximum(np.abs(v64), abs(float(t))), floor)
    if op == ">":
        m = cmp_v > ts[0]
    elif op == ">=":
        m = cmp_v >= ts[0]
    elif op == "<":
        m = cmp_v < ts[0]
    elif op == "<=":
        m = cmp_v <= ts[0]
    elif op == "==":
        m = cmp_v == ts[0]
    elif op == "!=":
        m = cmp_v != ts[0]
    else:
        m = np.zeros(n, bool)
        for t in ts:
            m |= cmp_v == t
        if op == "not in":
            m = ~m
    return m, marg


def keep_and_marginal(obj: dict, conds: Sequence[dict], combine: str = "all", g: float = 1e-5):
    """(keep mask, marginal mask) of a filter on one collection: an object is
    marginal when any of its float conditions is."""
    n = len(obj["pt"])
    if not conds:
        return np.ones(n, bool), np.zeros(n, bool)
    if combine not in ("all", "any"):
        raise ValueError(combine)
    keep = np.ones(n, bool) if combine == "all" else np.zeros(n, bool)
    marg = np.zeros(n, bool)
    for c in conds:
        m, mg = condition(obj, c, g)
        keep = keep & m if combine == "all" else keep | m
        marg |= mg
    return keep, marg


def keep_mask(obj: dict, conds: Sequence[dict], combine: str = "all", g: float = 1e-5):
    """(keep mask, number of marginal decisions) of a filter on one collection."""
    keep, marg = keep_and_marginal(obj, conds, combine, g)
    return keep, int(marg.sum())


def event_features(ref, ev, filt: Optional[dict] = None, g: float = 1e-5, flips: Optional[dict] = None) -> dict:
    """Filter one event's collections and compute H_T, missing E_T.

    ``filt`` = {"collection": one of COLLECTIONS, "combine": "all"|"any",
    "conditions": [...], "update_event_features": bool} or None (no filter).
    ``flips`` = {collection: object positions} takes those objects' filter
    decisions the other way; each must be marginal (ValueError otherwise),
    as the response oracle refuses to flip a decision that is not.
    Returns the surviving records' positions per collection ("keep"), the
    features, the number of marginal decisions and their positions
    ("marginal_at")."""
    obj = objects(ref, ev)
    keep = {k: np.ones(len(v["pt"]), bool) for k, v in obj.items()}
    marginal_at = {k: np.zeros(0, np.int64) for k in obj}
    n_marg = 0
    coll = None
    if filt is not None:
        coll = filt.get("collection", "pflow")
        if coll not in COLLECTIONS:
            raise ValueError(coll)
        targets = ("track", "neutral") if coll == "pflow" else (coll,)
        for k in targets:
            keep[k], mg = keep_and_marginal(obj[k], filt.get("conditions", []), filt.get("combine", "all"), g)
            marginal_at[k] = np.flatnonzero(mg)
            n_marg += int(mg.sum())
            f = np.asarray((flips or {}).get(k, ()), np.int64)
            if len(f):
                if not np.all(mg[f]):
                    raise ValueError(f"flip of a {k} filter decision that is not marginal")
                keep[k][f] = ~keep[k][f]
    if flips and any(len(v) for k, v in flips.items() if k not in marginal_at or not len(marginal_at[k])):
        raise ValueError("flip of a decision the filter did not take")
    from_survivors = filt is None or bool(filt.get("update_event_features", True))
    ht = mx = my = 0.0
    scale = 0.0  # sum of the terms' rounding scales (the pT, or a neutral's scale_pt if larger)
    n_terms = 0
    for k in ("track", "neutral"):
        sel = keep[k] if from_survivors else np.ones(len(obj[k]["pt"]), bool)
        pt = np.asarray(obj[k]["pt"], np.float64)[sel]
        phi = np.asarray(obj[k]["phi"], np.float64)[sel]
        ht += float(pt.sum())
        mx -= float((pt * np.cos(phi)).sum())
        my -= float((pt * np.sin(phi)).sum())
        sc = obj[k].get("scale_pt")
        scale += float(np.maximum(np.abs(pt), sc[sel]).sum() if sc is not None else np.abs(pt).sum())
        n_terms += int(sel.sum())
    return {"keep": keep, "objects": obj, "ht": ht, "met_x": mx, "met_y": my, "met": float(np.hypot(mx, my)),
            "marginal": n_marg, "marginal_at": marginal_at, "scale": scale, "n_terms": n_terms}


def pflow_four_momenta(ref, ev):
    """(px, py, pz, E) of the PFlow objects (tracks, then EFlow neutrals, in
    output order) for the jet clustering: tracks with their smeared pT,
    momentum direction and track energy; neutrals massless at the tower
    centre with E = dE."""
    o = objects(ref, ev)
    t, n = o["track"], o["neutral"]
    pt = np.concatenate([t["pt"], n["pt"]]).astype(np.float64)
    eta = np.concatenate([t["eta"], n["eta"]]).astype(np.float64)
    phi = np.concatenate([t["phi"], n["phi"]]).astype(np.float64)
    e = np.concatenate([t["e"], n["e"]]).astype(np.float64)
    return pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta), e


INVISIBLE = (12, 14, 16)


def truth_four_momenta(ev):
    """(px, py, pz, E) of the generated particles except neutrinos, in input
    order, E = sqrt(pT^2 cosh^2(eta) + m^2)."""
    pdg = np.abs(np.asarray(ev["pdg"], np.int64))
    sel = ~np.isin(pdg, INVISIBLE)
    pt, eta, phi, m = (np.asarray(ev[k], np.float64)[sel] for k in ("pt", "eta", "phi", "mass"))
    e = np.sqrt((pt * np.cosh(eta)) ** 2 + m * m)
    return pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta), e
