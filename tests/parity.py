"""Parity harness: CUDA path (through the C ABI) against the FP64 oracle.

Comparison protocol
-------------------
* Integer decisions that both sides take on the same float32 inputs (the
  efficiency draws u32 < floor(eff 2^32), table bins of input pT and |eta|,
  neutral tower ids from the axis origin, the barrel-reach test 2 pT >= c) must
  agree exactly.
* Decisions taken on computed floats (a charged particle's tower, barrel vs
  endcap, tower and EFlow thresholds, cone edges, I < I_max) are taken in
  float32 on both sides.  The oracle reports each one whose double value lies
  within a relative band g of its threshold as marginal.  Where the GPU took the
  other branch of a MARGINAL decision, the oracle is re-run with that decision
  flipped (the oracle refuses to flip a decision that is not marginal) and
  everything downstream must then agree.  A disagreement on a decision that is
  not marginal is a failure.
* Floats: smeared kinematics and tower energies within REL = 2e-6 relative;
  the energy-flow excess dE (a cancellation) within REL * max(E', E_track);
  propagated positions within REL * max(|eta|, 1) and REL * pi, also for
  endcap helices that have nearly closed (turning angle psi -> 2 pi), whose
  eta_pos is ill-conditioned in psi: the kernel takes pi - psi/2 in
  float-float there.
* Records come in particle order (towers and EFlow neutrals in the order of
  their lowest depositing particle), so sequences are compared exactly.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

import oracle

REL = 2e-6
G_BAND = 1e-5


@dataclass
class Stats:
    events: int = 0
    particles: int = 0
    flips: int = 0
    marginal: int = 0
    max_rel: dict = field(default_factory=dict)

    def upd(self, name, v):
        v = float(v)
        if v > self.max_rel.get(name, 0.0):
            self.max_rel[name] = v


def _rel(a, b, floor=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.maximum(np.maximum(np.abs(a), np.abs(b)), floor)
    den = np.where(den == 0, 1.0, den)
    return np.abs(a - b) / den


def _dphi(a, b):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return np.abs((d + math.pi) % (2 * math.pi) - math.pi)


def _marg(ref, kind, id_, aux=None, aux2=None):
    m = ref.marginal
    sel = (m["kind"] == kind) & (m["id"] == id_)
    if aux is not None:
        sel &= m["aux"] == aux
    if aux2 is not None:
        sel &= m["aux2"] == aux2
    return m[sel]


def _ring_phi(card, key):
    _, _, r, k = oracle.tower_centre(card, int(key))
    return r, k


class Mismatch(AssertionError):
    pass


def _particle_flips(card, ref, g, ev):
    """Decisions on particles where the GPU differs from ref (debug records)."""
    flips = []
    d = g["debug"]
    p = ref.particles
    n = len(p)
    gflags = d["flags"]
    rflags = p["flags"].astype(np.uint32)
    for i in np.flatnonzero((gflags & (oracle.F_REACH | oracle.F_BARREL)) != (rflags & (oracle.F_REACH | oracle.F_BARREL))):
        gb = bool(gflags[i] & oracle.F_BARREL)
        rb = bool(rflags[i] & oracle.F_BARREL)
        if gb != rb and len(_marg(ref, oracle.K_BARREL, i)):
            flips.append((oracle.K_BARREL, int(i), 0, 0))
        elif len(_marg(ref, oracle.K_LOOP, i)):
            flips.append((oracle.K_LOOP, int(i), 0, 0))
        else:
            raise Mismatch(f"particle {i}: reach/barrel differ (gpu {gflags[i]:#x}, oracle {rflags[i]:#x}) "
                           f"and no marginal decision explains it; pt={ev['pt'][i]} eta={ev['eta'][i]} "
                           f"q={ev['charge'][i]} pdg={ev['pdg'][i]}")
    if flips:
        return flips
    for i in np.flatnonzero(d["key"] != p["key"]):
        gk, rk = int(d["key"][i]), int(p["key"][i])
        if gk == oracle.NO_KEY or rk == oracle.NO_KEY or (gk >> 24) != (rk >> 24):
            # calorimeter coverage: an eta-ring decision at a coverage edge
            m = _marg(ref, oracle.K_ETA, i)
            if not len(m):
                raise Mismatch(f"particle {i}: tower {gk:#x} vs oracle {rk:#x}, no marginal coverage decision")
            flips.append((oracle.K_ETA, int(i), int(m[0]["aux"]), 0))
            continue
        calo = rk >> 24
        gr, gp = _ring_phi(card, gk)
        rr, rp = _ring_phi(card, rk)
        if gr != rr:
            if not len(_marg(ref, oracle.K_ETA, i, calo)):
                raise Mismatch(f"particle {i}: ring {gr} vs oracle {rr} (eta_pos gpu {d['eta_pos'][i]!r}, "
                               f"oracle {p['eta_pos'][i]!r}), not marginal")
            flips.append((oracle.K_ETA, int(i), calo, 0))
        elif gp != rp:
            if not len(_marg(ref, oracle.K_PHI, i, calo)):
                raise Mismatch(f"particle {i}: phi bin {gp} vs oracle {rp} (phi_pos gpu {d['phi_pos'][i]!r}, "
                               f"oracle {p['phi_pos'][i]!r}), not marginal")
            flips.append((oracle.K_PHI, int(i), calo, 0))
    return flips


def _threshold_flips(ref, gkeys, kind_e, kind_s, kept_field):
    flips = []
    t = ref.towers
    rk = set(int(k) for k in t["key"][t[kept_field] != 0])
    gk = set(int(k) for k in gkeys)
    for key in sorted(rk ^ gk):
        want = key in gk  # the GPU kept it
        cands = []
        for kind in (kind_e, kind_s):
            m = _marg(ref, kind, key)
            if len(m) and bool(m[0]["taken"]) != want:
                cands.append((kind, key, 0, 0))
        if not cands:
            raise Mismatch(f"tower {key:#x}: kept={want} on GPU, oracle differs, no marginal threshold")
        flips.extend(cands[:1] if want is False else cands)
    return flips


def _iso_flips(ref, g):
    flips = []
    gc = g["cands"]
    for j, c in enumerate(ref.cands):
        gs = float(gc["iso_sum"][j])
        diff = gs - c["iso_sum"]
        if abs(diff) <= REL * max(abs(gs), abs(c["iso_sum"]), 1e-3) + 1e-6:
            gi = bool(gc["info"][j] >> 31)
            if gi != bool(c["isolated"]):
                if not len(_marg(ref, oracle.K_ISOLATED, int(c["idx"]))):
                    raise Mismatch(f"candidate {c['idx']}: isolated flag differs, I={c['iso_rel']}, not marginal")
                flips.append((oracle.K_ISOLATED, int(c["idx"]), 0, 0))
            continue
        m = ref.marginal
        pm = m[((m["kind"] == oracle.K_ISO_DR) | (m["kind"] == oracle.K_ISO_DRMIN)) & (m["id"] == c["idx"])]
        om = m[m["kind"] == oracle.K_ISO_PT]
        options = [((int(x["kind"]), int(x["id"]), int(x["aux"]), int(x["aux2"])),
                    -x["w"] if x["taken"] else x["w"]) for x in pm]
        if len(options) > 12:
            raise Mismatch(f"candidate {c['idx']}: too many marginal pairs")
        found = None
        for r in range(1, len(options) + 1):
            for sub in itertools.combinations(options, r):
                if abs(c["iso_sum"] + sum(w for _, w in sub) - gs) <= REL * max(abs(gs), 1e-3) + 1e-6:
                    found = [f for f, _ in sub]
                    break
            if found:
                break
        if found is None and len(om):
            raise Mismatch(f"candidate {c['idx']}: iso sum {gs} vs oracle {c['iso_sum']} "
                           f"(marginal object pT cuts present: {len(om)})")
        if found is None:
            raise Mismatch(f"candidate {c['idx']}: iso sum {gs} vs oracle {c['iso_sum']}, "
                           f"no marginal cone decision explains it")
        flips.extend(found)
    return flips


def compare_event(card, ev: dict, g: dict, seed: int, event: int, stats: Stats, g_band=G_BAND):
    """Check one event's GPU records against the oracle (raises Mismatch)."""
    flips = []
    for _ in range(10):
        ref = oracle.run_event(card, ev, seed, event, g=g_band, flips=flips)
        new = []
        if "debug" in g:
            new = _particle_flips(card, ref, g, ev)
        if not new:
            new = _threshold_flips(ref, g["towers"]["key"], oracle.K_TWR_E, oracle.K_TWR_S, "kept")
            new += _threshold_flips(ref, g["eflow"]["key"], oracle.K_EF_E, oracle.K_EF_S, "eflow_kept")
        if not new and len(ref.cands) == len(g["cands"]["pt"]):
            new = _iso_flips(ref, g)
        if not new:
            break
        flips += new
    else:
        raise Mismatch("flip iteration did not converge")
    stats.flips += len(flips)
    stats.marginal += len(ref.marginal)
    stats.events += 1
    stats.particles += len(ev["pt"])
    p = ref.particles
    n = len(p)
    # ---- per particle
    if "debug" in g:
        d = g["debug"]
        assert np.array_equal(d["key"], p["key"]), "tower keys"
        gf = d["flags"] & 0x3F
        assert np.array_equal(gf, p["flags"].astype(np.uint32)), \
            f"flags differ at {np.flatnonzero(gf != p['flags'])[:5]}"
        reach = (p["flags"] & oracle.F_REACH) != 0
        tol_e = REL * np.maximum(np.abs(p["eta_pos"][reach]), 1.0)
        ge, oe = d["eta_pos"][reach].astype(np.float64), p["eta_pos"][reach]
        # (a helix that ends on the axis at the endcap has eta_pos = +-inf on both sides)
        with np.errstate(invalid="ignore"):
            e_err = np.where(ge == oe, 0.0, np.abs(ge - oe) / tol_e * REL)
        p_err = _dphi(d["phi_pos"][reach], p["phi_pos"][reach]) / math.pi
        if reach.any():
            # (the largest conditioning of eta_pos on the turning angle seen:
            # context for the eta_pos error, not an error itself)
            stats.upd("eta_pos_cond", p["cond"][reach].max())
            stats.upd("eta_pos", e_err.max())
            stats.upd("phi_pos", p_err.max())
            assert e_err.max() <= REL, f"eta_pos error {e_err.max()}"
            assert p_err.max() <= REL, f"phi_pos error {p_err.max()}"
    # ---- tracks
    gt, rt = g["tracks"], ref.tracks
    assert np.array_equal(gt["idx"], rt["idx"]), "track indices"
    assert np.array_equal(gt["eta"], rt["eta"].astype(np.float32)) and np.array_equal(gt["phi"], rt["phi"].astype(np.float32))
    if len(rt):
        r = _rel(gt["pt"], rt["pt"])
        stats.upd("track_pt", r.max())
        assert r.max() <= REL, f"track pT error {r.max()}"
    # ---- towers (kept), in owner order
    t = ref.towers
    kt = t[t["kept"] != 0]
    kt = kt[np.argsort(kt["owner"], kind="stable")]
    gw = g["towers"]
    assert np.array_equal(gw["key"], kt["key"]), "tower keys / order"
    if len(kt):
        r = np.maximum(_rel(gw["e"], kt["e"]), _rel(gw["et"], kt["et"]))
        stats.upd("tower_e", r.max())
        assert r.max() <= REL, f"tower energy error {r.max()}"
    # ---- EFlow neutrals
    ef = t[t["eflow_kept"] != 0]
    ef = ef[np.argsort(ef["owner"], kind="stable")]
    gf_ = g["eflow"]
    assert np.array_equal(gf_["key"], ef["key"]), "EFlow keys / order"
    if len(ef):
        scale = np.maximum(ef["e"], ef["etrk"])
        r = np.abs(gf_["e"] - ef["eflow_e"]) / scale
        r2 = np.abs(gf_["et"] - ef["eflow_et"]) / (scale / np.cosh(ef["eta_c"]))
        stats.upd("eflow_e", max(r.max(), r2.max()))
        assert r.max() <= REL and r2.max() <= REL, f"EFlow energy error {r.max()} {r2.max()}"
    # ---- candidates and isolation
    gc, rc = g["cands"], ref.cands
    assert np.array_equal(gc["info"] & 0x0FFFFFFF, rc["idx"]), "candidate indices"
    assert np.array_equal((gc["info"] >> 28) & 3, rc["cls"]), "candidate classes"
    assert np.array_equal(gc["info"] >> 31, rc["isolated"]), "isolation flags"
    if len(rc):
        r = _rel(gc["pt"], rc["pt"])
        stats.upd("cand_pt", r.max())
        assert r.max() <= REL, f"candidate pT error {r.max()}"
        r = np.abs(gc["iso_sum"] - rc["iso_sum"]) / np.maximum(np.abs(rc["iso_sum"]), 1e-3)
        stats.upd("iso_sum", r.max())
        assert r.max() <= REL, f"isolation sum error {r.max()}"
        r = np.abs(gc["iso_rel"] - rc["iso_rel"]) / np.maximum(np.abs(rc["iso_rel"]), 1e-6)
        assert r.max() <= 2 * REL, f"isolation ratio error {r.max()}"
    return ref


# ---------------------------------------------------------------------------
# running the CUDA path
# ---------------------------------------------------------------------------
def run_gpu(ctx, card_id, batch, seed, event_base=0, debug=True, launch=None, per_event=False, outs=None,
            dev=None):
    """Run a synth.EventBatch through pdr_run and return host copies (slot layout)."""
    import torch
    from paper_2606_26089_b300 import binding as B
    dev = dev or B.batch_to_device(batch)
    o = outs or B.alloc_outputs(batch.n_events, batch.n_particles, debug=debug)
    b = B.make_batch(dev, card_id, seed, event_base, debug=debug)
    if per_event:
        ctx.run_per_event(b, B.make_outputs(o))
    else:
        ctx.run(b, B.make_outputs(o), launch=launch)
    torch.cuda.synchronize()
    ctx.check()
    host = {k: (v.cpu().numpy() if v is not None else None) for k, v in o.items()}
    host["counts"] = host["counts"].view(np.uint32)[:batch.n_events]
    return host


def gpu_event(host, batch, e):
    from paper_2606_26089_b300 import binding as B
    return B.event_records(host, host["counts"], batch.offsets, e)


def check_counts_sane(host, batch):
    n = batch.multiplicities()
    c = host["counts"].astype(np.int64)
    assert np.all(c >= 0) and np.all(c <= n[:, None]), "counts exceed multiplicities"
