"""Track impact parameters on the GPU (pdr_track_ip) against the oracle (the
output table of Sec. 2.5: d0, z0 and their errors for charged particles).

Each event's response is first checked against the oracle (its track list is
the oracle's, after any marginal-decision flips); every track's (d0', z0',
sigma_d0, sigma_z0) is then compared with the oracle's for the same generated
particle: within 2e-6 of the scale of each quantity (|v0| + |d0| + sigma_d0
for d0; |vz| + (|s| + |v0|) cosh(eta) + sigma_z0 for z0, s the transverse
path to the closest approach), the errors within 2e-6 relative.  Vertices are
displaced in x, y and z; the field is the card's, reversed, and zero.
"""
import json
import math

import numpy as np
import pytest

import oracle
from tests import parity as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED = 53
RES = (10e-6, 50e-6, 30e-6, 80e-6)


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


def _displaced_batch(n_events, seed):
    from paper_2606_26089_b300 import synth
    b = synth.make_batched(n_events, seed=seed)
    rng = np.random.default_rng(seed)
    n = b.n_particles
    disp = rng.random(n) < 0.4
    vx = np.where(disp, rng.normal(0.0, 0.003, n), 0.0).astype(np.float32)
    vy = np.where(disp, rng.normal(0.0, 0.003, n), 0.0).astype(np.float32)
    b.vz = rng.normal(0.0, 0.05, n).astype(np.float32)
    return b, vx, vy


def _check(B, ctx, card_json, batch, vx, vy, v0_zero=False):
    cid = ctx.card_load(card_json)
    card = oracle.load_card(card_json)
    dev = B.batch_to_device(batch)
    out = B.alloc_outputs(batch.n_events, batch.n_particles, debug=True)
    host = P.run_gpu(ctx, cid, batch, SEED, dev=dev, outs=out)
    ip = torch.full((batch.n_particles, 4), float("nan"), device="cuda")
    tvx, tvy = torch.from_numpy(vx).cuda(), torch.from_numpy(vy).cuda()
    b = B.make_batch(dev, cid, SEED, debug=True)
    ctx.track_ip(b, B.make_outputs(out), B.make_ip_params(RES, tvx, tvy), ip)
    torch.cuda.synchronize()
    ctx.check()
    ip = ip.cpu().numpy()
    prm = oracle.IPParams(*RES)
    stats = P.Stats()
    n_trk = 0
    worst = [0.0, 0.0, 0.0]
    for e in range(batch.n_events):
        ev = batch.event(e)
        ref = P.compare_event(card, ev, P.gpu_event(host, batch, e), SEED, e, stats)
        a = int(batch.offsets[e])
        ev = dict(ev, vx=vx[a:int(batch.offsets[e + 1])], vy=vy[a:int(batch.offsets[e + 1])])
        o = oracle.event_track_ip(card, prm, ev, ref, SEED, e)
        g = ip[a:a + len(ref.tracks)]
        assert not np.isnan(g).any()
        for k, i in enumerate(ref.tracks["idx"].astype(np.int64)):
            x0, y0 = float(ev["vx"][i]), float(ev["vy"][i])
            zv = 0.0 if ev.get("vz") is None else float(ev["vz"][i])
            d0, z0, s = oracle.track_ip(card, ev["pt"][i], ev["eta"][i], ev["phi"][i], ev["charge"][i], x0, y0, zv)
            if v0_zero:
                assert abs(d0) < 1e-12 and abs(s) < 1e-12   # (FP64 rounding of the circle geometry)
            v0 = math.hypot(x0, y0)
            sd = 2e-6 * (v0 + abs(d0) + o[k, 2]) + 1e-12
            sz = 2e-6 * (abs(zv) + (abs(s) + v0) * math.cosh(ev["eta"][i]) + o[k, 3]) + 1e-12
            r = (abs(g[k, 0] - o[k, 0]) / sd, abs(g[k, 1] - o[k, 1]) / sz,
                 max(abs(g[k, 2] / o[k, 2] - 1), abs(g[k, 3] / o[k, 3] - 1)) / 2e-6)
            worst = [max(x, y) for x, y in zip(worst, r)]
            assert r[0] <= 1.0 and r[1] <= 1.0 and r[2] <= 1.0, (e, k, g[k], o[k], d0, z0)
        n_trk += len(ref.tracks)
    assert n_trk > 1000
    return worst


def test_displaced_vertices_cms_like(B, ctx):
    batch, vx, vy = _displaced_batch(80, 29)
    _check(B, ctx, "cms_like", batch, vx, vy)


def test_reversed_and_zero_field(B, ctx):
    batch, vx, vy = _displaced_batch(40, 31)
    base = json.load(open(B.card_path("cms_like")))
    for field in (-3.8, 0.0):
        _check(B, ctx, dict(base, B=field, name=f"cms_like_ip_B{field}"), batch, vx, vy)


def test_vertices_on_the_axis_ee_like(B, ctx):
    """No vertex arrays at all (vz absent, vx = vy = 0): true d0 = 0, z0 = 0,
    the records are the smearing alone."""
    from paper_2606_26089_b300 import synth
    batch = synth.make_batched(20, seed=33)
    z = np.zeros(batch.n_particles, np.float32)
    _check(B, ctx, "ee_like", batch, z, z, v0_zero=True)


def test_wide_displacements_and_momenta(B, ctx):
    """Charged pions and doubly charged ions with pT from 0.12 GeV to 1 TeV
    (helix radii from 0.1 m to about 1 km), vertices from 1 um to 0.5 m off
    the axis in every direction (inside and outside the helix), |vz| up to
    0.3 m, on the CMS-like card: the closed form's cancellations at both ends
    of the range against the oracle."""
    from paper_2606_26089_b300 import synth
    rng = np.random.default_rng(71)
    events, vxs, vys = [], [], []
    for e in range(40):
        ev = []
        for k in range(80):
            q = int(rng.choice([1, -1, 2, -2]))
            pdg = {1: 211, -1: -211, 2: 1000020040, -2: -1000020040}[q]
            m = 0.13957039 if abs(q) == 1 else 3.727
            pt = float(np.exp(rng.uniform(np.log(0.12), np.log(1000.0))))
            rad, ang = float(np.exp(rng.uniform(np.log(1e-6), np.log(0.5)))), float(rng.uniform(-np.pi, np.pi))
            ev.append((pt, float(rng.uniform(-2.4, 2.4)), float(rng.uniform(-np.pi, np.pi)), m, pdg, q,
                       float(rng.uniform(-0.3, 0.3))))
            vxs.append(rad * np.cos(ang))
            vys.append(rad * np.sin(ang))
        events.append(ev)
    batch = synth.from_particles(events)
    worst = _check(B, ctx, "cms_like", batch, np.asarray(vxs, np.float32), np.asarray(vys, np.float32))
    print("wide displacements: worst d0, z0, errors (fractions of tolerance)", worst)


def test_bad_resolutions_are_rejected(B, ctx):
    from paper_2606_26089_b300 import synth
    batch = synth.make_batched(2, seed=1)
    cid = ctx.card_load("cms_like")
    dev = B.batch_to_device(batch)
    out = B.alloc_outputs(batch.n_events, batch.n_particles)
    ip = torch.empty((batch.n_particles, 4), device="cuda")
    with pytest.raises(B.PdrError):
        ctx.track_ip(B.make_batch(dev, cid, SEED), B.make_outputs(out), B.make_ip_params((-1.0, 0, 0, 0)), ip)


def test_fused_form_equals_the_separate_pass(B, ctx):
    """pdr_run_ip (impact parameters written by the response kernel's smearing
    jobs) gives the records of pdr_run followed by pdr_track_ip bit for bit,
    for every launch shape family (one-warp teams, CTA teams, the large-event
    path with optimistic shared tables) and with vertex arrays absent."""
    from paper_2606_26089_b300 import synth
    batch, vx, vy = _displaced_batch(60, 37)
    big = synth.make("pileup", n_events=2)
    for b, tvx, tvy in ((batch, vx, vy), (big, None, None)):
        cid = ctx.card_load("cms_like")
        dev = B.batch_to_device(b)
        txy = [None if v is None else torch.from_numpy(v).cuda() for v in (tvx, tvy)]
        prm = B.make_ip_params(RES, *txy)
        for team, block in ((32, 256), (256, 256), (1024, 1024)):
            l = B.pdr_launch()
            l.team, l.block, l.table_slots, l.grid = team, block, 0, 0
            o1 = B.alloc_outputs(b.n_events, b.n_particles)
            ip1 = torch.full((b.n_particles, 4), float("nan"), device="cuda")
            bt = B.make_batch(dev, cid, SEED)
            ctx.run(bt, B.make_outputs(o1), launch=l)
            ctx.track_ip(bt, B.make_outputs(o1), prm, ip1)
            o2 = B.alloc_outputs(b.n_events, b.n_particles)
            ip2 = torch.full((b.n_particles, 4), float("nan"), device="cuda")
            ctx.run_ip(bt, B.make_outputs(o2), prm, ip2, launch=l)
            torch.cuda.synchronize()
            ctx.check()
            assert torch.equal(o1["counts"], o2["counts"])
            counts = o1["counts"].cpu().numpy().view(np.uint32)
            for e in range(b.n_events):
                a, nt = int(b.offsets[e]), int(counts[e][0])
                assert torch.equal(o1["tracks"][a:a + nt].view(torch.int32), o2["tracks"][a:a + nt].view(torch.int32))
                assert torch.equal(ip1[a:a + nt].view(torch.int32), ip2[a:a + nt].view(torch.int32)), (team, e)
    with pytest.raises(B.PdrError):
        ctx.run_ip(bt, B.make_outputs(o2), B.make_ip_params((-1.0, 0, 0, 0)), ip2)
