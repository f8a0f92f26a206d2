"""Jet clustering on the GPU (pdr_cluster_jets) against the oracle (Sec. 2.4:
generalized-kT clustering of the PFlow or truth collection).

For PFlow jets each event's response is first checked against the oracle;
the oracle's PFlow objects of that event (after any marginal-decision flips)
are then clustered by the oracle.  The jets must agree.  Where some step of
the oracle's clustering is a near-tie within float32 uncertainty, either
choice is correct; when an event's jets differ, the oracle is re-run with
the runner-up decision forced at its marginal steps (one, then two, then
three of them; the oracle refuses to force a step that is not marginal) and
one of those runs must then agree exactly as below - no event is skipped.
The number of events that needed a forced step is printed.  Agreement means: the
same number, each oracle jet matched by a GPU jet with the same constituent
count, pT within 4e-6 relative (each constituent carries the response's 2e-6
and a float32 rounding; constituents within R are nearly collinear), eta and
phi within 1e-5, mass squared within 1e-5 of m^2 + pT^2, and the
substructure C2 and D2 within 3e-4 relative (float32 constituent directions
carry dR errors of a few 1e-7, amplified by the ratios of sums).
"""
import numpy as np
import pytest

import oracle
from oracle import features as OF
from tests import parity as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED = 61


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
def pflow(B, ctx):
    from paper_2606_26089_b300 import synth
    batch = synth.make_batched(80, seed=41)
    cid = ctx.card_load("cms_like")
    card = oracle.load_card("cms_like")
    dev = B.batch_to_device(batch)
    out = B.alloc_outputs(batch.n_events, batch.n_particles, debug=True)
    host = P.run_gpu(ctx, cid, batch, SEED, dev=dev, outs=out)
    stats = P.Stats()
    refs = [P.compare_event(card, batch.event(e), P.gpu_event(host, batch, e), SEED, e, stats)
            for e in range(batch.n_events)]
    return batch, cid, dev, out, refs


def _gpu_jets(B, ctx, batch, dev, cid, out, params):
    jets = torch.full((max(batch.n_particles, 1), 8), float("nan"), device="cuda")
    counts = torch.full((max(batch.n_events, 1),), -1, dtype=torch.int32, device="cuda")
    b = B.make_batch(dev, cid, SEED, debug=True)
    ctx.cluster_jets(b, B.make_outputs(out) if out is not None else None, params, jets, counts)
    torch.cuda.synchronize()
    ctx.check()
    return jets.cpu().numpy(), counts.cpu().numpy()


def _compare(g, o):
    assert len(g) == len(o), (len(g), len(o))
    gn = g[:, 5].view(np.uint32)
    used = np.zeros(len(g), bool)
    for j in o:
        cand = [k for k in range(len(g)) if not used[k] and gn[k] == j["nconst"]]
        assert cand, ("no GPU jet with", j["nconst"], "constituents")
        k = min(cand, key=lambda k: abs(g[k, 1] - j["eta"]) + abs(np.angle(np.exp(1j * (g[k, 2] - j["phi"])))))
        used[k] = True
        assert abs(g[k, 0] / j["pt"] - 1) <= 4e-6, (g[k], j)
        assert abs(g[k, 1] - j["eta"]) <= 1e-5 * max(1.0, abs(j["eta"])), (g[k], j)
        assert abs(np.angle(np.exp(1j * (g[k, 2] - j["phi"])))) <= 1e-5, (g[k], j)
        assert abs(g[k, 3] ** 2 - j["mass"] ** 2) <= 1e-5 * (j["mass"] ** 2 + j["pt"] ** 2) + 1e-6, (g[k], j)
        # substructure: float32 constituent directions give dR errors of a few 1e-7
        assert abs(g[k, 6] - j["c2"]) <= 3e-4 * abs(j["c2"]) + 1e-7, ("C2", g[k], j)
        assert abs(g[k, 7] - j["d2"]) <= 3e-4 * abs(j["d2"]) + 1e-7, ("D2", g[k], j)
    # decreasing pT
    assert np.all(np.diff(g[:, 0]) <= 1e-6 * g[:-1, 0])


def _agrees(g, o):
    try:
        _compare(g, o)
        return True
    except AssertionError:
        return False


def _match(g, fm, **kw):
    """Number of forced marginal steps (0, 1, 2 or 3) under which the oracle's
    jets equal the GPU's; fails if there is none."""
    o, steps = oracle.cluster_forced(*fm, **kw)
    if _agrees(g, o):
        return 0, len(o)
    frontier = [((), steps)]
    for depth in range(1, 4):
        nxt = []
        for flips, marg in frontier:
            for st in marg:
                if flips and st <= flips[-1]:
                    continue
                f2 = flips + (st,)
                try:
                    o2, m2 = oracle.cluster_forced(*fm, flips=f2, **kw)
                except ValueError:
                    continue
                if _agrees(g, o2):
                    return depth, len(o2)
                nxt.append((f2, m2))
        frontier = nxt[:200]
        if not frontier:
            break
    _compare(g, o)  # raises with the unforced run's difference
    raise AssertionError("unreachable")


def _check_pflow(B, ctx, pflow, algorithm, R, pt_min, nconst_min):
    batch, cid, dev, out, refs = pflow
    params = B.make_jet_params("pflow", algorithm, R, pt_min, nconst_min)
    g, gc = _gpu_jets(B, ctx, batch, dev, cid, out, params)
    forced = n_jets = 0
    for e in range(batch.n_events):
        ev = batch.event(e)
        fm = OF.pflow_four_momenta(refs[e], ev)
        a = int(batch.offsets[e])
        depth, nj = _match(g[a:a + gc[e]], fm, p=params.p, R=R, pt_min=pt_min, nconst_min=nconst_min)
        forced += depth > 0
        n_jets += nj
    print(f"{algorithm} R={R}: {batch.n_events} events, {n_jets} jets, {forced} needed a forced near-tie step")
    assert n_jets > 0
    return n_jets


def test_anti_kt_pflow_paper_configuration(B, ctx, pflow):
    """PFlowJetsAntiKt05: dr 0.5, pt_min 10 GeV, at least 2 constituents."""
    _check_pflow(B, ctx, pflow, "antikt", 0.5, 10.0, 2)


def test_anti_kt_pflow_all_jets(B, ctx, pflow):
    n = _check_pflow(B, ctx, pflow, "antikt", 0.4, 0.0, 1)
    assert n > 1000


def test_cambridge_and_kt(B, ctx, pflow):
    _check_pflow(B, ctx, pflow, "cambridge", 0.8, 5.0, 1)
    _check_pflow(B, ctx, pflow, "kt", 0.6, 5.0, 1)


def test_truth_jets(B, ctx):
    from paper_2606_26089_b300 import synth
    batch = synth.make_batched(40, seed=43)
    cid = ctx.card_load("cms_like")
    dev = B.batch_to_device(batch)
    params = B.make_jet_params("truth", "antikt", 0.5, 10.0, 2)
    g, gc = _gpu_jets(B, ctx, batch, dev, cid, None, params)
    forced = 0
    for e in range(batch.n_events):
        a = int(batch.offsets[e])
        depth, _ = _match(g[a:a + gc[e]], OF.truth_four_momenta(batch.event(e)), p=-1.0, R=0.5, pt_min=10.0,
                          nconst_min=2)
        forced += depth > 0
    print(f"truth anti-kT: {batch.n_events} events, {forced} needed a forced near-tie step")


def test_bad_parameters_are_rejected(B, ctx, pflow):
    batch, cid, dev, out, refs = pflow
    b = B.make_batch(dev, cid, SEED)
    jets = torch.empty((batch.n_particles, 8), device="cuda")
    counts = torch.empty((batch.n_events,), dtype=torch.int32, device="cuda")
    with pytest.raises(B.PdrError):
        ctx.cluster_jets(b, B.make_outputs(out), B.make_jet_params(R=0.0), jets, counts)
    with pytest.raises(B.PdrError):
        ctx.cluster_jets(b, None, B.make_jet_params("pflow"), jets, counts)


def test_ee_genkt_on_ee_events(B, ctx):
    """e+e- generalized kT (energies, opening angles) on the e+e- workload's
    PFlow objects (ALEPH-like card): anti-kT-like p = -1 with R = 0.7 and the
    Durham-like p = 1 with R = pi."""
    from paper_2606_26089_b300 import synth
    batch = synth.make_ee(60, seed=47)
    cid = ctx.card_load("ee_like")
    card = oracle.load_card("ee_like")
    dev = B.batch_to_device(batch)
    out = B.alloc_outputs(batch.n_events, batch.n_particles, debug=True)
    host = P.run_gpu(ctx, cid, batch, SEED, dev=dev, outs=out)
    stats = P.Stats()
    refs = [P.compare_event(card, batch.event(e), P.gpu_event(host, batch, e), SEED, e, stats)
            for e in range(batch.n_events)]
    for p_, R in ((-1.0, 0.7), (1.0, np.pi)):
        params = B.make_jet_params("pflow", "ee-genkt", R, 0.0, 1, p=p_)
        g, gc = _gpu_jets(B, ctx, batch, dev, cid, out, params)
        n_jets = 0
        for e in range(batch.n_events):
            fm = OF.pflow_four_momenta(refs[e], batch.event(e))
            a = int(batch.offsets[e])
            _, nj = _match(g[a:a + gc[e]], fm, p=p_, R=R, pt_min=0.0, nconst_min=1, ee=True)
            n_jets += nj
        assert n_jets >= batch.n_events   # (R = pi merges each event into one jet)


def test_many_coincident_objects(B, ctx):
    """200 massless objects in one direction (pairwise distances exactly 0, so
    all but one have the same nearest neighbour: a step re-searches far more
    objects than the fixed work list holds) among a random background; the
    jets equal the oracle's."""
    from paper_2606_26089_b300 import synth
    rng = np.random.default_rng(11)
    rows = [(float(k + 1), 0.3, 1.0, 0.0, 22, 0) for k in range(200)]
    n = 120
    rows += list(zip(rng.uniform(0.5, 20.0, n), rng.uniform(-3, 3, n), rng.uniform(-np.pi, np.pi, n),
                     np.zeros(n), np.full(n, 22), np.zeros(n, int)))
    rng.shuffle(rows)
    batch = synth.from_particles([rows])
    cid = ctx.card_load("cms_like")
    dev = B.batch_to_device(batch)
    for algorithm, p_ in (("antikt", -1.0), ("kt", 1.0)):
        params = B.make_jet_params("truth", algorithm, 0.4, 0.0, 1)
        g, gc = _gpu_jets(B, ctx, batch, dev, cid, None, params)
        _match(g[:gc[0]], OF.truth_four_momenta(batch.event(0)), p=p_, R=0.4, pt_min=0.0, nconst_min=1)
        # the coincident objects end in one jet with all 200 (and maybe neighbours)
        assert int(g[:gc[0], 5].view(np.uint32).max()) >= 200


def test_clustering_boundaries(B, ctx):
    """Truth events on the clustering's boundaries, against the oracle under
    the forced-step protocol: an empty event, a single object, pairs exactly
    R apart in rapidity (merge or beam is a tie), pairs straddling phi = +-pi,
    objects far forward (|eta| = 8), massive objects (y != eta), a jet of
    exactly pt_min, for anti-kT, C/A and kT."""
    from paper_2606_26089_b300 import synth
    f32 = lambda x: float(np.float32(x))
    M = 0.13957039
    events = [
        [],
        [(20.0, 0.5, 1.0, 0.0, 22, 0)],
        [(20.0, 0.0, 0.0, 0.0, 22, 0), (15.0, 0.5, 0.0, 0.0, 22, 0), (12.0, -2.0, 1.0, 0.0, 22, 0),
         (12.0, -2.0, f32(1.0 + 0.5), 0.0, 22, 0)],
        [(25.0, 1.0, f32(3.1), 0.0, 22, 0), (18.0, 1.05, f32(-3.1), 0.0, 22, 0),
         (11.0, -1.0, f32(np.pi), 0.0, 22, 0), (9.0, -1.0, f32(-np.pi), 0.0, 22, 0)],
        [(30.0, 8.0, 0.2, 0.0, 22, 0), (30.0, -8.0, 0.2, 0.0, 22, 0), (14.0, 7.8, 0.3, M, 211, 1)],
        [(40.0, 0.3, 0.5, 5.0, 211, 1), (40.0, 0.4, 0.6, 20.0, 211, 1), (10.0, -1.5, -2.0, 0.0, 22, 0),
         (f32(9.999999), 2.0, 2.0, 0.0, 22, 0)],
    ]
    batch = synth.from_particles(events)
    cid = ctx.card_load("cms_like")
    dev = B.batch_to_device(batch)
    for algorithm, p_ in (("antikt", -1.0), ("cambridge", 0.0), ("kt", 1.0)):
        params = B.make_jet_params("truth", algorithm, 0.5, 10.0, 1)
        g, gc = _gpu_jets(B, ctx, batch, dev, cid, None, params)
        assert gc[0] == 0 and gc[1] == 1
        for e in range(batch.n_events):
            a = int(batch.offsets[e])
            _match(g[a:a + gc[e]], OF.truth_four_momenta(batch.event(e)), p=p_, R=0.5, pt_min=10.0, nconst_min=1)


def test_event_beyond_the_shared_memory_workspace_is_refused(B, ctx):
    """An event with more clustering objects than one warp's shared-memory
    workspace holds is refused on the host (no launch)."""
    from paper_2606_26089_b300 import synth
    rng = np.random.default_rng(3)
    n = 11000
    rows = list(zip(rng.uniform(0.5, 5.0, n), rng.uniform(-4, 4, n), rng.uniform(-np.pi, np.pi, n),
                    np.full(n, 0.13957), np.full(n, 211), np.ones(n, int), np.zeros(n)))
    batch = synth.from_particles([rows])
    cid = ctx.card_load("cms_like")
    dev = B.batch_to_device(batch)
    jets = torch.empty((batch.n_particles, 8), device="cuda")
    counts = torch.empty((1,), dtype=torch.int32, device="cuda")
    with pytest.raises(B.PdrError, match="shared memory"):
        ctx.cluster_jets(B.make_batch(dev, cid, SEED), None, B.make_jet_params("truth"), jets, counts)
    ctx.check()
