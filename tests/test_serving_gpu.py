"""Serving loop on the GPU: continuous batching of requests of different sizes
and cards, admission by free device memory, graph-replayed waves; every
request's results equal the ones it gets alone (pdr_run, same seed and event
base), bit for bit."""
import time

import numpy as np
import pytest

from tests import parity as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26089_b300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def synth():
    from paper_2606_26089_b300 import synth as s
    return s


def _requests(synth):
    specs = []
    rng = np.random.default_rng(5)
    for k in range(14):
        wl, card = [("batched", "cms_like"), ("ee", "ee_like"), ("batched", "atlas_like"),
                    ("pileup", "cms_like"), ("tiny", "cms_like")][k % 5]
        nev = int(rng.integers(1, 60)) if wl != "pileup" else int(rng.integers(1, 4))
        specs.append((wl, card, nev, 100 + k, 1000 * k))
    return specs


def _alone(B, ctx, cid, batch, seed, base):
    return P.run_gpu(ctx, cid, batch, seed, event_base=base, debug=False)


def _compare(h_alone, h_served, batch):
    assert np.array_equal(h_alone["counts"], h_served["counts"])
    for e in range(batch.n_events):
        a = int(batch.offsets[e])
        for k, c in (("tracks", 0), ("towers", 1), ("eflow", 2), ("cands", 3), ("iso", 3)):
            n = int(h_alone["counts"][e][c])
            assert np.array_equal(h_alone[k][a:a + n].view(np.uint32), h_served[k][a:a + n].view(np.uint32)), (k, e)


@pytest.mark.parametrize("use_graphs", [1, 0])
def test_served_requests_match_alone(B, synth, use_graphs):
    ctx = B.Context(0, pool_bytes=2 << 30, max_tickets=256)
    try:
        cards = {n: ctx.card_load(n) for n in ("cms_like", "atlas_like", "ee_like")}
        specs = _requests(synth)
        batches = [synth.make(wl, n_events=nev) for wl, card, nev, seed, base in specs]
        alone = [_alone(B, ctx, cards[card], b, seed, base) for (wl, card, nev, seed, base), b in zip(specs, batches)]
        ctx.serve_start(use_graphs=use_graphs)
        keep, tickets = [], []
        for (wl, card, nev, seed, base), b in zip(specs, batches):
            hb, k = B.pinned_host_batch(b, cards[card], seed, base)
            keep.append(k)
            tickets.append(ctx.serve_submit(hb))
        for t, b, ha in zip(tickets, batches, alone):
            assert ctx.wait(t, 60_000) == 0
            hs = B.result_to_host(ctx.fetch(t))
            _compare(ha, hs, b)
            ctx.release(t)
        st = ctx.serve_stats()
        assert st["requests_done"] == len(specs)
        assert st["events_done"] == sum(b.n_events for b in batches)
        assert st["waves"] <= len(specs)
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        if use_graphs:
            assert st["graph_launches"] == st["waves"]
        ctx.serve_stop()
    finally:
        ctx.close()


def test_admission_waits_for_free_memory(B, synth):
    """With a pool that holds only a few requests, later ones wait until earlier
    ones are released, and all complete."""
    ctx = B.Context(0, pool_bytes=48 << 20, max_tickets=64)
    try:
        cid = ctx.card_load("cms_like")
        b = synth.make("batched", n_events=150)  # ~60k particles: ~9 MB of inputs and results
        ref = _alone(B, ctx, cid, b, 7, 0)
        ctx.serve_start()
        hb, keep = B.pinned_host_batch(b, cid, 7, 0)
        tickets = [ctx.serve_submit(hb) for _ in range(10)]
        for t in tickets:
            assert ctx.wait(t, 60_000) == 0
            _compare(ref, B.result_to_host(ctx.fetch(t)), b)
            ctx.release(t)
        st = ctx.serve_stats()
        assert st["requests_done"] == 10
        assert st["admission_waits"] >= 1
        ctx.serve_stop()
    finally:
        ctx.close()


def test_bounded_wait_times_out_instead_of_hanging(B, synth):
    ctx = B.Context(0, pool_bytes=256 << 20)
    try:
        cid = ctx.card_load("cms_like")
        b = synth.make("pileup", n_events=40)
        ctx.serve_start()
        hb, keep = B.pinned_host_batch(b, cid, 1, 0)
        t = ctx.serve_submit(hb)
        rc = ctx.wait(t, 0)  # immediately: still queued or running
        assert rc in (0, -4)
        assert ctx.wait(t, 60_000) == 0
        ctx.release(t)
        ctx.serve_stop()
    finally:
        ctx.close()


def test_graph_replay_keeps_its_shared_memory(B, synth):
    """Large events (whose shared tower tables are sized to fill the shared
    memory, so each event size gives its own launch shape): waves replayed
    from captured graphs after direct launches of the same kernel with other
    shared-memory sizes still run, and match the direct results."""
    ctx = B.Context(0, pool_bytes=1 << 30, max_tickets=64)
    try:
        cid = ctx.card_load("cms_like")
        batches = [synth.make_pileup(n_events=1, seed=40 + k, n_vertices=v)
                   for k, v in enumerate((100, 115, 130, 145, 160, 175))]
        ctx.serve_start(use_graphs=1)

        def serve(b):
            hb, keep = B.pinned_host_batch(b, cid, 9, 0)
            t = ctx.serve_submit(hb)
            assert ctx.wait(t, 60_000) == 0
            h = B.result_to_host(ctx.fetch(t))
            ctx.release(t)
            return h

        first = [serve(b) for b in batches]                     # each wave captures a graph
        alone = [_alone(B, ctx, cid, b, 9, 0) for b in batches]  # direct launches in between
        for b, f, a in zip(batches, first, alone):
            _compare(a, f, b)
        for b, a in zip(batches, alone):                         # the graphs replayed
            _compare(a, serve(b), b)
        st = ctx.serve_stats()
        assert st["graph_launches"] == st["waves"] == 2 * len(batches)
        ctx.serve_stop()
    finally:
        ctx.close()
