"""pdr_run_noalloc: the entry point for callers that may not allocate device
memory when they run the response (applications that own all device memory
through a fixed-budget allocator, latency-critical paths that cannot absorb an
allocation's synchronisation).  It keeps the card, an error word and the
tower tables of oversized events in one static device array inside the
library.

The main test calls it twice in a row through the C ABI on a batch whose
largest event overflows the shared-memory tower table (so the static array's
tables are used, and the second call starts from the first call's leftovers)
and checks each result against pdr_run, the allocating entry point, within
the tolerance the parity tests use; it also checks that the second call takes
no device memory.  The other tests cover the documented error returns: an
event above 49152 particles, an understated max_event_size and malformed CSR
offsets.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 2e-6


def _batch():
    from paper_2606_26089_b300 import synth
    big = synth.make("pileup", n_events=3)
    rows = []
    for e in range(3):
        ev = big.event(e)
        rows += list(zip(ev["pt"], ev["eta"], ev["phi"], ev["mass"], ev["pdg"], ev["charge"], ev["vz"]))
    small = synth.make("batched", n_events=40)
    events = [list(zip(*(small.event(e)[k] for k in ("pt", "eta", "phi", "mass", "pdg", "charge"))))
              for e in range(40)]
    events.insert(17, [r[:6] for r in rows[:12000]])  # far beyond the 8192-slot shared table
    return synth.from_particles(events)


def _host(o, n_events):
    h = {k: (v.cpu().numpy() if v is not None else None) for k, v in o.items()}
    h["counts"] = h["counts"].view(np.uint32)[:n_events]
    return h


def _close(a, b, what):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.maximum(np.maximum(np.abs(a), np.abs(b)), 1e-30)
    assert np.all(np.abs(a - b) / den <= REL), what


def test_noalloc_matches_pdr_run_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26089_b300 import binding as B
    from paper_2606_26089_b300 import build
    build.build()
    L = B.lib()
    L.pdr_run_noalloc.argtypes = [ctypes.POINTER(B.pdr_card), ctypes.POINTER(B.pdr_batch),
                                  ctypes.POINTER(B.pdr_outputs), ctypes.c_void_p]
    L.pdr_run_noalloc.restype = ctypes.c_int
    b = _batch()
    assert int(b.multiplicities().max()) == 12000
    card = B.card_from_json("cms_like")
    dev = B.batch_to_device(b)
    stream = torch.cuda.current_stream().cuda_stream

    # reference: the allocating entry point
    ctx = B.Context(0, pool_bytes=256 << 20)
    try:
        cid = ctx.card_load(card)
        ref_o = B.alloc_outputs(b.n_events, b.n_particles)
        ctx.run(B.make_batch(dev, cid, 21), B.make_outputs(ref_o))
        torch.cuda.synchronize()
        ctx.check()
        ref = _host(ref_o, b.n_events)
    finally:
        ctx.close()

    for call in range(2):
        o = B.alloc_outputs(b.n_events, b.n_particles)
        batch = B.make_batch(dev, 0, 21, max_event_size=0 if call == 0 else 12000)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = L.pdr_run_noalloc(ctypes.byref(card), ctypes.byref(batch), ctypes.byref(B.make_outputs(o)), stream)
        assert rc == 0, L.pdr_last_error(None)
        if call == 1:  # the set-up of the first call may commit the static array; later calls take nothing
            assert torch.cuda.mem_get_info()[0] == free0, "the call took device memory"
        h = _host(o, b.n_events)
        assert np.array_equal(h["counts"], ref["counts"]), f"call {call}: counts"
        for e in range(b.n_events):
            g1 = B.event_records(h, h["counts"], b.offsets, e)
            g0 = B.event_records(ref, ref["counts"], b.offsets, e)
            assert np.array_equal(g1["tracks"]["idx"], g0["tracks"]["idx"])
            assert np.array_equal(g1["towers"]["key"], g0["towers"]["key"])
            assert np.array_equal(g1["eflow"]["key"], g0["eflow"]["key"])
            assert np.array_equal(g1["cands"]["info"], g0["cands"]["info"])
            _close(g1["tracks"]["pt"], g0["tracks"]["pt"], f"call {call} event {e} track pT")
            _close(g1["towers"]["e"], g0["towers"]["e"], f"call {call} event {e} tower E")
            _close(g1["eflow"]["e"], g0["eflow"]["e"], f"call {call} event {e} EFlow E")
            _close(g1["cands"]["pt"], g0["cands"]["pt"], f"call {call} event {e} candidate pT")
            _close(g1["cands"]["iso_sum"], g0["cands"]["iso_sum"], f"call {call} event {e} isolation")


def _lib():
    from paper_2606_26089_b300 import binding as B
    from paper_2606_26089_b300 import build
    build.build()
    L = B.lib()
    L.pdr_run_noalloc.argtypes = [ctypes.POINTER(B.pdr_card), ctypes.POINTER(B.pdr_batch),
                                  ctypes.POINTER(B.pdr_outputs), ctypes.c_void_p]
    L.pdr_run_noalloc.restype = ctypes.c_int
    L.pdr_last_error.restype = ctypes.c_char_p
    return B, L


def test_noalloc_error_returns():
    """The documented error returns, each on a batch whose every range stays
    inside the arrays the test allocated: an event above 49152 particles
    (PDR_EOVERFLOW, found before any launch), an understated max_event_size
    (the oversized event is skipped and reported: PDR_EDEVICE), and an interior
    offset past the batch's end (PDR_EDEVICE, CSR), found by the sizing pass
    when max_event_size is 0 and by the kernel otherwise."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26089_b300 import synth
    B, L = _lib()
    card = B.card_from_json("cms_like")
    stream = torch.cuda.current_stream().cuda_stream

    def run(batch_np, max_n, offsets=None, n_events=None):
        dev = B.batch_to_device(batch_np)
        if offsets is not None:
            dev["offsets"] = offsets
            dev["n_events"] = n_events
        o = B.alloc_outputs(batch_np.n_events, batch_np.n_particles)
        rc = L.pdr_run_noalloc(ctypes.byref(card), ctypes.byref(B.make_batch(dev, 0, 5, max_event_size=max_n)),
                               ctypes.byref(B.make_outputs(o)), stream)
        return rc, (L.pdr_last_error(None) or b"").decode(), o

    small = synth.make("batched", n_events=3)
    ev = small.event(0)
    row = [(float(ev["pt"][k]), float(ev["eta"][k]), float(ev["phi"][k]), float(ev["mass"][k]),
            int(ev["pdg"][k]), int(ev["charge"][k])) for k in range(len(ev["pt"]))]
    huge = synth.from_particles([(row * (49153 // len(row) + 1))[:49153]])
    rc, msg, _ = run(huge, 0)
    assert rc == -8 and "49152" in msg, (rc, msg)

    mixed = synth.from_particles([row[:50], (row * 10)[:3000], row[:50]])
    rc, msg, o = run(mixed, 100)
    assert rc == -5, (rc, msg)
    counts = o["counts"].cpu().numpy()
    assert counts[1].sum() == 0 and counts[0].sum() > 0

    five = synth.make("tiny", n_events=5)
    end4 = int(five.offsets[4])
    off = B.batch_to_device(five)["offsets"][:5].clone()
    off[1] = end4 + (five.n_particles - end4) // 2
    for max_n in (0, five.n_particles):
        rc, msg, o = run(five, max_n, offsets=off, n_events=4)
        assert rc == -5 and "CSR" in msg, (max_n, rc, msg)
    # a good call right after the failures still succeeds
    rc, msg, _ = run(small, 0)
    assert rc == 0, msg
