"""Thin ctypes binding of the CUDA library (include/pdr.h).

Argument marshalling only: every step of the detector response runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  If the
built library is missing or cannot be loaded this module raises - there is no
CPU fallback.

The functions keep the C names (``pdr_create``, ``pdr_run``, ...); ``Context``
wraps them for convenience.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PDR_LIB_VARIANT=bounds loads the bounds-checking debug build (libpdr_bounds.so)
LIB_PATH = os.path.join(HERE, "libpdr_bounds.so" if os.environ.get("PDR_LIB_VARIANT") == "bounds" else "libpdr.so")
CARD_DIR = os.path.join(HERE, "cards")

MAXSEG, MAXEDGE = 4, 8
ECAL, HCAL = 0, 1
BATCH_DEBUG = 0x1
F_REACH, F_BARREL, F_TRACKED, F_CAND, F_ECAL, F_HCAL = 0x01, 0x02, 0x04, 0x08, 0x10, 0x20
NO_KEY = 0xFFFFFFFF
STATUS = {0: "PDR_OK", -1: "PDR_EINVAL", -2: "PDR_ENOMEM", -3: "PDR_ECARD", -4: "PDR_ETIMEDOUT",
          -5: "PDR_EDEVICE", -6: "PDR_EBUSY", -7: "PDR_ENOTFOUND", -8: "PDR_EOVERFLOW"}


class PdrError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


class pdr_card(C.Structure):
    _fields_ = [
        ("B", C.c_double), ("R", C.c_double), ("L", C.c_double),
        ("nseg", C.c_int32 * 2),
        ("seg_eta_hi", (C.c_double * MAXSEG) * 2),
        ("seg_neta", (C.c_int32 * MAXSEG) * 2),
        ("seg_nphi", (C.c_int32 * MAXSEG) * 2),
        ("trk_npt", C.c_int32), ("trk_neta", C.c_int32),
        ("trk_pt_edges", C.c_double * MAXEDGE),
        ("trk_eta_edges", C.c_double * MAXEDGE),
        ("trk_eff", ((C.c_double * MAXEDGE) * MAXEDGE) * 3),
        ("res_n", C.c_int32 * 4),
        ("res_edges", (C.c_double * MAXEDGE) * 4),
        ("res_abcd", ((C.c_double * 4) * MAXEDGE) * 4),
        ("id_n", C.c_int32),
        ("id_edges", C.c_double * MAXEDGE),
        ("id_eff", (C.c_double * MAXEDGE) * 3),
        ("e_min", C.c_double * 2), ("s_min", C.c_double * 2),
        ("cand_ptmin", C.c_double),
        ("iso_dr", C.c_double), ("iso_drmin", C.c_double), ("iso_ptmin", C.c_double),
        ("iso_imax", C.c_double),
    ]


class pdr_batch(C.Structure):
    _fields_ = [
        ("n_events", C.c_uint64), ("offsets", C.c_void_p),
        ("pt", C.c_void_p), ("eta", C.c_void_p), ("phi", C.c_void_p), ("mass", C.c_void_p),
        ("pdg", C.c_void_p), ("charge", C.c_void_p), ("vz", C.c_void_p),
        ("seed", C.c_uint64), ("event_index_base", C.c_uint32), ("card_id", C.c_uint32),
        ("max_event_size", C.c_uint32), ("flags", C.c_uint32),
    ]


class pdr_outputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("tracks", "towers", "eflow", "cands", "iso", "counts", "debug")]


class pdr_launch(C.Structure):
    _fields_ = [("team", C.c_uint32), ("block", C.c_uint32), ("table_slots", C.c_uint32),
                ("grid", C.c_uint32)]

    def as_dict(self):
        return dict(team=self.team, block=self.block, table_slots=self.table_slots, grid=self.grid)


class pdr_options(C.Structure):
    _fields_ = [("pool_bytes", C.c_uint64), ("max_tickets", C.c_uint32), ("flags", C.c_uint32)]


class pdr_serve_options(C.Structure):
    _fields_ = [("max_inflight_waves", C.c_uint32), ("max_wave_requests", C.c_uint32),
                ("max_wave_particles", C.c_uint64), ("use_graphs", C.c_uint32), ("flags", C.c_uint32)]


class pdr_serve_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("requests_done", "events_done", "particles_done", "waves",
                                          "admission_waits", "graph_launches")] + [
        (n, C.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "span_s")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class pdr_pileup(C.Structure):
    _fields_ = [("n_pool", C.c_uint64)] + [(n, C.c_void_p) for n in (
        "offsets", "pt", "eta", "phi", "mass", "pdg", "charge")] + [
        ("mean", C.c_double), ("sigma_z", C.c_double), ("max_z", C.c_double),
        ("sigma_t", C.c_double), ("max_t", C.c_double),
        ("smear_hs", C.c_uint32), ("pad", C.c_uint32)]


class pdr_particles(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("pt", "eta", "phi", "mass", "vz", "vt", "pdg", "charge")]


MAX_CONDITIONS = 8
MAX_VALUES = 8
COLLECTIONS = {"pflow": 0, "track": 1, "neutral": 2, "tower": 3, "cand": 4}
FIELDS = {"pt": 0, "eta": 1, "phi": 2, "e": 3, "et": 4, "pdg": 5, "charge": 6}
OPS = {">": 0, ">=": 1, "<": 2, "<=": 3, "==": 4, "!=": 5, "in": 6, "not in": 7}


class pdr_condition(C.Structure):
    _fields_ = [("field", C.c_uint32), ("op", C.c_uint32), ("abs", C.c_uint32), ("n_values", C.c_uint32),
                ("values", C.c_double * MAX_VALUES)]


class pdr_filter(C.Structure):
    _fields_ = [("collection", C.c_uint32), ("combine", C.c_uint32), ("n_conditions", C.c_uint32),
                ("compact", C.c_uint32), ("update_features", C.c_uint32), ("pad", C.c_uint32),
                ("cond", pdr_condition * MAX_CONDITIONS)]


class pdr_ip_params(C.Structure):
    _fields_ = [("a_d0", C.c_double), ("b_d0", C.c_double), ("a_z0", C.c_double), ("b_z0", C.c_double),
                ("vx", C.c_void_p), ("vy", C.c_void_p)]


# impact-parameter resolutions sigma = sqrt(a^2 + (b / pT)^2), project-chosen
# tracker-like values (m, m GeV): d0 10 um (+) 50 um GeV / pT, z0 30 um (+) 80 um GeV / pT
IP_RESOLUTION = (10e-6, 50e-6, 30e-6, 80e-6)


def make_ip_params(resolution=IP_RESOLUTION, vx=None, vy=None) -> pdr_ip_params:
    return pdr_ip_params(*[float(x) for x in resolution], _ptr(vx), _ptr(vy))


class pdr_jet_params(C.Structure):
    _fields_ = [("collection", C.c_uint32), ("nconst_min", C.c_uint32), ("p", C.c_double), ("R", C.c_double),
                ("pt_min", C.c_double), ("ee", C.c_uint32), ("pad", C.c_uint32)]


JET_ALGORITHMS = {"antikt": -1.0, "cambridge": 0.0, "kt": 1.0}


def make_jet_params(collection: str = "pflow", algorithm: str = "antikt", R: float = 0.5, pt_min: float = 0.0,
                    nconst_min: int = 2, p: Optional[float] = None, ee: bool = False) -> pdr_jet_params:
    """Clustering pipeline parameters (collection, algorithm or exponent p, dr, pt_min, nconst_min;
    ee: the e+e- generalized kT, algorithm "ee-genkt" with p).  The defaults are the
    clustering pipeline's (App. C: pflow, antikt, dr 0.5, pt_min 0, nconst_min 2)."""
    if algorithm == "ee-genkt":
        ee = True
        algorithm = "antikt" if p is None else algorithm
    return pdr_jet_params({"pflow": 0, "truth": 1}[collection], int(nconst_min),
                          float(JET_ALGORITHMS[algorithm] if p is None else p), float(R), float(pt_min),
                          int(bool(ee)), 0)


class pdr_features(C.Structure):
    _fields_ = [("ht", C.c_float), ("met_x", C.c_float), ("met_y", C.c_float), ("met", C.c_float)]


def make_filter(spec: dict, compact: bool = True) -> pdr_filter:
    """pdr_filter from {"collection", "combine", "conditions": [{"field", "op",
    "value", "abs"}], "update_event_features"} (the filter pipeline's fields)."""
    f = pdr_filter()
    f.collection = COLLECTIONS[spec.get("collection", "pflow")]
    f.combine = {"all": 0, "any": 1}[spec.get("combine", "all")]
    conds = spec.get("conditions", [])
    if len(conds) > MAX_CONDITIONS:
        raise ValueError("at most 8 conditions")
    f.n_conditions = len(conds)
    f.compact = int(bool(compact))
    f.update_features = int(bool(spec.get("update_event_features", True)))
    for k, c in enumerate(conds):
        d = f.cond[k]
        d.field, d.op, d.abs = FIELDS[c["field"]], OPS[c["op"]], int(bool(c.get("abs", False)))
        vals = list(c["value"]) if c["op"] in ("in", "not in") else [c["value"]]
        if len(vals) > MAX_VALUES:
            raise ValueError("at most 8 values")
        d.n_values = len(vals)
        for j, v in enumerate(vals):
            d.values[j] = float(v)
    return f


class pdr_result(C.Structure):
    _fields_ = [("n_events", C.c_uint64), ("n_particles", C.c_uint64)] + [
        (n, C.c_void_p) for n in ("offsets", "counts", "tracks", "towers", "eflow", "cands", "iso", "debug")]


_lib = None


def lib():
    """Load libpdr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run python -m paper_2606_26089_b300.build)")
        L = C.CDLL(LIB_PATH)
        P, I = C.c_void_p, C.c_int
        sig = {
            "pdr_abi_version": ([], I),
            "pdr_create": ([C.POINTER(P), I, C.POINTER(pdr_options)], I),
            "pdr_destroy": ([P], I),
            "pdr_last_error": ([P], C.c_char_p),
            "pdr_card_load": ([P, C.POINTER(pdr_card), C.POINTER(C.c_uint32)], I),
            "pdr_card_unload": ([P, C.c_uint32], I),
            "pdr_card_towers": ([P, C.c_uint32, I, C.POINTER(C.c_uint32)], I),
            "pdr_run": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), C.POINTER(pdr_launch), P], I),
            "pdr_run_per_event": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), P], I),
            "pdr_run_multi": ([P, C.POINTER(pdr_batch), C.c_uint32, C.POINTER(pdr_outputs),
                               C.POINTER(pdr_launch), P], I),
            "pdr_run_host": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), C.POINTER(pdr_launch), P], I),
            "pdr_autotune": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), P, C.POINTER(pdr_launch)], I),
            "pdr_max_event_size": ([P, C.POINTER(pdr_batch), P, C.POINTER(C.c_uint32)], I),
            "pdr_check": ([P, P], I),
            "pdr_submit": ([P, C.POINTER(pdr_batch), P, C.POINTER(C.c_uint64)], I),
            "pdr_wait": ([P, C.c_uint64, I], I),
            "pdr_fetch": ([P, C.c_uint64, C.POINTER(pdr_result)], I),
            "pdr_release": ([P, C.c_uint64], I),
            "pdr_serve_start": ([P, C.POINTER(pdr_serve_options)], I),
            "pdr_serve_submit": ([P, C.POINTER(pdr_batch), C.POINTER(C.c_uint64)], I),
            "pdr_serve_stats_get": ([P, C.POINTER(pdr_serve_stats)], I),
            "pdr_serve_stop": ([P], I),
            "pdr_run_noalloc": ([C.POINTER(pdr_card), C.POINTER(pdr_batch), C.POINTER(pdr_outputs), P], I),
            "pdr_pileup_offsets": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_pileup), P, C.POINTER(C.c_uint64), P], I),
            "pdr_pileup_merge": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_pileup), P, C.POINTER(pdr_particles), P], I),
            "pdr_postprocess": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), C.POINTER(pdr_filter), P, P], I),
            "pdr_track_ip": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), C.POINTER(pdr_ip_params), P, P], I),
            "pdr_run_ip": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), C.POINTER(pdr_ip_params), P,
                            C.POINTER(pdr_launch), P], I),
            "pdr_math_eval": ([C.c_int, P, P, P, C.c_uint64, P], I),
            "pdr_cluster_jets": ([P, C.POINTER(pdr_batch), C.POINTER(pdr_outputs), C.POINTER(pdr_jet_params), P, P,
                                  P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("pdr_")]


MATH_FN = {"asin_half": 0, "sin_half_turn": 1, "ln_unit": 2, "log1p_pos": 3, "cos_two_pi": 4, "cosh": 5, "sinh": 6,
           "asinh": 7, "u01": 8, "normal": 9, "rcp": 10, "sqrt": 11, "exp_ff_hi": 12, "exp_ff_lo": 13,
           "sinh_ff_hi": 14, "sinh_ff_lo": 15}


def math_eval(name: str, x, x2=None, stream=None):
    """One of the kernels' float32 function approximations on a device float32
    tensor x (for "u01" and "normal" the tensors carry 32-bit words: x.view)."""
    torch = _torch()
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    rc = lib().pdr_math_eval(MATH_FN[name], _ptr(x), _ptr(x2), _ptr(y), int(x.numel()), s)
    if rc:
        raise PdrError(rc, "pdr_math_eval", (lib().pdr_last_error(None) or b"").decode())
    return y


def card_path(name: str) -> str:
    return name if name.endswith(".json") else os.path.join(CARD_DIR, name + ".json")


def card_from_json(name_or_dict) -> pdr_card:
    """Fill a pdr_card from the card JSON (raw detector parameters)."""
    d = name_or_dict if isinstance(name_or_dict, dict) else json.load(open(card_path(name_or_dict)))
    c = pdr_card()
    c.B, c.R, c.L = d["B"], d["R"], d["L"]
    for calo, cname in ((ECAL, "ecal"), (HCAL, "hcal")):
        segs = d[cname]["segments"]
        c.nseg[calo] = len(segs)
        for s, seg in enumerate(segs):
            c.seg_eta_hi[calo][s] = seg["eta_hi"]
            c.seg_neta[calo][s] = seg["n_eta"]
            c.seg_nphi[calo][s] = seg["n_phi"]
    te = d["track_eff"]
    c.trk_npt, c.trk_neta = len(te["pt_edges"]), len(te["abseta_edges"])
    for k, v in enumerate(te["pt_edges"]):
        c.trk_pt_edges[k] = v
    for k, v in enumerate(te["abseta_edges"]):
        c.trk_eta_edges[k] = v
    for t, name in enumerate(("hadron", "electron", "muon")):
        for i, row in enumerate(te[name]):
            for j, v in enumerate(row):
                c.trk_eff[t][i][j] = v
    for comp, name in enumerate(("track", "muon", "ecal", "hcal")):
        r = d["resolution"][name]
        c.res_n[comp] = len(r["abseta_edges"])
        for k, v in enumerate(r["abseta_edges"]):
            c.res_edges[comp][k] = v
        for k, abcd in enumerate(r["abcd"]):
            for j in range(4):
                c.res_abcd[comp][k][j] = abcd[j]
    ie = d["id_eff"]
    c.id_n = len(ie["abseta_edges"])
    for k, v in enumerate(ie["abseta_edges"]):
        c.id_edges[k] = v
    for t, name in enumerate(("electron", "muon", "photon")):
        for k, v in enumerate(ie[name]):
            c.id_eff[t][k] = v
    th = d["thresholds"]
    c.e_min[ECAL], c.s_min[ECAL] = th["ecal"]["e_min"], th["ecal"]["s_min"]
    c.e_min[HCAL], c.s_min[HCAL] = th["hcal"]["e_min"], th["hcal"]["s_min"]
    iso = d["isolation"]
    c.cand_ptmin = iso["cand_ptmin"]
    c.iso_dr, c.iso_drmin, c.iso_ptmin, c.iso_imax = iso["dr"], iso["dr_min"], iso["pt_min"], iso["i_max"]
    return c


# ---------------------------------------------------------------------------
# torch marshalling helpers
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def batch_to_device(batch, device="cuda"):
    """Copy a synth.EventBatch (numpy) to device tensors."""
    torch = _torch()
    out = {}
    for k in ("offsets", "pt", "eta", "phi", "mass", "pdg", "charge", "vz"):
        v = getattr(batch, k)
        if v is None:
            out[k] = None
            continue
        a = np.ascontiguousarray(v)
        if k == "offsets":
            a = a.astype(np.int64)
        out[k] = torch.from_numpy(a).to(device)
    out["n_events"] = batch.n_events
    out["n_particles"] = batch.n_particles
    out["max_event_size"] = int(batch.multiplicities().max()) if batch.n_events else 0
    return out


def alloc_outputs(n_events: int, n_particles: int, debug: bool = False, device="cuda"):
    """Device output buffers in the slot layout of pdr_outputs (torch tensors)."""
    torch = _torch()
    cap = max(n_particles, 1)
    f = dict(dtype=torch.float32, device=device)
    o = dict(tracks=torch.empty((cap, 4), **f), towers=torch.empty((cap, 3), **f),
             eflow=torch.empty((cap, 3), **f), cands=torch.empty((cap, 4), **f),
             iso=torch.empty((cap, 2), **f),
             counts=torch.zeros((max(n_events, 1), 4), dtype=torch.int32, device=device),
             debug=torch.empty((cap, 4), **f) if debug else None)
    return o


def make_batch(dev, card_id: int, seed: int, event_base: int = 0, debug: bool = False,
               max_event_size: Optional[int] = None) -> pdr_batch:
    b = pdr_batch()
    b.n_events = dev["n_events"]
    for k in ("offsets", "pt", "eta", "phi", "mass", "pdg", "charge", "vz"):
        setattr(b, k, _ptr(dev[k]))
    b.seed = seed & (2**64 - 1)
    b.event_index_base = event_base & 0xFFFFFFFF
    b.card_id = card_id
    b.max_event_size = dev.get("max_event_size", 0) if max_event_size is None else max_event_size
    b.flags = BATCH_DEBUG if debug else 0
    return b


def make_outputs(o) -> pdr_outputs:
    r = pdr_outputs()
    for k in ("tracks", "towers", "eflow", "cands", "iso", "counts", "debug"):
        setattr(r, k, _ptr(o.get(k)))
    return r


class Context:
    """A pdr_ctx on one CUDA device."""

    def __init__(self, device: int = 0, pool_bytes: int = 0, max_tickets: int = 0):
        self.L = lib()
        opt = pdr_options(pool_bytes, max_tickets, 0)
        h = C.c_void_p()
        self._check(self.L.pdr_create(C.byref(h), device, C.byref(opt)), "pdr_create", None)
        self.h = h
        self.device = device

    def _check(self, rc, where, h="self"):
        if rc != 0:
            handle = self.h if h == "self" else h
            msg = self.L.pdr_last_error(handle)
            raise PdrError(rc, where, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.L.pdr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        if stream is None:
            return _torch().cuda.current_stream().cuda_stream
        return stream if isinstance(stream, int) else stream.cuda_stream

    def card_load(self, card) -> int:
        c = card if isinstance(card, pdr_card) else card_from_json(card)
        cid = C.c_uint32()
        self._check(self.L.pdr_card_load(self.h, C.byref(c), C.byref(cid)), "pdr_card_load")
        return cid.value

    def card_unload(self, card_id: int):
        self._check(self.L.pdr_card_unload(self.h, card_id), "pdr_card_unload")

    def card_towers(self, card_id: int, calo: int) -> int:
        n = C.c_uint32()
        self._check(self.L.pdr_card_towers(self.h, card_id, calo, C.byref(n)), "pdr_card_towers")
        return n.value

    def run(self, batch: pdr_batch, out: pdr_outputs, launch: Optional[pdr_launch] = None, stream=None):
        self._check(self.L.pdr_run(self.h, C.byref(batch), C.byref(out),
                                   C.byref(launch) if launch is not None else None,
                                   self._stream(stream)), "pdr_run")

    def run_multi(self, batches, outs, launch: Optional[pdr_launch] = None, stream=None):
        n = len(batches)
        ba = (pdr_batch * max(n, 1))(*batches)
        oa = (pdr_outputs * max(n, 1))(*outs)
        self._check(self.L.pdr_run_multi(self.h, ba, n, oa, C.byref(launch) if launch is not None else None,
                                         self._stream(stream)), "pdr_run_multi")

    def run_per_event(self, batch: pdr_batch, out: pdr_outputs, stream=None):
        self._check(self.L.pdr_run_per_event(self.h, C.byref(batch), C.byref(out), self._stream(stream)),
                    "pdr_run_per_event")

    def run_host(self, batch: pdr_batch, out: pdr_outputs, launch: Optional[pdr_launch] = None, stream=None):
        self._check(self.L.pdr_run_host(self.h, C.byref(batch), C.byref(out),
                                        C.byref(launch) if launch is not None else None,
                                        self._stream(stream)), "pdr_run_host")

    def autotune(self, batch: pdr_batch, out: pdr_outputs, stream=None) -> pdr_launch:
        best = pdr_launch()
        self._check(self.L.pdr_autotune(self.h, C.byref(batch), C.byref(out), self._stream(stream),
                                        C.byref(best)), "pdr_autotune")
        return best

    def max_event_size(self, batch: pdr_batch, stream=None) -> int:
        n = C.c_uint32()
        self._check(self.L.pdr_max_event_size(self.h, C.byref(batch), self._stream(stream), C.byref(n)),
                    "pdr_max_event_size")
        return n.value

    def check(self, stream=None):
        self._check(self.L.pdr_check(self.h, self._stream(stream)), "pdr_check")

    def submit(self, batch: pdr_batch, stream=None) -> int:
        t = C.c_uint64()
        self._check(self.L.pdr_submit(self.h, C.byref(batch), self._stream(stream), C.byref(t)), "pdr_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        return self.L.pdr_wait(self.h, ticket, timeout_ms)

    def fetch(self, ticket: int) -> pdr_result:
        r = pdr_result()
        self._check(self.L.pdr_fetch(self.h, ticket, C.byref(r)), "pdr_fetch")
        return r

    def release(self, ticket: int):
        self._check(self.L.pdr_release(self.h, ticket), "pdr_release")

    # ---- pile-up merging
    def pileup_offsets(self, hard: pdr_batch, pu: pdr_pileup, merged_offsets, stream=None) -> int:
        """First pass: merged CSR offsets into a device tensor [n_events + 1]; returns the total."""
        tot = C.c_uint64()
        self._check(self.L.pdr_pileup_offsets(self.h, C.byref(hard), C.byref(pu), _ptr(merged_offsets),
                                              C.byref(tot), self._stream(stream)), "pdr_pileup_offsets")
        return tot.value

    def pileup_merge(self, hard: pdr_batch, pu: pdr_pileup, merged_offsets, out: dict, stream=None):
        """Second pass: fill the merged particle arrays (device tensors)."""
        o = pdr_particles(*[_ptr(out.get(k)) for k in ("pt", "eta", "phi", "mass", "vz", "vt", "pdg", "charge")])
        self._check(self.L.pdr_pileup_merge(self.h, C.byref(hard), C.byref(pu), _ptr(merged_offsets), C.byref(o),
                                            self._stream(stream)), "pdr_pileup_merge")

    # ---- filter and event features
    def postprocess(self, batch: pdr_batch, out: pdr_outputs, filt: Optional[pdr_filter] = None, features=None,
                    stream=None):
        """Filter (in place if filt.compact) and H_T / missing E_T into `features`
        (a device float32 tensor [n_events, 4]: ht, met_x, met_y, met) or None."""
        self._check(self.L.pdr_postprocess(self.h, C.byref(batch), C.byref(out),
                                           C.byref(filt) if filt is not None else None, _ptr(features),
                                           self._stream(stream)), "pdr_postprocess")

    # ---- track impact parameters
    def track_ip(self, batch: pdr_batch, out: pdr_outputs, params: pdr_ip_params, ip, stream=None):
        """d0', z0', sigma_d0, sigma_z0 of every track record into `ip` (a device
        float32 tensor [n_particles, 4], slot layout parallel to the tracks)."""
        self._check(self.L.pdr_track_ip(self.h, C.byref(batch), C.byref(out), C.byref(params), _ptr(ip),
                                        self._stream(stream)), "pdr_track_ip")

    def run_ip(self, batch: pdr_batch, out: pdr_outputs, params: pdr_ip_params, ip,
               launch: Optional[pdr_launch] = None, stream=None):
        """pdr_run with the tracks' impact parameters computed in the same
        launch, into `ip` (device float32 [n_particles, 4], parallel to the tracks)."""
        self._check(self.L.pdr_run_ip(self.h, C.byref(batch), C.byref(out), C.byref(params), _ptr(ip),
                                      C.byref(launch) if launch is not None else None, self._stream(stream)),
                    "pdr_run_ip")

    # ---- jet clustering
    def cluster_jets(self, batch: pdr_batch, out: Optional[pdr_outputs], params: pdr_jet_params, jets, jet_counts,
                     stream=None):
        """Jets into `jets` (device float32 tensor [n_particles, 8]: pt, eta, phi,
        mass, e, nconst (as uint32), C2, D2; slot layout) and `jet_counts`
        (device int32 [n_events])."""
        self._check(self.L.pdr_cluster_jets(self.h, C.byref(batch), C.byref(out) if out is not None else None,
                                            C.byref(params), _ptr(jets), _ptr(jet_counts), self._stream(stream)),
                    "pdr_cluster_jets")

    # ---- serving
    def serve_start(self, max_inflight_waves=0, max_wave_requests=0, max_wave_particles=0, use_graphs=1):
        o = pdr_serve_options(max_inflight_waves, max_wave_requests, max_wave_particles, use_graphs, 0)
        self._check(self.L.pdr_serve_start(self.h, C.byref(o)), "pdr_serve_start")

    def serve_submit(self, host_batch: pdr_batch) -> int:
        t = C.c_uint64()
        self._check(self.L.pdr_serve_submit(self.h, C.byref(host_batch), C.byref(t)), "pdr_serve_submit")
        return t.value

    def serve_stats(self) -> dict:
        st = pdr_serve_stats()
        self._check(self.L.pdr_serve_stats_get(self.h, C.byref(st)), "pdr_serve_stats_get")
        return st.as_dict()

    def serve_stop(self):
        self._check(self.L.pdr_serve_stop(self.h), "pdr_serve_stop")


def pinned_host_batch(batch, card_id: int, seed: int, event_base: int = 0):
    """A pdr_batch with HOST pointers into pinned copies of a synth.EventBatch.

    Returns (pdr_batch, keepalive) - keep the second value alive while the
    library may read the arrays."""
    import torch
    keep = {}
    b = pdr_batch()
    b.n_events = batch.n_events
    for k in ("offsets", "pt", "eta", "phi", "mass", "pdg", "charge", "vz"):
        v = getattr(batch, k)
        if v is None:
            setattr(b, k, None)
            continue
        a = np.ascontiguousarray(v)
        if k == "offsets":
            a = a.astype(np.int64)
        t = torch.from_numpy(a).pin_memory()
        keep[k] = t
        setattr(b, k, t.data_ptr())
    b.seed = seed & (2**64 - 1)
    b.event_index_base = event_base & 0xFFFFFFFF
    b.card_id = card_id
    b.max_event_size = int(batch.multiplicities().max()) if batch.n_events else 0
    b.flags = 0
    return b, keep


def result_to_host(res: pdr_result) -> dict:
    """Copy a pdr_result (device, slot layout) into host numpy arrays."""
    cudart = C.CDLL("libcudart.so.13")
    cudart.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
    n, ne = int(res.n_particles), int(res.n_events)
    cap = max(n, 1)
    out = dict(tracks=np.zeros((cap, 4), np.float32), towers=np.zeros((cap, 3), np.float32),
               eflow=np.zeros((cap, 3), np.float32), cands=np.zeros((cap, 4), np.float32),
               iso=np.zeros((cap, 2), np.float32), counts=np.zeros((max(ne, 1), 4), np.uint32),
               offsets=np.zeros(ne + 1, np.uint64))
    for k in ("tracks", "towers", "eflow", "cands", "iso", "counts", "offsets"):
        src = getattr(res, k)
        if src and out[k].nbytes:
            nb = out[k][:ne].nbytes if k == "counts" else out[k].nbytes
            assert cudart.cudaMemcpy(out[k].ctypes.data, src, nb, 2) == 0, k
    out["counts"] = out["counts"][:ne]
    return out


# ---------------------------------------------------------------------------
# views of the output records
# ---------------------------------------------------------------------------
def event_records(out_host: dict, counts: np.ndarray, offsets: np.ndarray, e: int) -> dict:
    """Slot-layout host copies -> the records of event e (numpy, typed)."""
    a = int(offsets[e])
    nt, nw, nf, nc = (int(x) for x in counts[e])
    tr = out_host["tracks"][a:a + nt]
    tw = out_host["towers"][a:a + nw]
    ef = out_host["eflow"][a:a + nf]
    cd = out_host["cands"][a:a + nc]
    iso = out_host["iso"][a:a + nc]
    r = dict(
        tracks=dict(pt=tr[:, 0], eta=tr[:, 1], phi=tr[:, 2], idx=tr[:, 3].view(np.uint32)),
        towers=dict(key=tw[:, 0].view(np.uint32), e=tw[:, 1], et=tw[:, 2]),
        eflow=dict(key=ef[:, 0].view(np.uint32), e=ef[:, 1], et=ef[:, 2]),
        cands=dict(pt=cd[:, 0], eta=cd[:, 1], phi=cd[:, 2], info=cd[:, 3].view(np.uint32),
                   iso_sum=iso[:, 0], iso_rel=iso[:, 1]),
    )
    if out_host.get("debug") is not None:
        d = out_host["debug"][a:int(offsets[e + 1])]
        r["debug"] = dict(key=d[:, 0].view(np.uint32), eta_pos=d[:, 1], phi_pos=d[:, 2],
                          flags=d[:, 3].view(np.uint32))
    return r


# ---------------------------------------------------------------------------
# pile-up merging helpers
# ---------------------------------------------------------------------------
# defaults of the pile-up block (Sec. 2.2; App. C, parametric pile-up fields)
SIGMA_Z = 0.053
MAX_Z = 0.25
SIGMA_T = 160e-12
MAX_T = 800e-12


def make_pileup(pool_dev: dict, mean: float, sigma_z: float = SIGMA_Z, max_z: float = MAX_Z, smear_hs: bool = True,
                sigma_t: float = SIGMA_T, max_t: float = MAX_T) -> pdr_pileup:
    """pdr_pileup over a device pool (batch_to_device of the minimum-bias batch)."""
    p = pdr_pileup()
    p.n_pool = pool_dev["n_events"]
    for k in ("offsets", "pt", "eta", "phi", "mass", "pdg", "charge"):
        setattr(p, k, _ptr(pool_dev[k]))
    p.mean, p.sigma_z, p.max_z, p.smear_hs = float(mean), float(sigma_z), float(max_z), int(bool(smear_hs))
    p.sigma_t, p.max_t = float(sigma_t), float(max_t)
    return p


def merge_pileup(ctx: "Context", hard_dev: dict, pool_dev: dict, mean: float, sigma_z: float, max_z: float,
                 smear_hs: bool, seed: int, event_base: int = 0, stream=None, sigma_t: float = SIGMA_T,
                 max_t: float = MAX_T, with_time: bool = True) -> dict:
    """Both passes; returns the merged batch as device tensors (batch_to_device
    layout, plus the vertex times "vt" unless with_time is false)."""
    torch = _torch()
    hb = make_batch(hard_dev, 0, seed, event_base=event_base)
    pu = make_pileup(pool_dev, mean, sigma_z, max_z, smear_hs, sigma_t, max_t)
    n = hard_dev["n_events"]
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    total = ctx.pileup_offsets(hb, pu, off, stream)
    cap = max(total, 1)
    f = dict(dtype=torch.float32, device="cuda")
    out = dict(pt=torch.empty(cap, **f), eta=torch.empty(cap, **f), phi=torch.empty(cap, **f),
               mass=torch.empty(cap, **f), vz=torch.empty(cap, **f),
               vt=torch.empty(cap, **f) if with_time else None,
               pdg=torch.empty(cap, dtype=torch.int32, device="cuda"),
               charge=torch.empty(cap, dtype=torch.int8, device="cuda"))
    ctx.pileup_merge(hb, pu, off, out, stream)
    out["offsets"] = off
    out["n_events"] = n
    out["n_particles"] = total
    return out
