"""FP64 CPU oracle (TEST INFRASTRUCTURE): ctypes wrapper around ``oracle.c``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does, and this package imports nothing from the product: it
parses the detector card JSON itself and has its own C implementation of every
step of the method.

The C oracle follows the paper's TorchDelphes module chain (Sec. 2.2, App. D)
and the isolation definition of Sec. 2.4 (Eq. 1); see ``oracle.h``.
"""

from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

MAXSEG, MAXEDGE = 4, 8
ECAL, HCAL = 0, 1
CLS_E, CLS_MU, CLS_GAMMA, CLS_CHAD, CLS_NHAD, CLS_INVIS = range(6)
RES_TRACK, RES_MUON, RES_ECAL, RES_HCAL = range(4)
PURPOSE_TRACK, PURPOSE_ID, PURPOSE_TOWER_ECAL, PURPOSE_TOWER_HCAL = 1, 2, 3, 4
(K_BARREL, K_LOOP, K_ETA, K_PHI, K_TWR_E, K_TWR_S, K_EF_E, K_EF_S, K_ISO_PT, K_ISO_DR,
 K_ISO_DRMIN, K_ISOLATED) = range(1, 13)
F_REACH, F_BARREL, F_TRACKED, F_CAND, F_ECAL, F_HCAL = 0x01, 0x02, 0x04, 0x08, 0x10, 0x20
NO_KEY = 0xFFFFFFFF
DEFAULT_G = 1e-5


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (plain C, -O2, no fast-math)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra", "-Wno-unused-parameter",
               "-o", _LIB + ".tmp", _SRC, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Card(C.Structure):
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
        ("cand_ptmin", C.c_double), ("iso_dr", C.c_double), ("iso_drmin", C.c_double),
        ("iso_ptmin", C.c_double), ("iso_imax", C.c_double),
    ]


PARTICLE = np.dtype([("eta_pos", "f8"), ("phi_pos", "f8"), ("e", "f8"), ("cond", "f8"), ("key", "u4"),
                     ("flags", "u4"), ("cls", "u4"), ("pad", "u4")])
TRACK = np.dtype([("pt", "f8"), ("eta", "f8"), ("phi", "f8"), ("e", "f8"), ("idx", "u4"),
                  ("pad", "u4")])
TOWER = np.dtype([("esum", "f8"), ("etrk", "f8"), ("e", "f8"), ("et", "f8"), ("sigma", "f8"),
                  ("eflow_e", "f8"), ("eflow_et", "f8"), ("eta_c", "f8"), ("phi_c", "f8"),
                  ("key", "u4"), ("owner", "u4"), ("kept", "u4"), ("eflow_kept", "u4")])
CAND = np.dtype([("pt", "f8"), ("eta", "f8"), ("phi", "f8"), ("iso_sum", "f8"),
                 ("iso_rel", "f8"), ("idx", "u4"), ("cls", "u4"), ("isolated", "u4"),
                 ("pad", "u4")])
MARGINAL = np.dtype([("kind", "u4"), ("id", "u4"), ("aux", "u4"), ("aux2", "u4"), ("v", "f8"),
                     ("t", "f8"), ("w", "f8"), ("taken", "i4"), ("alt", "i4")])
FLIP = np.dtype([("kind", "u4"), ("id", "u4"), ("aux", "u4"), ("aux2", "u4")])


class Counts(C.Structure):
    _fields_ = [(n, C.c_int32) for n in
                ("n_trk", "n_twr", "n_twr_kept", "n_eflow", "n_cand", "n_marg", "err", "pad")]


class PileUp(C.Structure):
    _fields_ = [("mean", C.c_double), ("sigma_z", C.c_double), ("max_z", C.c_double),
                ("sigma_t", C.c_double), ("max_t", C.c_double),
                ("smear_hs", C.c_int32), ("pad", C.c_int32)]


class IPParams(C.Structure):
    """Impact-parameter resolutions: sigma = sqrt(a^2 + (b / pT)^2) (m, m GeV)."""
    _fields_ = [("a_d0", C.c_double), ("b_d0", C.c_double), ("a_z0", C.c_double), ("b_z0", C.c_double)]


# vertex-time width and truncation of the pile-up block's defaults (Sec. 2.2,
# parametric pile-up fields): 160 ps and 800 ps
SIGMA_T = 160e-12
MAX_T = 800e-12


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.oracle_philox4x32_10.argtypes = [P, P, P]
        _lib.oracle_u01.argtypes = [C.c_uint32]
        _lib.oracle_u01.restype = C.c_double
        _lib.oracle_normal.argtypes = [C.c_uint32, C.c_uint32]
        _lib.oracle_normal.restype = C.c_double
        _lib.oracle_lognormal.argtypes = [C.c_double, C.c_double, C.c_double]
        _lib.oracle_lognormal.restype = C.c_double
        _lib.oracle_rel_resolution.argtypes = [C.POINTER(Card), C.c_int, C.c_double, C.c_double]
        _lib.oracle_rel_resolution.restype = C.c_double
        _lib.oracle_eff_threshold.argtypes = [C.c_double]
        _lib.oracle_eff_threshold.restype = C.c_uint64
        _lib.oracle_classify.argtypes = [C.c_int32, C.c_int32]
        _lib.oracle_propagate.argtypes = [C.POINTER(Card), C.c_double, C.c_double, C.c_double,
                                          C.c_int32, C.c_double, P, P, P]
        _lib.oracle_tower_key.argtypes = [C.POINTER(Card), C.c_int, C.c_double, C.c_double]
        _lib.oracle_tower_key.restype = C.c_uint32
        _lib.oracle_tower_centre.argtypes = [C.POINTER(Card), C.c_uint32, P, P, P, P]
        _lib.oracle_n_towers.argtypes = [C.POINTER(Card), C.c_int]
        _lib.oracle_philox_n.argtypes = [C.c_int64, P, P, P]
        _lib.oracle_normal_n.argtypes = [C.c_int64, P, P, P]
        _lib.oracle_lognormal_n.argtypes = [C.c_int64, C.c_double, C.c_double, P, P]
        _lib.oracle_run_event.argtypes = [C.POINTER(Card), C.c_int64, P, P, P, P, P, P, P,
                                          C.c_uint64, C.c_uint32, C.c_double, P, C.c_int32,
                                          P, P, P, P, P, C.c_int32, C.POINTER(Counts)]
        _lib.oracle_run_batch.argtypes = [C.POINTER(Card), C.c_int64, P, P, P, P, P, P, P, P,
                                          C.c_uint64, C.c_uint32, C.c_int32, P]
        _lib.oracle_poisson_thresholds.argtypes = [C.c_double, P, C.c_int32]
        _lib.oracle_poisson_thresholds.restype = C.c_int32
        _lib.oracle_pileup_draws.argtypes = [C.POINTER(PileUp), P, C.c_int32, C.c_uint64, C.c_uint64,
                                             C.c_uint32, C.c_double, P, P, P, P, C.c_int32, P, P]
        _lib.oracle_pileup_draws.restype = C.c_int32
        _lib.oracle_pileup_draws_forced.argtypes = [C.POINTER(PileUp), P, C.c_int32, C.c_uint64, C.c_uint64,
                                                    C.c_uint32, C.c_double, P, P, P, P, C.c_int32, P, P,
                                                    P, C.c_int32, P, C.c_int32]
        _lib.oracle_pileup_draws_forced.restype = C.c_int32
        D = C.c_double
        _lib.oracle_track_ip.argtypes = [C.POINTER(Card), D, D, D, C.c_int32, D, D, D, P, P, P]
        _lib.oracle_track_ip.restype = None
        _lib.oracle_track_ip_smeared.argtypes = [C.POINTER(Card), C.POINTER(IPParams), D, D, D, C.c_int32, D, D, D,
                                                 C.c_uint64, C.c_uint32, C.c_uint32, P]
        _lib.oracle_track_ip_smeared.restype = None
        _lib.oracle_cluster.argtypes = [C.c_int64, P, P, P, P, D, D, D, C.c_int32, C.c_int32, P, P]
        _lib.oracle_cluster.restype = C.c_int32
        _lib.oracle_cluster_forced.argtypes = [C.c_int64, P, P, P, P, D, D, D, C.c_int32, C.c_int32, P, P,
                                               P, C.c_int32, P, C.c_int32]
        _lib.oracle_cluster_forced.restype = C.c_int32
    return _lib


# ----------------------------------------------------------------------------
# card parsing (the oracle's own; the CUDA binding has a separate one)
# ----------------------------------------------------------------------------
CARD_DIR = os.path.join(os.path.dirname(_HERE), "paper_2606_26089_b300", "cards")


def card_path(name: str) -> str:
    return name if name.endswith(".json") else os.path.join(CARD_DIR, name + ".json")


def load_card(name_or_dict) -> Card:
    d = name_or_dict if isinstance(name_or_dict, dict) else json.load(open(card_path(name_or_dict)))
    c = Card()
    c.B, c.R, c.L = d["B"], d["R"], d["L"]
    for calo, cname in ((ECAL, "ecal"), (HCAL, "hcal")):
        segs = d[cname]["segments"]
        assert 1 <= len(segs) <= MAXSEG
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
    c.cand_ptmin, c.iso_dr, c.iso_drmin = iso["cand_ptmin"], iso["dr"], iso["dr_min"]
    c.iso_ptmin, c.iso_imax = iso["pt_min"], iso["i_max"]
    return c


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------
def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_n(ctr: np.ndarray, key: Sequence[int]) -> np.ndarray:
    """Philox4x32-10 of each row of ctr [n, 4] under one key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().oracle_philox_n(c.shape[0], _ptr(c), _ptr(k), _ptr(out))
    return out


def normal_n(wa: np.ndarray, wb: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(wa, np.uint32)
    b = np.ascontiguousarray(wb, np.uint32)
    out = np.zeros(a.shape[0], np.float64)
    lib().oracle_normal_n(a.shape[0], _ptr(a), _ptr(b), _ptr(out))
    return out


def lognormal_n(x: float, rel: float, z: np.ndarray) -> np.ndarray:
    zz = np.ascontiguousarray(z, np.float64)
    out = np.zeros(zz.shape[0], np.float64)
    lib().oracle_lognormal_n(zz.shape[0], x, rel, _ptr(zz), _ptr(out))
    return out


def u01(w: int) -> float:
    return lib().oracle_u01(int(w))


def normal(wa: int, wb: int) -> float:
    return lib().oracle_normal(int(wa), int(wb))


def lognormal(x: float, rel: float, z: float) -> float:
    return lib().oracle_lognormal(x, rel, z)


def rel_resolution(card: Card, comp: int, abseta: float, x: float) -> float:
    return lib().oracle_rel_resolution(C.byref(card), comp, abseta, x)


def eff_threshold(eff: float) -> int:
    return int(lib().oracle_eff_threshold(eff))


def classify(pdg: int, charge: int) -> int:
    return lib().oracle_classify(int(pdg), int(charge))


def propagate(card: Card, pt, eta, phi, q, vz=0.0):
    """(reach, barrel, eta_pos, phi_pos) of one particle."""
    b = C.c_int32()
    ep, pp = C.c_double(), C.c_double()
    reach = lib().oracle_propagate(C.byref(card), pt, eta, phi, int(q), vz, C.byref(b),
                                   C.byref(ep), C.byref(pp))
    return reach, b.value, ep.value, pp.value


def tower_key(card: Card, calo: int, eta_pos: float, phi_pos: float) -> int:
    return int(lib().oracle_tower_key(C.byref(card), calo, eta_pos, phi_pos))


def tower_centre(card: Card, key: int):
    ec, pc = C.c_double(), C.c_double()
    r, k = C.c_int32(), C.c_int32()
    rc = lib().oracle_tower_centre(C.byref(card), key, C.byref(ec), C.byref(pc), C.byref(r),
                                   C.byref(k))
    if rc:
        raise ValueError(f"bad tower key {key:#x}")
    return ec.value, pc.value, r.value, k.value


def n_towers(card: Card, calo: int) -> int:
    return lib().oracle_n_towers(C.byref(card), calo)


# ----------------------------------------------------------------------------
# events
# ----------------------------------------------------------------------------
class EventResult:
    """Oracle output for one event (numpy structured arrays)."""

    def __init__(self, particles, tracks, towers, cands, marginal, counts):
        self.particles = particles
        self.tracks = tracks
        self.towers = towers
        self.cands = cands
        self.marginal = marginal
        self.counts = counts

    @property
    def kept_towers(self):
        return self.towers[self.towers["kept"] != 0]

    @property
    def eflow(self):
        return self.towers[self.towers["eflow_kept"] != 0]


def run_event(card: Card, ev: dict, seed: int, event: int, g: float = DEFAULT_G,
              flips: Optional[Sequence[tuple]] = None, marg_cap: Optional[int] = None) -> EventResult:
    """Run one event.  ``ev`` holds float32/int arrays pt, eta, phi, mass, pdg, charge[, vz]."""
    pt = np.ascontiguousarray(ev["pt"], np.float32)
    n = pt.shape[0]
    eta = np.ascontiguousarray(ev["eta"], np.float32)
    phi = np.ascontiguousarray(ev["phi"], np.float32)
    mass = np.ascontiguousarray(ev["mass"], np.float32)
    pdg = np.ascontiguousarray(ev["pdg"], np.int32)
    charge = np.ascontiguousarray(ev["charge"], np.int8)
    vz = ev.get("vz")
    vz = None if vz is None else np.ascontiguousarray(vz, np.float32)
    cap = max(n, 1)
    part = np.zeros(cap, PARTICLE)
    trk = np.zeros(cap, TRACK)
    twr = np.zeros(cap, TOWER)
    cand = np.zeros(cap, CAND)
    mcap = marg_cap if marg_cap is not None else 64 + 16 * n
    marg = np.zeros(max(mcap, 1), MARGINAL)
    fl = np.zeros(max(len(flips or ()), 1), FLIP)
    for i, f in enumerate(flips or ()):
        fl[i] = tuple(f) + (0,) * (4 - len(f))
    cnt = Counts()
    rc = lib().oracle_run_event(C.byref(card), n, _ptr(pt), _ptr(eta), _ptr(phi), _ptr(mass),
                                _ptr(pdg), _ptr(charge), _ptr(vz), int(seed) & (2**64 - 1),
                                int(event) & 0xFFFFFFFF, g, _ptr(fl), len(flips or ()),
                                _ptr(part), _ptr(trk), _ptr(twr), _ptr(cand), _ptr(marg), mcap,
                                C.byref(cnt))
    if rc:
        raise RuntimeError(f"oracle_run_event failed: {rc} (-2: flip of a non-marginal decision)")
    return EventResult(part[:n], trk[:cnt.n_trk], twr[:cnt.n_twr], cand[:cnt.n_cand],
                       marg[:cnt.n_marg], cnt)


def run_batch(card: Card, batch, seed: int, event_base: int = 0, nthreads: Optional[int] = None):
    """Counts [n_events, 4] (tracks, kept towers, EFlow neutrals, candidates) for a CSR batch."""
    nthreads = nthreads or os.cpu_count() or 1
    ne = batch.n_events
    counts = np.zeros((max(ne, 1), 4), np.uint32)
    off = np.ascontiguousarray(batch.offsets, np.uint64)
    arr = [np.ascontiguousarray(getattr(batch, k)) for k in ("pt", "eta", "phi", "mass", "pdg", "charge")]
    vz = None if batch.vz is None else np.ascontiguousarray(batch.vz, np.float32)
    rc = lib().oracle_run_batch(C.byref(card), ne, _ptr(off), *[_ptr(a) for a in arr], _ptr(vz),
                                int(seed) & (2**64 - 1), int(event_base) & 0xFFFFFFFF, int(nthreads),
                                _ptr(counts))
    if rc:
        raise RuntimeError(f"oracle_run_batch failed: {rc}")
    return counts[:ne]


# ----------------------------------------------------------------------------
# pile-up merging (Sec. 2.2; readings in oracle.h)
# ----------------------------------------------------------------------------
def poisson_thresholds(mean: float, kmax: int = 8192) -> np.ndarray:
    """Integer thresholds T[k] = floor(P(N <= k) 2^32) of the Poisson(mean) CDF (last entry 2^32)."""
    T = np.zeros(kmax, np.uint64)
    K = lib().oracle_poisson_thresholds(float(mean), _ptr(T), int(kmax))
    if K < 0:
        raise ValueError("Poisson table does not end within kmax entries")
    return T[:K]


def pileup_draws(pu: PileUp, T: np.ndarray, n_pool: int, seed: int, event: int, g: float = DEFAULT_G,
                 cap: int = 65536, flips: Sequence[tuple] = (), marginal_out: Optional[list] = None):
    """(n, pool indices, vertex z [m], vertex t [s], hard vertex shift z_hs [m],
    hard vertex time t_hs [s], marginal count) of one hard event.  flips lists
    truncation decisions (purpose, slot, attempt) to take the other way (each
    must be marginal: else ValueError); marginal_out, if given, receives the
    (purpose, slot, attempt) triples of the run's marginal decisions."""
    n = C.c_int32()
    zhs, ths = C.c_double(), C.c_double()
    idx = np.zeros(cap, np.uint32)
    z = np.zeros(cap, np.float64)
    t = np.zeros(cap, np.float64)
    T = np.ascontiguousarray(T, np.uint64)
    fl = np.ascontiguousarray(np.asarray(list(flips) or [(0, 0, 0)], np.uint32).reshape(-1, 3))
    mcap = 4096
    mo = np.zeros((mcap, 3), np.uint32)
    m = lib().oracle_pileup_draws_forced(C.byref(pu), _ptr(T), int(T.shape[0]), int(n_pool), int(seed) & (2**64 - 1),
                                         int(event) & 0xFFFFFFFF, float(g), C.byref(n), _ptr(idx), _ptr(z), _ptr(t),
                                         int(cap), C.byref(zhs), C.byref(ths), _ptr(fl), len(flips), _ptr(mo), mcap)
    if m == -2:
        raise ValueError("a forced truncation decision is not marginal or does not occur")
    if m < 0:
        raise ValueError("more interactions than cap")
    if marginal_out is not None:
        marginal_out.extend(tuple(int(x) for x in r) for r in mo[:min(m, mcap)])
    k = n.value
    return k, idx[:k].copy(), z[:k].copy(), t[:k].copy(), zhs.value, ths.value, m


def pileup_merge(hard, pool, mean: float, sigma_z: float, max_z: float, smear_hs: bool, seed: int,
                 event_base: int = 0, g: float = DEFAULT_G, sigma_t: float = SIGMA_T, max_t: float = MAX_T,
                 flips: Optional[dict] = None) -> dict:
    """The merged batch: per hard event its own particles (vertex z plus the hard
    shift), then the pool events of its interactions in draw order, each at its
    interaction's vertex z and time (the hard particles at time t_hs).  Returns
    the merged CSR arrays (vz and vt in float64), the
    draws, the number of marginal truncation decisions, the events holding
    them and, per such event, its marginal decisions.  flips maps an event
    to the truncation decisions to force the other way (see pileup_draws)."""
    pu = PileUp(float(mean), float(sigma_z), float(max_z), float(sigma_t), float(max_t), int(bool(smear_hs)), 0)
    T = poisson_thresholds(mean)
    po = np.asarray(pool.offsets, np.int64)
    psz = np.diff(po)
    ho = np.asarray(hard.offsets, np.int64)
    starts, lens, zs, ts, srcs = [], [], [], [], []
    draws = []
    n_marg = 0
    marg_events = []
    marg_decisions = {}
    for e in range(hard.n_events):
        mlist = []
        k, idx, z, t, zhs, ths, m = pileup_draws(pu, T, pool.n_events, seed, event_base + e, g,
                                                 flips=(flips or {}).get(e, ()), marginal_out=mlist)
        n_marg += m
        if m:
            marg_events.append(e)
            marg_decisions[e] = mlist
        draws.append((k, idx, z, t, zhs, ths))
        starts.append(ho[e]); lens.append(ho[e + 1] - ho[e]); zs.append(zhs); ts.append(ths); srcs.append(0)
        for j in range(k):
            starts.append(po[idx[j]]); lens.append(psz[idx[j]]); zs.append(z[j]); ts.append(t[j]); srcs.append(1)
    starts = np.asarray(starts, np.int64); lens = np.asarray(lens, np.int64)
    zs = np.asarray(zs, np.float64); ts = np.asarray(ts, np.float64); srcs = np.asarray(srcs, np.int8)
    seg = np.repeat(np.arange(lens.shape[0]), lens)
    pos = np.arange(int(lens.sum()), dtype=np.int64) - np.repeat(np.cumsum(lens) - lens, lens)
    src_index = starts[seg] + pos
    from_pool = srcs[seg] == 1
    out = {}
    for key in ("pt", "eta", "phi", "mass", "pdg", "charge"):
        h, pl = np.asarray(getattr(hard, key)), np.asarray(getattr(pool, key))
        v = np.empty(src_index.shape[0], h.dtype)
        v[~from_pool] = h[src_index[~from_pool]]
        v[from_pool] = pl[src_index[from_pool]]
        out[key] = v
    hvz = np.zeros(ho[-1] if ho.shape[0] else 0, np.float64) if hard.vz is None else np.asarray(hard.vz, np.float64)
    vz = zs[seg].copy()
    vz[~from_pool] += hvz[src_index[~from_pool]]
    out["vz"] = vz
    out["vt"] = ts[seg].copy()
    per_event = np.asarray([ho[e + 1] - ho[e] + sum(int(psz[i]) for i in d[1]) for e, d in enumerate(draws)],
                           np.int64)
    off = np.zeros(hard.n_events + 1, np.uint64)
    np.cumsum(per_event, out=off[1:])
    out["offsets"] = off
    out["draws"] = draws
    out["marginal"] = n_marg
    out["marginal_events"] = marg_events
    out["marginal_decisions"] = marg_decisions
    return out


# ----------------------------------------------------------------------------
# track impact parameters
# ----------------------------------------------------------------------------
def track_ip(card: Card, pt: float, eta: float, phi: float, q: int, x0: float, y0: float, z0: float):
    """(d0, z0, s) of one particle's helix (see oracle.h)."""
    d0, zz, s = C.c_double(), C.c_double(), C.c_double()
    lib().oracle_track_ip(C.byref(card), float(pt), float(eta), float(phi), int(q), float(x0), float(y0),
                          float(z0), C.byref(d0), C.byref(zz), C.byref(s))
    return d0.value, zz.value, s.value


def track_ip_smeared(card: Card, ip: IPParams, pt, eta, phi, q, x0, y0, z0, seed: int, event: int, idx: int):
    """(d0', z0', sigma_d0, sigma_z0) of one particle."""
    out = np.zeros(4, np.float64)
    lib().oracle_track_ip_smeared(C.byref(card), C.byref(ip), float(pt), float(eta), float(phi), int(q),
                                  float(x0), float(y0), float(z0), int(seed) & (2**64 - 1),
                                  int(event) & 0xFFFFFFFF, int(idx) & 0xFFFFFFFF, _ptr(out))
    return tuple(out)


def event_track_ip(card: Card, ip: IPParams, ev: dict, ref: "EventResult", seed: int, event: int) -> np.ndarray:
    """[n_tracks, 4] (d0', z0', sigma_d0, sigma_z0) of an event's tracks, in the
    order of ref.tracks; ev may hold vx, vy, vz (absent: 0)."""
    n = len(ev["pt"])
    vx = np.zeros(n) if ev.get("vx") is None else np.asarray(ev["vx"], np.float64)
    vy = np.zeros(n) if ev.get("vy") is None else np.asarray(ev["vy"], np.float64)
    vz = np.zeros(n) if ev.get("vz") is None else np.asarray(ev["vz"], np.float64)
    out = np.zeros((len(ref.tracks), 4), np.float64)
    for k, i in enumerate(ref.tracks["idx"].astype(np.int64)):
        out[k] = track_ip_smeared(card, ip, ev["pt"][i], ev["eta"][i], ev["phi"][i], ev["charge"][i], vx[i], vy[i],
                                  vz[i], seed, event, int(i))
    return out


# ----------------------------------------------------------------------------
# jet clustering
# ----------------------------------------------------------------------------
JET = np.dtype([("px", "f8"), ("py", "f8"), ("pz", "f8"), ("e", "f8"), ("pt", "f8"), ("eta", "f8"),
                ("phi", "f8"), ("mass", "f8"), ("e2", "f8"), ("e3", "f8"), ("c2", "f8"), ("d2", "f8"),
                ("nconst", "i4"), ("pad", "i4")])
ALGORITHM_P = {"antikt": -1.0, "cambridge": 0.0, "kt": 1.0}


def cluster(px, py, pz, e, p: float = -1.0, R: float = 0.5, pt_min: float = 0.0, nconst_min: int = 1,
            ee: bool = False):
    """(jets structured array, marginal steps) of one event's objects (see oracle.h);
    ee: the e+e- generalized kT (energies and angles)."""
    arr = [np.ascontiguousarray(x, np.float64) for x in (px, py, pz, e)]
    n = arr[0].shape[0]
    jets = np.zeros(max(n, 1), JET)
    m = C.c_int32()
    k = lib().oracle_cluster(n, *[_ptr(a) for a in arr], float(p), float(R), float(pt_min), int(nconst_min),
                             int(bool(ee)), _ptr(jets), C.byref(m))
    if k < 0:
        raise ValueError("bad clustering arguments")
    return jets[:k].copy(), m.value


def cluster_forced(px, py, pz, e, p: float = -1.0, R: float = 0.5, pt_min: float = 0.0, nconst_min: int = 1,
                   ee: bool = False, flips: Sequence[int] = ()):
    """(jets, indices of the marginal steps) of one event, taking the runner-up
    decision at each listed step (steps counted from 0 in recombination order);
    raises ValueError if a listed step is not marginal."""
    arr = [np.ascontiguousarray(x, np.float64) for x in (px, py, pz, e)]
    n = arr[0].shape[0]
    jets = np.zeros(max(n, 1), JET)
    m = C.c_int32()
    fl = np.ascontiguousarray(list(flips) or [0], np.int32)
    cap = max(n, 1)
    steps = np.zeros(cap, np.int32)
    k = lib().oracle_cluster_forced(n, *[_ptr(a) for a in arr], float(p), float(R), float(pt_min), int(nconst_min),
                                    int(bool(ee)), _ptr(jets), C.byref(m), _ptr(fl), len(flips), _ptr(steps), cap)
    if k == -2:
        raise ValueError("a forced step is not marginal")
    if k < 0:
        raise ValueError("bad clustering arguments")
    return jets[:k].copy(), steps[:min(m.value, cap)].tolist()


def four_momenta(pt, eta, phi, e):
    """(px, py, pz, E) of objects given pT, eta, phi and energy."""
    pt, eta, phi, e = (np.asarray(x, np.float64) for x in (pt, eta, phi, e))
    return pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta), e
