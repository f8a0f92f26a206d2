"""Seeded synthetic truth events shaped like the paper's workloads.

The paper's samples (Pythia8 H->ZZ->4l, ttW and ee->ZZ->qq HepMC files, and the
MinBias pile-up file; Sec. 3 performance table and App. D validation) are not
available, so these generators stand in for them.  They only draw truth-level
particles; nothing here computes any part of the detector response, so both the
CUDA path and the CPU oracle can take their inputs from this module.

Every workload is a ragged CSR batch in SoA layout:

* ``offsets``  uint64 [n_events + 1]   particle range of event e is offsets[e]:offsets[e+1]
* ``pt``       float32 [N]  transverse momentum (GeV)
* ``eta``      float32 [N]  pseudorapidity of the momentum
* ``phi``      float32 [N]  azimuth of the momentum, in [-pi, pi)
* ``mass``     float32 [N]  (GeV)
* ``pdg``      int32   [N]  PDG id
* ``charge``   int8    [N]  electric charge in units of e
* ``vz``       float32 [N] or None   production vertex z (m); None means all at z = 0

Workloads (sizes as the benchmark configurations name them):

* ``tiny``     100 events, Poisson(50)                                   seed 0
* ``batched``  100k events, Poisson(400) + 4 hard objects                seed 1
* ``ee``       1M events, Poisson(35), isotropic, sum E = 91.2 GeV       seed 2
* ``pileup``   10k events, Poisson(400) + 170 vertices x Poisson(30)     seed 3

For pile-up merging on the device: a minimum-bias pool (``make_minbias_pool``,
Poisson(30) particles an interaction, seed 5) and hard-scatter events
(``make_hard``, Poisson(400), seed 6).

All use numpy's PCG64 ``default_rng(seed)``, so a workload is a pure function of
(seed, n_events).
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# Species of the soft-particle mix: (|pdg|, charged?, mass GeV, fraction).
# Masses are the PDG values.  pi+- 55%, gamma 25%, K+- 8%, K_L 3%, n 3%,
# p 4%, e+- 1%, mu+- 1%.
_SPECIES = (
    (211, True, 0.13957039, 0.55),
    (22, False, 0.0, 0.25),
    (321, True, 0.493677, 0.08),
    (130, False, 0.497611, 0.03),
    (2112, False, 0.93956542, 0.03),
    (2212, True, 0.93827209, 0.04),
    (11, True, 0.00051099895, 0.01),
    (13, True, 0.1056583755, 0.01),
)
_ABS_PDG = np.array([s[0] for s in _SPECIES], dtype=np.int32)
_CHARGED = np.array([s[1] for s in _SPECIES], dtype=bool)
_MASS = np.array([s[2] for s in _SPECIES], dtype=np.float64)
_FRAC = np.array([s[3] for s in _SPECIES], dtype=np.float64)
_FRAC = _FRAC / _FRAC.sum()

ETA_MAX = 4.9
PT_CAP = 500.0


@dataclasses.dataclass
class EventBatch:
    offsets: np.ndarray
    pt: np.ndarray
    eta: np.ndarray
    phi: np.ndarray
    mass: np.ndarray
    pdg: np.ndarray
    charge: np.ndarray
    vz: Optional[np.ndarray] = None
    name: str = ""

    @property
    def n_events(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_particles(self) -> int:
        return int(self.offsets[-1])

    def multiplicities(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def slice_events(self, e0: int, e1: int) -> "EventBatch":
        """Events [e0, e1) as a batch of their own (offsets rebased to 0)."""
        a, b = int(self.offsets[e0]), int(self.offsets[e1])
        return EventBatch(
            offsets=(self.offsets[e0:e1 + 1] - self.offsets[e0]).astype(np.uint64),
            pt=self.pt[a:b], eta=self.eta[a:b], phi=self.phi[a:b],
            mass=self.mass[a:b], pdg=self.pdg[a:b], charge=self.charge[a:b],
            vz=None if self.vz is None else self.vz[a:b],
            name=f"{self.name}[{e0}:{e1}]")

    def event(self, e: int) -> dict:
        a, b = int(self.offsets[e]), int(self.offsets[e + 1])
        return dict(pt=self.pt[a:b], eta=self.eta[a:b], phi=self.phi[a:b],
                    mass=self.mass[a:b], pdg=self.pdg[a:b], charge=self.charge[a:b],
                    vz=None if self.vz is None else self.vz[a:b])

    def nbytes_input(self) -> int:
        n = self.pt.nbytes + self.eta.nbytes + self.phi.nbytes + self.mass.nbytes
        n += self.pdg.nbytes + self.charge.nbytes + self.offsets.nbytes
        if self.vz is not None:
            n += self.vz.nbytes
        return int(n)


def _offsets(counts: np.ndarray) -> np.ndarray:
    off = np.zeros(counts.shape[0] + 1, dtype=np.uint64)
    np.cumsum(counts, out=off[1:])
    return off


def _phi32(rng, n):
    phi = rng.uniform(-np.pi, np.pi, n).astype(np.float32)
    # float32 rounding can land exactly on +pi; keep the documented [-pi, pi).
    phi[phi >= np.float32(np.pi)] = np.float32(-np.pi)
    return phi


def _species(rng, n):
    """Draw species index, pdg id and charge for n soft particles."""
    sp = rng.choice(len(_SPECIES), size=n, p=_FRAC)
    neg = rng.random(n) < 0.5
    charged = _CHARGED[sp]
    q = np.where(charged, np.where(neg, -1, 1), 0).astype(np.int8)
    apdg = _ABS_PDG[sp]
    # Leptons: e-/mu- carry the positive pdg id; hadrons carry the charge sign.
    lepton = (apdg == 11) | (apdg == 13)
    sign = np.where(lepton, -q, q)
    pdg = np.where(charged, apdg * sign.astype(np.int32), apdg).astype(np.int32)
    return sp, pdg, q


def _soft(rng, n, pt_min, index):
    """Soft particles: pT = pt_min (1-u)^(-1/index) capped, flat eta and phi."""
    sp, pdg, q = _species(rng, n)
    u = rng.random(n)
    pt = np.minimum(pt_min * (1.0 - u) ** (-1.0 / index), PT_CAP).astype(np.float32)
    eta = rng.uniform(-ETA_MAX, ETA_MAX, n).astype(np.float32)
    phi = _phi32(rng, n)
    mass = _MASS[sp].astype(np.float32)
    return pt, eta, phi, mass, pdg, q


def make_tiny(n_events: int = 100, seed: int = 0) -> EventBatch:
    """Plain tiny workload: Poisson(50) soft particles per event."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(50.0, n_events)
    pt, eta, phi, mass, pdg, q = _soft(rng, int(counts.sum()), 0.5, 2.5)
    return EventBatch(_offsets(counts), pt, eta, phi, mass, pdg, q, None, "tiny")


def make_batched(n_events: int = 100_000, seed: int = 1) -> EventBatch:
    """Poisson(400) soft particles plus 4 hard objects per event.

    Hard objects follow the soft ones inside each event: two opposite-charge
    leptons of one flavour (e or mu, 50/50 per event) and two photons, each with
    pT ~ U(30, 300) GeV, |eta| < 2.5 uniform, phi uniform.
    """
    rng = np.random.default_rng(seed)
    soft_n = rng.poisson(400.0, n_events)
    counts = soft_n + 4
    off = _offsets(counts)
    n = int(off[-1])
    pt = np.empty(n, np.float32); eta = np.empty(n, np.float32)
    phi = np.empty(n, np.float32); mass = np.empty(n, np.float32)
    pdg = np.empty(n, np.int32); q = np.empty(n, np.int8)
    # index of each particle inside its event, and whether it is a hard object
    ev = np.repeat(np.arange(n_events), counts)
    local = np.arange(n, dtype=np.int64) - off[:-1][ev].astype(np.int64)
    hard = local >= soft_n[ev]
    ns = int((~hard).sum())
    s_pt, s_eta, s_phi, s_mass, s_pdg, s_q = _soft(rng, ns, 0.5, 2.5)
    pt[~hard] = s_pt; eta[~hard] = s_eta; phi[~hard] = s_phi
    mass[~hard] = s_mass; pdg[~hard] = s_pdg; q[~hard] = s_q
    # hard objects, 4 per event in a fixed order: l+, l-, gamma, gamma
    nh = 4 * n_events
    flav_mu = rng.random(n_events) < 0.5
    h_pt = rng.uniform(30.0, 300.0, nh).astype(np.float32)
    h_eta = rng.uniform(-2.5, 2.5, nh).astype(np.float32)
    h_phi = _phi32(rng, nh)
    slot = np.tile(np.arange(4), n_events)
    fmu = np.repeat(flav_mu, 4)
    apdg = np.where(fmu, 13, 11)
    h_q = np.select([slot == 0, slot == 1], [1, -1], 0).astype(np.int8)
    h_pdg = np.where(slot < 2, -apdg * h_q.astype(np.int32), 22).astype(np.int32)
    h_mass = np.where(slot < 2, np.where(fmu, _MASS[7], _MASS[6]), 0.0).astype(np.float32)
    pt[hard] = h_pt; eta[hard] = h_eta; phi[hard] = h_phi
    mass[hard] = h_mass; pdg[hard] = h_pdg; q[hard] = h_q
    return EventBatch(off, pt, eta, phi, mass, pdg, q, None, "batched")


def make_ee(n_events: int = 1_000_000, seed: int = 2, sqrt_s: float = 91.2) -> EventBatch:
    """e+e- events: Poisson(35) particles, isotropic, energies sum to sqrt_s.

    Energies w_i ~ Exp(1), E_i = sqrt_s * w_i / sum(w); |p| = sqrt(max(E^2 - m^2, 0));
    cos(theta) ~ U(-1, 1), phi ~ U[-pi, pi).  Species mix as the soft particles.
    """
    rng = np.random.default_rng(seed)
    counts = rng.poisson(35.0, n_events)
    off = _offsets(counts)
    n = int(off[-1])
    sp, pdg, q = _species(rng, n)
    w = rng.exponential(1.0, n)
    ev = np.repeat(np.arange(n_events), counts)
    wsum = np.bincount(ev, weights=w, minlength=n_events)
    e = sqrt_s * w / wsum[ev]
    m = _MASS[sp]
    p = np.sqrt(np.maximum(e * e - m * m, 0.0))
    u = rng.random(n)
    cos_t = 2.0 * u - 1.0
    cos_t = np.clip(cos_t, -1.0 + 1e-15, 1.0 - 1e-15)
    sin_t = np.sqrt(1.0 - cos_t * cos_t)
    pt = (p * sin_t).astype(np.float32)
    eta = np.arctanh(cos_t).astype(np.float32)
    phi = _phi32(rng, n)
    return EventBatch(off, pt, eta, phi, m.astype(np.float32), pdg, q, None, "ee")


def make_pileup(n_events: int = 10_000, seed: int = 3, n_vertices: int = 170,
                mu_pu: float = 30.0, sigma_z: float = 0.05, max_z: float = 0.25) -> EventBatch:
    """Hard event Poisson(400) at z = 0 plus n_vertices pile-up vertices.

    Each pile-up vertex holds Poisson(mu_pu) particles with pT = 0.3 (1-u)^(-1/3)
    (capped at 500 GeV) and flat |eta| < 4.9; its z ~ N(0, sigma_z) truncated to
    |z| < max_z (redrawn until inside).  Inside an event the hard particles come
    first, then the vertices in order.
    """
    rng = np.random.default_rng(seed)
    n_seg = n_vertices + 1
    seg_counts = np.empty((n_events, n_seg), dtype=np.int64)
    seg_counts[:, 0] = rng.poisson(400.0, n_events)
    seg_counts[:, 1:] = rng.poisson(mu_pu, (n_events, n_vertices))
    z = rng.normal(0.0, sigma_z, (n_events, n_vertices))
    bad = np.abs(z) >= max_z
    while bad.any():
        z[bad] = rng.normal(0.0, sigma_z, int(bad.sum()))
        bad = np.abs(z) >= max_z
    seg_z = np.zeros((n_events, n_seg), dtype=np.float64)
    seg_z[:, 1:] = z
    counts = seg_counts.sum(axis=1)
    off = _offsets(counts)
    n = int(off[-1])
    flat_counts = seg_counts.reshape(-1)
    is_pu = np.repeat(np.tile(np.arange(n_seg) > 0, n_events), flat_counts)
    vz = np.repeat(seg_z.reshape(-1), flat_counts).astype(np.float32)
    sp, pdg, q = _species(rng, n)
    u = rng.random(n)
    pt = np.where(is_pu, 0.3 * (1.0 - u) ** (-1.0 / 3.0), 0.5 * (1.0 - u) ** (-1.0 / 2.5))
    pt = np.minimum(pt, PT_CAP).astype(np.float32)
    eta = rng.uniform(-ETA_MAX, ETA_MAX, n).astype(np.float32)
    phi = _phi32(rng, n)
    return EventBatch(off, pt, eta, phi, _MASS[sp].astype(np.float32), pdg, q, vz, "pileup")


def make_minbias_pool(n_events: int = 10_000, seed: int = 5, mu: float = 30.0) -> EventBatch:
    """Minimum-bias interactions for pile-up merging: Poisson(mu) particles of
    the soft species mix, pT = 0.3 (1-u)^(-1/3) capped at 500 GeV, flat
    |eta| < 4.9; no vertex (the merger assigns one per interaction)."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(mu, n_events)
    n = int(counts.sum())
    sp, pdg, q = _species(rng, n)
    u = rng.random(n)
    pt = np.minimum(0.3 * (1.0 - u) ** (-1.0 / 3.0), PT_CAP).astype(np.float32)
    eta = rng.uniform(-ETA_MAX, ETA_MAX, n).astype(np.float32)
    phi = _phi32(rng, n)
    return EventBatch(_offsets(counts), pt, eta, phi, _MASS[sp].astype(np.float32), pdg, q, None, "minbias")


def make_hard(n_events: int = 10_000, seed: int = 6) -> EventBatch:
    """Hard-scatter events for pile-up merging: Poisson(400) soft particles at
    the origin (the pile-up workload's hard event)."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(400.0, n_events)
    pt, eta, phi, mass, pdg, q = _soft(rng, int(counts.sum()), 0.5, 2.5)
    return EventBatch(_offsets(counts), pt, eta, phi, mass, pdg, q, None, "hard")


WORKLOADS = {
    "tiny": (make_tiny, "cms_like", 100),
    "batched": (make_batched, "cms_like", 100_000),
    "ee": (make_ee, "ee_like", 1_000_000),
    "pileup": (make_pileup, "cms_like", 10_000),
}


def make(name: str, n_events: Optional[int] = None) -> EventBatch:
    fn, _card, n_def = WORKLOADS[name]
    return fn(n_events=n_def if n_events is None else n_events)


def card_for(name: str) -> str:
    return WORKLOADS[name][1]


def from_particles(events: list) -> EventBatch:
    """Build a batch from explicit per-event particle lists (hand-made test events).

    Each event is a list of tuples (pt, eta, phi, mass, pdg, charge[, vz]).
    """
    counts = np.array([len(ev) for ev in events], dtype=np.int64)
    rows = [p for ev in events for p in ev]
    has_vz = any(len(p) > 6 for p in rows)
    col = lambda k, dt: np.array([p[k] for p in rows], dtype=dt) if rows else np.zeros(0, dt)
    vz = None
    if has_vz:
        vz = np.array([p[6] if len(p) > 6 else 0.0 for p in rows], dtype=np.float32)
    return EventBatch(_offsets(counts), col(0, np.float32), col(1, np.float32),
                      col(2, np.float32), col(3, np.float32), col(4, np.int32),
                      col(5, np.int8), vz, "hand")


# ---------------------------------------------------------------------------
# serving workload
# ---------------------------------------------------------------------------
SERVING_GENERATORS = ("batched", "ee", "pileup")
SERVING_CARDS = ("cms_like", "atlas_like", "ee_like")


@dataclasses.dataclass
class Request:
    t_arrival: float      # seconds after the start
    generator: str        # which event pool the events come from
    card: str             # detector card of the request
    n_events: int
    start: int            # first event of the request in its pool
    seed: int


def serving_schedule(rate_hz: float, duration_s: float, pool_events: int = 5000,
                     seed: int = 4, max_events: int = 5000) -> list:
    """Poisson arrivals at rate_hz for duration_s; each request holds
    log-uniform(1, max_events) events from a generator drawn uniformly among the
    batched, e+e- and pile-up workloads, with a card drawn uniformly among the
    three; its events are a random contiguous range of that generator's pool."""
    rng = np.random.default_rng(seed + int(rate_hz * 1000))
    out = []
    t = 0.0
    k = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n = int(np.floor(np.exp(rng.uniform(0.0, np.log(max_events + 1)))))
        n = max(1, min(n, max_events, pool_events))
        gen = SERVING_GENERATORS[int(rng.integers(3))]
        card = SERVING_CARDS[int(rng.integers(3))]
        start = int(rng.integers(0, pool_events - n + 1))
        out.append(Request(t, gen, card, n, start, 1000 + k))
        k += 1
    return out


def serving_pools(pool_events: int = 5000) -> dict:
    """The event pools the serving requests slice (one per generator)."""
    return {"batched": make_batched(pool_events, seed=11), "ee": make_ee(pool_events, seed=12),
            "pileup": make_pileup(pool_events, seed=13)}
