// The fused detector-response kernel (sm_103a).
//
// One persistent launch walks a ragged CSR batch.  A "team" of TEAM threads
// (a warp ... a whole CTA) owns one event at a time and runs the TorchDelphes
// chain of the paper (Sec. 2.2, App. D.1) plus the isolation of Sec. 2.4:
//
//   phase 1, per particle (chunks of TEAM particles, coalesced SoA loads):
//     S0 classify, S1 propagate to the calorimeter surface, S2 tracking
//     efficiency, S3 momentum smearing, S4 e/mu/gamma identification and
//     smearing, S5 tower lookup and deposit into the event's tower table;
//     tracks and candidates are compacted in particle order (warp ballot +
//     team scan) straight into their output slots.
//   phase 2, per tower (each tower is processed by its lowest-index
//     depositing particle, so towers come out in a deterministic order):
//     S6 tower smearing and thresholds, S7 energy-flow subtraction.
//   phase 3, per event with candidates: S8 cone isolation over the event's
//     energy-flow tracks and neutrals.
//   S9: per-event counts.
//
// Each CTA first copies the card's hot tables (ring edges, per-segment tower
// bases and phi tables, per-ring centres, efficiency and resolution tables,
// about 13 KB for the CMS-like card) into shared memory: placing a deposit
// then needs no global-memory lookups.  Tower sums are exact 64-bit
// fixed-point integer sums (quantum 2^-36 GeV): the first depositor of a tower
// stores its value, later ones add with shared-memory integer atomics, so the
// sums are bitwise deterministic without float atomics and independent of the
// launch shape.  Random numbers are counter-based (Philox4x32-10 keyed by seed,
// counter (slot, event, purpose, 0)), so every draw is reproducible and
// independent of scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "pdr_ff.cuh"
#include "pdr_internal.h"
#include "pdr_ip.cuh"
#include "pdr_math.cuh"

namespace pdr {

// ---------------------------------------------------- bounds-checking build
// Built with -DPDR_BOUNDS (libpdr_bounds.so, a debug build of the library):
// every index into a batch array (inputs, outputs, debug records) is checked
// against the batch's end offsets[n_events], every event index against
// n_events and every table index against the table's size.  An index out of
// range sets a sticky flag and is replaced by 0 (an index inside the array),
// so the access never leaves the arrays; each team ORs the flag into the
// launch's error word (ERR_BOUNDS) when it finishes.  In the normal build the
// checks are the identity.
#ifdef PDR_BOUNDS
__device__ uint32_t g_bounds_flag;
__device__ __forceinline__ uint64_t bchk(uint64_t i, uint64_t n) {
  if (i < n) return i;
  atomicOr(&g_bounds_flag, 1u);
  return 0;
}
#define PDR_B(S, i) bchk((uint64_t)(i), (S).offsets[(S).n_events])
#define PDR_BE(S, e) bchk((uint64_t)(e), (S).n_events)
#define PDR_BT(i, n) ((uint32_t)bchk((uint64_t)(i), (uint64_t)(n)))
#else
#define PDR_B(S, i) (i)
#define PDR_BE(S, e) (e)
#define PDR_BT(i, n) (i)
#endif

// Log-normal with mean x and relative variance rel2 = (sigma/x)^2.
__device__ __forceinline__ float lognormal(float x, float rel2, float z) {
  const float s2 = log1p_pos(rel2);
  const float s = sqrt_approx(s2);
  return x * expf(fmaf(s, z, -0.5f * s2));
}

// (sigma/x)^2 = a^2/x + b^2/x^2 + c^2 + d^2 x^2, coefficients r = (a^2, b^2, c^2, d^2).
__device__ __forceinline__ float rel2_of(float4 r, float x) {
  const float ix = rcp_approx(x);
  return fmaf(fmaf(r.y, ix, r.x), ix, fmaf(r.w * x, x, r.z));
}

// Largest k < n with edges[k] <= x (-1 if none): piecewise-constant tables.
// The card pads each table to PDR_MAXEDGE edges with +inf, so for sorted edges
// the count of edges <= x is that index plus one (two vector loads).
__device__ __forceinline__ int small_lookup(const float* edges, int n, float x) {
  const float4 a = *reinterpret_cast<const float4*>(edges);
  const float4 b = *reinterpret_cast<const float4*>(edges + 4);
  const int c = (int)(a.x <= x) + (int)(a.y <= x) + (int)(a.z <= x) + (int)(a.w <= x) +
                (int)(b.x <= x) + (int)(b.y <= x) + (int)(b.z <= x) + (int)(b.w <= x);
  return min(c, n) - 1;
}

// Fixed-point energy (quantum 2^-36 GeV) with 32-bit conversions only: the
// integer part of 16 v in the high word, the remaining fraction times 2^32 in
// the low word (the split is exact; only the low word is rounded).
__device__ __forceinline__ unsigned long long to_fp(float v) {
  const float x = v * 16.0f;
  const float hi = truncf(x);
  const float frac = x - hi;
  const uint32_t h = __float2uint_rz(hi);
  const uint32_t l = __float2uint_rn(frac * 4294967296.0f);
  return ((unsigned long long)h << 32) | l;
}

__device__ __forceinline__ float from_fp(unsigned long long v) {
  const float hi = __uint2float_rn((uint32_t)(v >> 32));
  const float lo = __uint2float_rn((uint32_t)v);
  return fmaf(hi, 4294967296.0f, lo) * PDR_FP_INV;
}

__device__ __forceinline__ int classify(int32_t pdg, int q) {
  const int a = pdg < 0 ? -pdg : pdg;
  if (a == 11) return CLS_E;
  if (a == 13) return CLS_MU;
  if (a == 22) return CLS_GAMMA;
  if (a == 12 || a == 14 || a == 16) return CLS_INVIS;
  return q != 0 ? CLS_CHAD : CLS_NHAD;
}

// ------------------------------------------------------------- propagation
struct Prop {
  int reach, barrel;
  float eta_pos, phi_pos;
};

// S1: straight line (neutral, or B = 0) or helix from (0, 0, vz) to the
// cylinder R, +-L.  Helix radius r = pT / (0.299792458 |q| |B|); the barrel is
// reached iff 2 pT >= c = 0.299792458 |q| |B| R, at turning angle
// 2 asin(c / 2pT); otherwise the endcap after psi = s_z / r < 2 pi.  Both
// crossings are computed for every particle and the valid one is selected
// (one path for the warp instead of four).  UNIFORM: the near-loop
// recomputation below runs as a warp-uniform branch over the lanes that need
// it (one-warp teams, whose warps run apart); otherwise as a divergent branch
// around an out-of-line call.
template <bool UNIFORM>
__device__ __forceinline__ Prop propagate(const HotCard& K, float pt, float eta, float sh, float phi,
                                          int q, float vz) {
  const bool charged = q != 0 && K.has_field;
  const int aq = q < 0 ? -q : q;
  const float kq = K.kB * (float)aq;
  const float r = fdiv(pt, kq);
  const float h = ((q > 0) == (K.Bsign > 0)) ? 1.0f : -1.0f;
  const int qi = min(aq, PDR_MAXQ);
  const float cR = aq <= PDR_MAXQ ? K.cR_hi[qi] : kq * K.R;
  const float cRl = aq <= PDR_MAXQ ? K.cR_lo[qi] : 0.0f;
  const float twopt = 2.0f * pt;
  // barrel: half turning angle a = asin(x), x = c / 2pT; near the tangent
  // point (x > 1/2) through pi/2 - 2 asin(sqrt((1 - x)/2)) with
  // 1 - x = (2pT - c) / 2pT, where 2pT - c_hi is exact (Sterbenz)
  const float x = fdiv(cR, twopt);
  const bool near = x > 0.5f;
  const float omx = fmaxf(fdiv((twopt - cR) - cRl, twopt), 0.0f);
  const float as = asin_half(near ? sqrt_approx(0.5f * omx) : fminf(x, 0.5f));
  const float a = near ? (PIO2_HI - 2.0f * as) + PIO2_LO : as;
  // crossing z: helix 2 r a sinh(eta), straight line R sinh(eta)
  const float zb = fmaf(charged ? 2.0f * r * a : K.R, sh, vz);
  const bool barrel = (!charged || twopt >= cR) && fabsf(zb) <= K.L;
  // endcap: the transverse distance rho at z = +-L is s_z = (z_e - vz) / sinh(eta)
  // for a straight line, 2 r sin(psi / 2) for the helix, psi = s_z / r taken as
  // (z_e - vz) kq / (pT sinh(eta)) (relative error below 7.5e-7: the card's L
  // to float32 and its remainder, six roundings, sinh's 4e-7 and the
  // reciprocal's 2^-23)
  const float ze = sh > 0.0f ? K.L : -K.L;
  const float dz = (ze - vz) + (sh > 0.0f ? K.L_lo : -K.L_lo);   // z_e - vz with the card's L to 2^-48
  const float sz = fdiv(dz, sh);
  const float psi = dz * kq * rcp_approx(pt * sh);
  const float yh = 0.5f * psi;
  const float sy = sin_half_turn(fminf(yh, PI_F));
  bool endcap = sh != 0.0f && (!charged || psi < TWO_PI_F);  // else pz = 0, or a looper
  // a straight line from the axis origin keeps its direction
  const bool origin = !charged && vz == 0.0f;
  // (rho = 2 r |sin(psi / 2)|: psi < 0 for a vertex just beyond the endcap plane)
  float eta_s = origin ? eta : asinh_fast(barrel ? fdiv(zb, K.R) : fdiv(ze, charged ? 2.0f * r * fabsf(sy) : sz));
  // A helix that has nearly closed (psi / 2 -> pi): eta_pos carries psi's
  // relative error times |(psi/2) cot(psi/2)| = (psi/2) cos(d) / sin(d),
  // d = pi - psi/2, on top of the endcap path's other roundings (below
  // 6e-7 + 2.5e-7 max(|eta_pos|, 1)).  Where that sum could pass
  // 2e-6 max(|eta_pos|, 1), pi - psi/2 is recomputed in float-float
  // (half_turn_gap) and the loop decision taken on it.
  const bool near_loop = charged && !barrel && yh >= 1.6f && yh <= 3.1417f &&
                         !(7.5e-7f * yh * sqrt_approx(fmaf(-sy, sy, 1.0f)) <=
                           fmaf(1.75e-6f, fmaxf(fabsf(eta_s), 1.0f), -6e-7f) * sy);
  if constexpr (UNIFORM) {
    if (__any_sync(__activemask(), near_loop)) {
      const float g = half_turn_gap(pt, eta, vz, aq, K.L, K.L_lo, K.kB, K.kB_lo);
      const float es = asinh_fast(fdiv(ze, 2.0f * r * sin_quarter(fmaxf(g, 0.0f))));
      endcap = near_loop ? g > 0.0f : endcap;
      eta_s = near_loop ? es : eta_s;
    }
  } else if (near_loop) {
    const float g = half_turn_gap_call(pt, eta, vz, aq, K.L, K.L_lo, K.kB, K.kB_lo);
    endcap = g > 0.0f;
    eta_s = asinh_fast(fdiv(ze, 2.0f * r * sin_quarter(fmaxf(g, 0.0f))));
  }
  Prop P;
  P.reach = (fabsf(vz) <= K.L) && (barrel || endcap);
  P.barrel = P.reach && (origin ? fabsf(K.R * sh) <= K.L : barrel);
  P.eta_pos = P.reach ? eta_s : 0.0f;
  const float turn = charged ? h * (barrel ? a : 0.5f * psi) : 0.0f;
  float pphi = phi - turn;
  pphi = pphi < -PI_F ? pphi + TWO_PI_F : (pphi >= PI_F ? pphi - TWO_PI_F : pphi);
  P.phi_pos = P.reach ? pphi : 0.0f;
  return P;
}

// Ring record of the shared-memory card: x = eta_c, y = 1 / cosh(eta_c),
// z = first tower id (int bits), w = phi-table offset | nphi << 16 | row << 27.
__device__ __forceinline__ float4 ring_rec(const HotCard& K, const float* KD, int calo, int r) {
  return reinterpret_cast<const float4*>(KD + K.calo[calo].ring_off)[r];
}

// S5 tower of a surface position in one calorimeter, from the shared-memory
// card: ring = largest r with edge[r] <= eta (guessed from the segment's
// uniform binning, then checked against the float32 edges), phi bin likewise
// from the ring's record, tower id = the ring's first id + phi bin.  Returns
// false outside coverage.
__device__ __forceinline__ bool tower_of(const HotCard& K, const float* KD, int calo, float v, float phi,
                                         uint32_t& id, int& ring) {
  const HotCalo& C = K.calo[calo];
  const float* edge = KD + C.edge_off;
  const int nr = C.nring;
  if (!(v >= edge[0]) || !(v < edge[nr])) return false;
  const float av = fabsf(v);
  int s = 0;
  while (s < C.nseg - 1 && av >= C.seg[s].hi) ++s;
  int j = (int)((av - C.seg[s].lo) * C.seg[s].scale);
  j = min(max(j, 0), C.seg[s].n - 1) + C.seg[s].first;
  const int m = C.m;
  int r = v >= 0.0f ? m + j : m - 1 - j;
  r = min(max(r, 0), nr - 1);
  while (r > 0 && v < edge[r]) --r;
  while (r < nr - 1 && v >= edge[r + 1]) ++r;
  const float4 rec = ring_rec(K, KD, calo, r);
  const uint32_t w = __float_as_uint(rec.w);
  const int nphi = (int)((w >> 16) & 0x7FFu);
  const float* pe = KD + (w & 0xFFFFu);
  // phi bin: largest k with edge[k] <= phi, clamped to [0, nphi - 1]
  int k = (int)((phi + PI_F) * ((float)nphi * (1.0f / TWO_PI_F)));
  k = min(max(k, 0), nphi - 1);
  while (k > 0 && phi < pe[k]) --k;
  while (k < nphi - 1 && phi >= pe[k + 1]) ++k;
  id = (uint32_t)(__float_as_int(rec.z) + k);
  ring = r;
  return true;
}

// phi_c of tower id in a known ring.
__device__ __forceinline__ float tower_phi_c(const HotCard& K, const float* KD, int calo, uint32_t id, int r) {
  const float4 rec = ring_rec(K, KD, calo, r);
  const uint32_t w = __float_as_uint(rec.w);
  return KD[(w & 0xFFFFu) + ((w >> 16) & 0x7FFu) + 1 + ((int)id - __float_as_int(rec.z))];
}

// Ring, eta_c and phi_c of a tower id.
__device__ __forceinline__ void tower_decode(const HotCard& K, const float* KD, int calo, uint32_t id,
                                             int& ring, float& eta_c, float& phi_c) {
  const HotCalo& C = K.calo[calo];
  const int m = C.m;
  int r = 0;
  for (int s = 0; s < C.nseg; ++s) {
    const HotSeg& S = C.seg[s];
    const uint32_t span = (uint32_t)(S.n * S.nphi);
    if (id - (uint32_t)S.base_neg < span) r = (m - S.first - S.n) + (int)((id - (uint32_t)S.base_neg) / (uint32_t)S.nphi);
    else if (id - (uint32_t)S.base_pos < span) r = m + S.first + (int)((id - (uint32_t)S.base_pos) / (uint32_t)S.nphi);
  }
  ring = r;
  eta_c = ring_rec(K, KD, calo, r).x;
  phi_c = tower_phi_c(K, KD, calo, id, r);
}

// ------------------------------------------------------------------ teams
template <int TEAM>
struct TeamCtx {
  int tid, tix;
  __device__ __forceinline__ void sync() const {
    if (TEAM == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(tix + 1), "r"(TEAM) : "memory");
  }
};

// Exclusive team prefix of two flags packed as (a | b << 16); total via ref.
// Includes a team barrier (a warp barrier for one-warp teams).
template <int TEAM>
__device__ __forceinline__ uint32_t team_scan2(bool fa, bool fb, uint32_t* wbuf, uint32_t& total,
                                               const TeamCtx<TEAM>& t) {
  const uint32_t ma = __ballot_sync(PDR_FULL, fa), mb = __ballot_sync(PDR_FULL, fb);
  const int lane = t.tid & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t lane_pre = __popc(ma & lt) | ((uint32_t)__popc(mb & lt) << 16);
  const uint32_t wtot = __popc(ma) | ((uint32_t)__popc(mb) << 16);
  if (TEAM == 32) {
    __syncwarp();  // orders the lanes' shared-memory writes before what follows
    total = wtot;
    return lane_pre;
  }
  constexpr int NW = TEAM / 32;
  const int w = t.tid >> 5;
  if (lane == 0) wbuf[w] = wtot;
  t.sync();
  uint32_t v = lane < NW ? wbuf[lane] : 0u;
#pragma unroll
  for (int o = 1; o < NW; o <<= 1) {
    const uint32_t u = __shfl_up_sync(PDR_FULL, v, o);
    if (lane >= o) v += u;
  }
  total = __shfl_sync(PDR_FULL, v, NW - 1);
  const uint32_t incl_w = __shfl_sync(PDR_FULL, v, w);
  return incl_w - wtot + lane_pre;
}

// ------------------------------------------------------- per-particle stage
// Phase 1a of a particle: S0, S1 and the tower of S5, plus its smearing job,
// if any: a tracking job (S2, S3, and S4 for a tracked e/mu) for a charged
// particle that reached the surface inside a tracking-efficiency bin with
// non-zero efficiency, or an identification job (S4) for a photon in ECAL
// above the candidate pT floor.  Jobs run afterwards from a dense list in
// particle order, so the warps that hold no job skip their arithmetic.
struct PartA {
  uint32_t key, ring, flags, job;  // job: entry below, or PDR_EMPTY
  float E, eta_pos, phi_pos;
};

// Job entry: particle index (16 bits) | pT bin << 16 | |eta| bin << 20 |
// tracking-efficiency table (0 hadron, 1 electron, 2 muon) << 24 | photon << 28.
#define PDR_JOB_PHOTON (1u << 28)

template <int TEAM>
__device__ __forceinline__ void particle_stage_a(const KSeg& S, const HotCard& K, const float* KD,
                                                 uint64_t g, uint32_t i, PartA& o) {
  g = PDR_B(S, g);
  const float PT = __ldg(S.pt + g), ETA = __ldg(S.eta + g), PHI = __ldg(S.phi + g);
  const float M = __ldg(S.mass + g);
  const int32_t PDG = __ldg(S.pdg + g);
  const int Q = (int)__ldg(S.charge + g);
  const float VZ = S.vz ? __ldg(S.vz + g) : 0.0f;
  o.key = PDR_NO_KEY; o.ring = 0; o.flags = 0; o.job = PDR_EMPTY;
  o.eta_pos = 0.0f; o.phi_pos = 0.0f;
  const int cls = classify(PDG, Q);
  float ch, sh;
  cosh_sinh(ETA, ch, sh);
  const float pc = PT * ch;
  o.E = sqrt_approx(fmaf(pc, pc, M * M));
  if (cls == CLS_INVIS) return;
  // S1
  const Prop P = propagate<TEAM == 32>(K, PT, ETA, sh, PHI, Q, VZ);
  if (!P.reach) return;
  o.flags = PDR_F_REACH | (P.barrel ? PDR_F_BARREL : 0u);
  o.eta_pos = P.eta_pos;
  o.phi_pos = P.phi_pos;
  // S5 tower placement: e/gamma to ECAL (or HCAL beyond ECAL), hadrons to HCAL
  int calo = -1, ring = -1;
  uint32_t id = 0;
  const bool em = cls == CLS_E || cls == CLS_GAMMA;
  if (em || cls == CLS_CHAD || cls == CLS_NHAD) {
    const float* e0 = KD + K.calo[0].edge_off;
    const int cal = (em && P.eta_pos >= e0[0] && P.eta_pos < e0[K.calo[0].nring]) ? 0 : 1;
    if (tower_of(K, KD, cal, P.eta_pos, P.phi_pos, id, ring)) calo = cal;
  }
  if (calo >= 0) {
    o.key = ((uint32_t)calo << 24) | id;
    o.ring = (uint32_t)ring;
    o.flags |= calo == 0 ? PDR_F_ECAL : PDR_F_HCAL;
  }
  if (Q != 0) {
    const int tc = cls == CLS_E ? 1 : (cls == CLS_MU ? 2 : 0);
    const int kp = small_lookup(K.trk_pt_edges, K.trk_npt, PT);
    const int ke = small_lookup(K.trk_eta_edges, K.trk_neta, fabsf(ETA));
    if (kp >= 0 && ke >= 0 && K.trk_T[tc][kp][ke] != 0ull)
      o.job = i | ((uint32_t)kp << 16) | ((uint32_t)ke << 20) | ((uint32_t)tc << 24);
  } else if (cls == CLS_GAMMA && calo == 0 && PT > K.cand_ptmin) {
    o.job = i | PDR_JOB_PHOTON;
  }
}

// Phase 1b: one job.  Each stage is an efficiency draw and, if accepted, a
// log-normal smearing: S2 + S3 for a tracking job (then S4 for a tracked e/mu
// above the candidate pT floor), S4 alone for a photon.  Returns the smeared
// track pT and energy and the candidate pT and class through the references.
struct JobOut {
  bool tracked, cand;
  float ptp, etrk, cpt;
  int cc;
};

__device__ __forceinline__ void run_job(const KSeg& S, const HotCard& K, uint64_t a, uint32_t job,
                                        uint32_t event, JobOut& r) {
  const uint32_t i = job & 0xFFFFu;
  const bool photon = (job & PDR_JOB_PHOTON) != 0u;
  const uint64_t g = PDR_B(S, a + i);
  const float PT = __ldg(S.pt + g), ETA = __ldg(S.eta + g), M = __ldg(S.mass + g);
  const float aeta = fabsf(ETA);
  float ch, sh;
  cosh_sinh(ETA, ch, sh);
  const float pc = PT * ch;
  const float E = sqrt_approx(fmaf(pc, pc, M * M));
  r.tracked = false; r.cand = false; r.ptp = 0.0f; r.etrk = 0.0f; r.cpt = 0.0f;
  // first stage
  uint32_t purpose;
  unsigned long long T;
  int comp;
  float x;
  if (!photon) {
    const int kp = (int)((job >> 16) & 15u), ke = (int)((job >> 20) & 15u), tc = (int)((job >> 24) & 3u);
    purpose = 1u; T = K.trk_T[tc][kp][ke]; comp = RES_TRACK; x = PT;
    r.cc = tc == 1 ? 0 : (tc == 2 ? 1 : -1);
  } else {
    const int ke = small_lookup(K.id_edges, K.id_n, aeta);
    purpose = 2u; T = ke >= 0 ? K.id_T[2][ke] : 0ull; comp = RES_ECAL; x = E;
    r.cc = 2;
  }
  for (;;) {
    bool ok = false;
    float sm = 0.0f;
    if (T != 0ull) {
      const uint4 w = philox(i, event, purpose, 0u, S.rk);
      if ((unsigned long long)w.x < T) {
        ok = true;
        const float z = normal(w.y, w.z);
        const int rb = max(small_lookup(K.res_edges[comp], K.res_n[comp], aeta), 0);
        const float r2 = rel2_of(K.res[comp][rb], x);
        sm = lognormal(x, r2, z);
      }
    }
    if (purpose == 2u) {  // identification stage: done
      r.cand = ok;
      if (ok) r.cpt = r.cc != 1 ? sm / ch : sm;
      return;
    }
    r.tracked = ok;
    if (!ok) return;
    r.ptp = sm;
    const float pcp = sm * ch;
    r.etrk = sqrt_approx(fmaf(pcp, pcp, M * M));
    if (r.cc < 0 || !(PT > K.cand_ptmin)) return;
    // a tracked e/mu goes on to identification
    const int ke = small_lookup(K.id_edges, K.id_n, aeta);
    purpose = 2u; T = ke >= 0 ? K.id_T[r.cc][ke] : 0ull;
    comp = r.cc == 0 ? RES_ECAL : RES_MUON; x = r.cc == 0 ? E : PT;
  }
}

// Adds v to the 64-bit fixed-point sum at p with two native 32-bit atomics (a
// 64-bit shared-memory atomic add is a compare-and-swap loop): the low word,
// then the high word plus the carry out of the low word.  Every term's carry
// is added exactly once, so the sum is exact in any order.
__device__ __forceinline__ void fp_add(unsigned long long* p, unsigned long long v) {
  uint32_t* w = reinterpret_cast<uint32_t*>(p);
  const uint32_t lo = (uint32_t)v;
  const uint32_t old = atomicAdd(w, lo);
  const uint32_t hi = (uint32_t)(v >> 32) + (old + lo < old ? 1u : 0u);
  if (hi != 0u) atomicAdd(w + 1, hi);
}

// ------------------------------------------------------------ tower table
// Per-team open-addressing table (linear probing, multiplicative hash) keyed
// by tower key; per particle an info word (slot | ring << 16, or empty); the
// event's job list.  Between events every key is empty; the
// other slot fields are initialised by the thread that claims the slot.
struct Tbl {
  unsigned char* base;
  uint32_t nslots;  // any multiple of 32 (the hash is scaled, not masked)
  uint32_t nmax;    // particles per event
  // field addresses are recomputed from the base (fewer live registers)
  __device__ __forceinline__ uint32_t* keys() const { return reinterpret_cast<uint32_t*>(base); }
  __device__ __forceinline__ uint32_t* owner() const { return reinterpret_cast<uint32_t*>(base) + nslots; }
  __device__ __forceinline__ unsigned long long* esum() const {
    return reinterpret_cast<unsigned long long*>(base + 8ull * nslots);
  }
  __device__ __forceinline__ unsigned long long* etrk() const {
    return reinterpret_cast<unsigned long long*>(base + 16ull * nslots);
  }
  __device__ __forceinline__ uint32_t* pinfo() const { return reinterpret_cast<uint32_t*>(base + 24ull * nslots); }
  // smearing jobs of the event, in particle order
  __device__ __forceinline__ uint32_t* jobs() const { return pinfo() + nmax; }
};

// Set when the block's shared table fills up, in kernels built for a shared
// table sized below the particle count (one team a block); see process_event.
__shared__ uint32_t s_table_full;

__device__ __forceinline__ Tbl carve(unsigned char* base, uint32_t slots, uint32_t nmax) {
  Tbl t;
  t.base = base;
  t.nslots = slots;
  t.nmax = nmax;
  return t;
}

// Find or claim the slot of key (each probe is one compare-and-swap, which also
// reads the slot).  The thread that claims an empty slot writes
// its own deposit, track energy and index with plain stores (before the team
// barrier that precedes any accumulation); every other depositor adds with
// atomics after that barrier.  Returns the slot; *claimed tells which case.
template <bool OVF>
__device__ __forceinline__ uint32_t table_insert(const Tbl& T, uint32_t key, uint32_t i,
                                                 unsigned long long e_fp, unsigned long long t_fp,
                                                 bool* claimed, uint32_t* err) {
  // multiplicative hash scaled to [0, nslots): the high word of h * nslots
  uint32_t h = PDR_BT(__umulhi(key * 0x9E3779B1u, T.nslots), T.nslots);
  *claimed = false;
  for (uint32_t probe = 0; probe < T.nslots; ++probe) {
    const uint32_t prev = atomicCAS(&T.keys()[h], PDR_EMPTY, key);
    if (prev == PDR_EMPTY) {
      T.owner()[h] = i;
      T.esum()[h] = e_fp;
      T.etrk()[h] = t_fp;
      *claimed = true;
      return h;
    }
    if (prev == key) return h;
    h = h + 1 == T.nslots ? 0u : h + 1;
  }
  // full: OVF flags it for the block (read after the particle phase, which
  // then hands the event to a larger table); otherwise it is an error
  if constexpr (OVF) s_table_full = 1u;
  else atomicOr(err, ERR_TABLE);
  return PDR_EMPTY;
}

// ---------------------------------------------------------- per-tower stage
struct TowerOut {
  float e, et, de, det;
  bool kept, ef;
};

__device__ __forceinline__ void tower_stage(const HotCard& K, const float* KD, uint32_t key,
                                            uint32_t ring, unsigned long long es, unsigned long long et,
                                            uint32_t event, const uint32_t* rk, TowerOut& o) {
  const int calo = (int)(key >> 24);
  const uint32_t id = key & 0xFFFFFFu;
  const float4 rec = ring_rec(K, KD, calo, (int)ring);
  const float ich = rec.y;  // 1 / cosh(eta_c)
  const int rb = (int)(__float_as_uint(rec.w) >> 27);
  const int comp = calo == 0 ? RES_ECAL : RES_HCAL;
  const float4 rc = K.res[comp][rb];
  const float Es = from_fp(es);
  const float Et = from_fp(et);
  const uint4 w = philox(id, event, 3u + (uint32_t)calo, 0u, rk);
  const float z = normal(w.x, w.y);
  const float E1 = lognormal(Es, rel2_of(rc, Es), z);
  // E'/sigma(E') = 1 / sqrt(rel2(E')); dE/sigma(E') = dE / E' * that
  const float rs = rsqrtf(rel2_of(rc, E1));
  const float emin = K.e_min[calo], smin = K.s_min[calo];
  o.kept = (E1 > emin) & (rs > smin);
  o.e = E1;
  o.et = E1 * ich;
  const float dE = E1 - Et;
  o.ef = (dE > emin) & (dE * rs > smin * E1);
  o.de = dE;
  o.det = dE * ich;
}

// ------------------------------------------------------------ isolation
#define PDR_ISO_TRACK 0x80000000u    // object tag: a track (particle index), else a tower key

// Staged candidates mark their eta bin and both neighbours in a bit mask per
// bin (bins at least 1.001 cone radii wide, over [-8, 8], the ends clamped), so
// an object only tests the candidates of its own bin's mask - usually none.
__device__ __forceinline__ int iso_bin(const HotCard& K, float eta) {
  const int b = (int)((eta + 8.0f) * K.iso_inv_w);
  return min(max(b, 0), K.iso_nbin - 1);
}

// Adds an object's fixed-point pT to every staged candidate whose cone
// ΔR_min <= ΔR < ΔR_max holds it, skipping the object built from the
// candidate itself (its own track, by particle index, or the EFlow neutral of
// its own tower, by key).
__device__ __forceinline__ void iso_object(const HotCard& K, float4 obj, TeamTail& tt) {
  uint32_t m = tt.binmask[iso_bin(K, obj.x)];
  if (m == 0u) return;
  const uint32_t tag = __float_as_uint(obj.w);
  const bool is_trk = (tag & PDR_ISO_TRACK) != 0u;
  const uint32_t oid = tag & ~PDR_ISO_TRACK;
  const unsigned long long wgt = to_fp(obj.z);
  do {
    const uint32_t c = __ffs(m) - 1;
    m &= m - 1u;
    const float4 cv = tt.cf[c];
    if (is_trk ? (oid == __float_as_uint(cv.w)) : (oid == tt.ckey[c])) continue;
    const float de = obj.x - cv.x;
    float dp = obj.y - cv.y;
    if (dp >= PI_F) dp -= TWO_PI_F;
    else if (dp < -PI_F) dp += TWO_PI_F;
    const float dr2 = fmaf(de, de, dp * dp);
    if (dr2 < K.dr2max && dr2 >= K.dr2min) fp_add(&tt.csum[c], wgt);
  } while (m != 0u);
}

// ------------------------------------------------------------- one event
// A team of TEAM threads walks the event in chunks of TEAM particles:
//   1a  particles: S0, S1, S5 placement and deposit; the smearing jobs, in
//       particle order (one team scan per chunk)
//   1b  smearing jobs (S2, S3, S4), team-strided over the job list; tracks
//       and candidates in particle order; candidates staged for the isolation
//   2   towers (S6, S7) by their lowest-index depositor, records in that
//       order; EFlow neutrals and tracks add their pT to the staged
//       candidates' cones (S8)
//   3   isolation results; candidates beyond the staged ones loop over all
//       EFlow objects
// OVF: the table is a shared table sized below the particle count.  One that
// fills up sets s_table_full, and the function returns false after the
// particle phase, having written nothing but debug records, so that the
// caller redoes the event with a larger table.  (Otherwise a full table, which
// sizing by particle count rules out, reports an error.)
template <int TEAM, bool OVF, bool IP>
__device__ __forceinline__ bool process_event(const KSeg& S, uint32_t* err, const HotCard& K, const float* KD,
                                              const Tbl& T, TeamTail& tt, const TeamCtx<TEAM>& tc, uint64_t e,
                                              uint64_t a, uint32_t n) {
  const uint32_t event = S.event_base + (uint32_t)e;
  const bool dbg = S.debug != nullptr;
  uint32_t n_trk = 0, n_cand = 0, flip = 0;

  // ---- 1a: particles (S0, S1, S5 placement and deposit); job list
  uint32_t n_job = 0;
  for (uint32_t c0 = 0; c0 < n; c0 += TEAM) {
    const uint32_t i = c0 + (uint32_t)tc.tid;
    const bool valid = i < n;
    PartA o;
    o.key = PDR_NO_KEY; o.E = 0.0f; o.job = PDR_EMPTY;
    if (valid) particle_stage_a<TEAM>(S, K, KD, a + i, i, o);
    uint32_t slot = PDR_EMPTY;
    bool claimed = false;
    const unsigned long long e_fp = to_fp(o.E);
    if (valid && o.key != PDR_NO_KEY) slot = table_insert<OVF>(T, o.key, i, e_fp, 0ull, &claimed, err);
    if (valid) T.pinfo()[PDR_BT(i, T.nmax)] = slot == PDR_EMPTY ? PDR_EMPTY : (slot | (o.ring << 16));
    const bool has_job = o.job != PDR_EMPTY;
    uint32_t tot;
    const uint32_t pre = team_scan2<TEAM>(has_job, false, tt.wbuf + 32 * flip, tot, tc);
    flip ^= 1u;
    if (slot != PDR_EMPTY && !claimed) {  // after the barrier that orders the claimers' stores
      fp_add(&T.esum()[slot], e_fp);
      atomicMin(&T.owner()[slot], i);
    }
    if (has_job) T.jobs()[PDR_BT(n_job + (pre & 0xFFFFu), T.nmax)] = o.job;
    if (dbg && valid)
      reinterpret_cast<float4*>(S.debug)[PDR_B(S, a + i)] =
          make_float4(__uint_as_float(o.key), o.eta_pos, o.phi_pos, __uint_as_float(o.flags));
    n_job += tot & 0xFFFFu;
  }
  tc.sync();
  if constexpr (OVF) {
    if (s_table_full) return false;   // every thread reads it after the barrier
  }

  // ---- 1b: smearing jobs (S2, S3, S4) in particle order.  The last chunk's
  // tracks stay in registers (lt_*) and add to the cones once every candidate
  // is staged, after the barrier below; earlier chunks' tracks (events with
  // more jobs than the team has threads) do so in 2, from their records.
  uint32_t trk_reg0 = 0;   // first track of the last chunk
  float4 lt_obj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  bool lt_has = false;
  for (uint32_t j0 = 0; j0 < n_job; j0 += TEAM) {
    const uint32_t j = j0 + (uint32_t)tc.tid;
    JobOut r;
    r.tracked = false; r.cand = false;
    uint32_t i = 0;
    if (j < n_job) {
      const uint32_t job = T.jobs()[PDR_BT(j, T.nmax)];
      i = job & 0xFFFFu;
      run_job(S, K, a, job, event, r);
      if (r.tracked) {
        const uint32_t pi = T.pinfo()[PDR_BT(i, T.nmax)];
        if (pi != PDR_EMPTY) fp_add(&T.etrk()[PDR_BT(pi & 0xFFFFu, T.nslots)], to_fp(r.etrk));
      }
      if (dbg && (r.tracked || r.cand))
        reinterpret_cast<uint32_t*>(S.debug + PDR_B(S, a + i))[3] |=
            (r.tracked ? PDR_F_TRACKED : 0u) | (r.cand ? PDR_F_CAND : 0u);
    }
    uint32_t tot;
    const uint32_t pre = team_scan2<TEAM>(r.tracked, r.cand, tt.wbuf + 32 * flip, tot, tc);
    flip ^= 1u;
    trk_reg0 = n_trk;
    lt_has = false;
    if (r.tracked || r.cand) {
      const float eta = __ldg(S.eta + PDR_B(S, a + i)), phi = __ldg(S.phi + PDR_B(S, a + i));
      if (r.tracked) {
        reinterpret_cast<float4*>(S.tracks)[PDR_B(S, a + n_trk + (pre & 0xFFFFu))] =
            make_float4(r.ptp, eta, phi, __uint_as_float(i));
        if constexpr (IP) {  // the track's impact parameters, parallel to its record
          const uint64_t g = PDR_B(S, a + i);
          const float x0 = S.vx ? __ldg(S.vx + g) : 0.0f, y0 = S.vy ? __ldg(S.vy + g) : 0.0f;
          const float zv = S.vz ? __ldg(S.vz + g) : 0.0f;
          S.ip[PDR_B(S, a + n_trk + (pre & 0xFFFFu))] =
              track_ip_of(__ldg(S.pt + g), eta, phi, (int)__ldg(S.charge + g), x0, y0, zv, i, event, S.rk, S.ipc);
        }
        lt_has = r.ptp > K.iso_ptmin;
        lt_obj = make_float4(eta, phi, r.ptp, __uint_as_float(i | PDR_ISO_TRACK));
      }
      if (r.cand) {
        const uint32_t jc = n_cand + (pre >> 16);
        const uint32_t pi = T.pinfo()[PDR_BT(i, T.nmax)];
        const uint32_t key = pi == PDR_EMPTY ? PDR_NO_KEY : T.keys()[PDR_BT(pi & 0xFFFFu, T.nslots)];
        reinterpret_cast<float4*>(S.cands)[PDR_B(S, a + jc)] =
            make_float4(r.cpt, eta, phi, __uint_as_float(i | ((uint32_t)r.cc << 28)));
        // own tower key, read back by the isolation of candidates beyond the staged ones
        reinterpret_cast<float2*>(S.iso)[PDR_B(S, a + jc)] = make_float2(__uint_as_float(key), 0.0f);
        if (jc < PDR_CMAX) {  // staged for the isolation
          tt.cf[jc] = make_float4(eta, phi, r.cpt, __uint_as_float(i));
          tt.ckey[jc] = key;
          tt.cinfo[jc] = i | ((uint32_t)r.cc << 28);
          const int b = iso_bin(K, eta);
          const uint32_t bit = 1u << jc;
          if (b > 0) atomicOr(&tt.binmask[b - 1], bit);
          atomicOr(&tt.binmask[b], bit);
          if (b + 1 < K.iso_nbin) atomicOr(&tt.binmask[b + 1], bit);
        }
      }
    }
    n_trk += tot & 0xFFFFu;
    n_cand += tot >> 16;
  }
  tc.sync();
  const uint32_t gn0 = min(n_cand, (uint32_t)PDR_CMAX);
  if (lt_has && gn0 > 0) iso_object(K, lt_obj, tt);
  // ---- 2: towers (S6, S7), each by its lowest-index depositing particle;
  // EFlow neutrals and the earlier chunks' tracks add their pT to the staged
  // candidates' cones (S8)
  uint32_t n_twr = 0, n_ef = 0;
  for (uint32_t c0 = 0; c0 < n; c0 += TEAM) {
    const uint32_t i = c0 + (uint32_t)tc.tid;
    TowerOut to;
    to.kept = false; to.ef = false;
    uint32_t key = PDR_NO_KEY;
    if (i < n) {
      const uint32_t pi = T.pinfo()[PDR_BT(i, T.nmax)];
      if (pi != PDR_EMPTY) {
        const uint32_t slot = PDR_BT(pi & 0xFFFFu, T.nslots);
        if (T.owner()[slot] == i) {
          key = T.keys()[slot];
          tower_stage(K, KD, key, pi >> 16, T.esum()[slot], T.etrk()[slot], event, S.rk, to);
          T.keys()[slot] = PDR_EMPTY;  // leave the table empty for the next event
          if (to.ef && gn0 > 0 && to.det > K.iso_ptmin) {
            const int calo = (int)(key >> 24), ring = (int)(pi >> 16);
            const float oe = ring_rec(K, KD, calo, ring).x;
            if (tt.binmask[iso_bin(K, oe)] != 0u)  // else no staged candidate is near in eta
              iso_object(K, make_float4(oe, tower_phi_c(K, KD, calo, key & 0xFFFFFFu, ring), to.det,
                                        __uint_as_float(key)), tt);
          }
        }
      }
    }
    if (gn0 > 0 && i < trk_reg0) {
      const float4 t = reinterpret_cast<const float4*>(S.tracks)[PDR_B(S, a + i)];
      if (t.x > K.iso_ptmin)
        iso_object(K, make_float4(t.y, t.z, t.x, __uint_as_float(__float_as_uint(t.w) | PDR_ISO_TRACK)), tt);
    }
    uint32_t tot;
    const uint32_t pre = team_scan2<TEAM>(to.kept, to.ef, tt.wbuf + 32 * flip, tot, tc);
    flip ^= 1u;
    if (to.kept) {
      pdr_tower* r = S.towers + PDR_B(S, a + n_twr + (pre & 0xFFFFu));
      r->key = key; r->e = to.e; r->et = to.et;
    }
    if (to.ef) {
      pdr_eflow* r = S.eflow + PDR_B(S, a + n_ef + (pre >> 16));
      r->key = key; r->e = to.de; r->et = to.det;
    }
    n_twr += tot & 0xFFFFu;
    n_ef += tot >> 16;
  }

  // ---- 3: isolation results (S8).  The staged candidates received every
  // object's pT during 2 (its last team scan orders those sums before this
  // read); further groups of PDR_CMAX candidates loop over all EFlow objects.
  if (gn0 > 0) {
    for (uint32_t k = tc.tid; k < PDR_ISO_BINS; k += TEAM) tt.binmask[k] = 0u;  // read only during 2
    if ((uint32_t)tc.tid < gn0) {
      const uint32_t c = tc.tid;
      const float s = from_fp(tt.csum[c]);
      tt.csum[c] = 0ull;  // clean for the next group / event
      const float rel = s / tt.cf[c].z;
      reinterpret_cast<float2*>(S.iso)[PDR_B(S, a + c)] = make_float2(s, rel);
      reinterpret_cast<uint32_t*>(S.cands + PDR_B(S, a + c))[3] = tt.cinfo[c] | (rel < K.imax ? 0x80000000u : 0u);
    }
  }
  for (uint32_t g0 = PDR_CMAX; g0 < n_cand; g0 += PDR_CMAX) {
    const uint32_t gn = min((uint32_t)PDR_CMAX, n_cand - g0);
    const uint32_t n_obj = n_trk + n_ef;
    tc.sync();
    if ((uint32_t)tc.tid < gn) {  // candidates beyond the staged ones
      const uint64_t j = PDR_B(S, a + g0 + tc.tid);
      const float4 c = reinterpret_cast<const float4*>(S.cands)[j];
      tt.cf[tc.tid] = make_float4(c.y, c.z, c.x, __uint_as_float(__float_as_uint(c.w) & 0x0FFFFFFFu));
      tt.ckey[tc.tid] = __float_as_uint(reinterpret_cast<const float2*>(S.iso)[j].x);
      tt.cinfo[tc.tid] = __float_as_uint(c.w);
    }
    tc.sync();
    for (uint32_t j = tc.tid; j < n_obj; j += TEAM) {
      float oe, op, opt;
      uint32_t oid;
      bool is_trk;
      if (j < n_trk) {
        const float4 t = reinterpret_cast<const float4*>(S.tracks)[PDR_B(S, a + j)];
        opt = t.x; oe = t.y; op = t.z; oid = __float_as_uint(t.w); is_trk = true;
      } else {
        const pdr_eflow f = S.eflow[PDR_B(S, a + (j - n_trk))];
        int r;
        tower_decode(K, KD, (int)(f.key >> 24), f.key & 0xFFFFFFu, r, oe, op);
        opt = f.et; oid = f.key; is_trk = false;
      }
      if (!(opt > K.iso_ptmin)) continue;
      const unsigned long long wgt = to_fp(opt);
      for (uint32_t c = 0; c < gn; ++c) {
        const float4 cv = tt.cf[c];
        if (is_trk ? (oid == __float_as_uint(cv.w)) : (oid == tt.ckey[c])) continue;
        const float de = oe - cv.x;
        float dp = op - cv.y;
        if (dp >= PI_F) dp -= TWO_PI_F;
        else if (dp < -PI_F) dp += TWO_PI_F;
        const float dr2 = fmaf(de, de, dp * dp);
        if (dr2 < K.dr2max && dr2 >= K.dr2min) fp_add(&tt.csum[c], wgt);
      }
    }
    tc.sync();
    if ((uint32_t)tc.tid < gn) {
      const uint64_t j = PDR_B(S, a + g0 + tc.tid);
      const float s = from_fp(tt.csum[tc.tid]);
      tt.csum[tc.tid] = 0ull;
      const float rel = s / tt.cf[tc.tid].z;
      reinterpret_cast<float2*>(S.iso)[j] = make_float2(s, rel);
      reinterpret_cast<uint32_t*>(S.cands + j)[3] = tt.cinfo[tc.tid] | (rel < K.imax ? 0x80000000u : 0u);
    }
  }
  // the next event reuses the table, the staged candidates and the buffers
  tc.sync();
  if (tc.tid == 0)
    reinterpret_cast<uint4*>(S.counts)[PDR_BE(S, e)] = make_uint4(n_trk, n_twr, n_ef, n_cand);
  return true;
}

// The event on a global-memory table (events beyond the shared table, or
// the redo of an overflow): rare, so kept out of line, which keeps the
// kernel's hot code small for the instruction cache.
template <int TEAM, bool IP>
__device__ __noinline__ void process_event_global(const KSeg& S, uint32_t* err, const HotCard& K, const float* KD,
                                                  const Tbl& T, TeamTail& tt, const TeamCtx<TEAM>& tc, uint64_t e,
                                                  uint64_t a, uint32_t n) {
  process_event<TEAM, false, IP>(S, err, K, KD, T, tt, tc, e, a, n);
}

// The persistent event loop of one team.  ONE: the launch holds a single
// batch, whose fields the compiler then reads straight from the parameter
// block (no per-event segment lookup).
template <int TEAM, int BLOCK, bool ONE, bool OVF, bool IP>
__device__ __forceinline__ void event_loop(const KParams& p, unsigned char* smem, const TeamCtx<TEAM>& tc,
                                           const Tbl& st, TeamTail& tt) {
  constexpr int NT = BLOCK / TEAM;
  const uint64_t gteam = (uint64_t)blockIdx.x * NT + tc.tix;
  const uint64_t nteams = (uint64_t)gridDim.x * NT;
  uint32_t sg = 0;  // segment cursor: a team's events only move forward
  // A team's first event is its own index; with a work counter the later ones
  // are handed out as teams become free (event times vary, so a fixed
  // round-robin leaves a tail of teams with the slowest events).  The team's
  // next index is fetched when an event starts and passed to the team in a
  // double-buffered shared word: every event has a team barrier after the
  // write and before the reads, and one between the reads and the write two
  // events later.
  uint32_t turn = 0;
  for (uint64_t ge = gteam; ge < p.n_events; ge = p.work ? (uint64_t)tt.next[(turn++) & 1u] : ge + nteams) {
    if (p.work && tc.tid == 0) tt.next[turn & 1u] = (uint32_t)nteams + atomicAdd(p.work, 1u);
    if (!ONE)
      while (sg + 1 < p.n_segs && ge >= p.seg[sg + 1].event_start) ++sg;
    const KSeg& S = p.seg[ONE ? 0 : sg];
    const uint64_t e = ge - S.event_start;
    const HotCard& K = *reinterpret_cast<const HotCard*>(smem + p.hot_off[S.card]);
    const float* KD = reinterpret_cast<const float*>(smem + p.hot_off[S.card] + sizeof(HotCard));
    const uint64_t a = S.offsets[e], b = S.offsets[e + 1];
    if (!csr_ok(a, b, S.offsets[S.n_events]) || b - a >= (1ull << 28)) {
      if (tc.tid == 0) {
        atomicOr(p.err, ERR_CSR);
        reinterpret_cast<uint4*>(S.counts)[PDR_BE(S, e)] = make_uint4(0, 0, 0, 0);
      }
      if (p.work) tc.sync();
      continue;
    }
    const uint32_t n = (uint32_t)(b - a);
    if (n == 0) {  // nothing to do (a team barrier only for the work counter's hand-over)
      if (tc.tid == 0) reinterpret_cast<uint4*>(S.counts)[PDR_BE(S, e)] = make_uint4(0, 0, 0, 0);
      if (p.work) tc.sync();
      continue;
    }
    if (n <= p.nmax_smem) {
      if constexpr (!OVF) {
        process_event<TEAM, false, IP>(S, p.err, K, KD, st, tt, tc, e, a, n);
        continue;
      } else {
        if (process_event<TEAM, true, IP>(S, p.err, K, KD, st, tt, tc, e, a, n)) continue;
        // the shared table (sized below the particle count) filled up: reset
        // the flag, empty the table and redo the event with the global table
        tc.sync();
        if (tc.tid == 0) s_table_full = 0u;
        for (uint32_t s = tc.tid; s < p.table_slots; s += TEAM) st.keys()[s] = PDR_EMPTY;
        tc.sync();
      }
    }
    if (p.gscratch != nullptr && n <= p.g_nmax) {
      const Tbl gt = carve(p.gscratch + gteam * p.g_team_bytes, p.g_slots, p.g_nmax);
      for (uint32_t s = tc.tid; s < p.g_slots; s += TEAM) gt.keys()[s] = PDR_EMPTY;
      tc.sync();
      process_event_global<TEAM, IP>(S, p.err, K, KD, gt, tt, tc, e, a, n);
    } else {
      if (tc.tid == 0) {
        atomicOr(p.err, ERR_OVERSIZE);
        reinterpret_cast<uint4*>(S.counts)[PDR_BE(S, e)] = make_uint4(0, 0, 0, 0);
      }
      if (p.work) tc.sync();
    }
  }
#ifdef PDR_BOUNDS
  if (tc.tid == 0 && *(volatile uint32_t*)&g_bounds_flag) atomicOr(p.err, ERR_BOUNDS);
#endif
  // the launch's last team to finish resets the counter for the next launch
  // on this stream (every team's last fetch precedes its count of finished
  // teams)
  if (p.work && tc.tid == 0) {
    __threadfence();
    if (atomicAdd(p.work + 1, 1u) == (uint32_t)nteams - 1u) {
      atomicExch(p.work, 0u);
      atomicExch(p.work + 1, 0u);
    }
  }
}

// ------------------------------------------------------------------ kernel
// Shared memory: the card images of the launch (hot_total), then per team its
// tower table, particle info, scan buffers and isolation candidates.
// Register cap: at most 64 registers a thread (1024 / BLOCK resident CTAs).
// The launch covers up to PDR_LAUNCH_SEGS batches (each with its own card,
// inputs, outputs and seed) as one launch-wide sequence of events.
// IP: also the impact parameters of every accepted track (pdr_run_ip).
template <int TEAM, int BLOCK, bool OVF, bool IP>
__global__ void __launch_bounds__(BLOCK, (1024 / BLOCK) > 0 ? (1024 / BLOCK) : 1)
    fused_kernel(const __grid_constant__ KParams p) {
  static_assert(!OVF || TEAM == BLOCK, "the table-full flag is one per block");
  extern __shared__ __align__(16) unsigned char smem[];
  for (uint32_t c = 0; c < p.n_cards; ++c)
    for (uint32_t k = threadIdx.x; k < p.hot_bytes[c] / 16; k += BLOCK)
      reinterpret_cast<uint4*>(smem + p.hot_off[c])[k] = __ldg(reinterpret_cast<const uint4*>(p.hot[c]) + k);
  TeamCtx<TEAM> tc;
  tc.tix = (int)threadIdx.x / TEAM;
  tc.tid = (int)threadIdx.x % TEAM;
  const uint64_t tbytes = team_smem_bytes(TEAM, p.table_slots, p.nmax_smem);
  unsigned char* mine = smem + p.hot_total + (uint64_t)tc.tix * tbytes;
  const Tbl st = carve(mine, p.table_slots, p.nmax_smem);
  unsigned char* tail = mine + table_bytes(p.table_slots, p.nmax_smem);
  TeamTail& tt = *reinterpret_cast<TeamTail*>(tail);
  for (uint32_t s = tc.tid; s < p.table_slots; s += TEAM) st.keys()[s] = PDR_EMPTY;
  if ((uint32_t)tc.tid < PDR_CMAX) tt.csum[tc.tid] = 0ull;
  for (uint32_t k = tc.tid; k < PDR_ISO_BINS; k += TEAM) tt.binmask[k] = 0u;
  if constexpr (OVF) {
    if (tc.tid == 0) s_table_full = 0u;
  }
  __syncthreads();
  if (p.n_segs == 1) event_loop<TEAM, BLOCK, true, OVF, IP>(p, smem, tc, st, tt);
  else event_loop<TEAM, BLOCK, false, OVF, IP>(p, smem, tc, st, tt);
}

// ------------------------------------------------------- auxiliary kernels
__global__ void max_event_kernel(const uint64_t* __restrict__ offsets, uint64_t n_events,
                                 uint32_t* out, uint32_t* err) {
  uint32_t m = 0;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n_events;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = offsets[e], b = offsets[e + 1];
    if (!csr_ok(a, b, offsets[n_events])) atomicOr(err, ERR_CSR);
    else m = max(m, (uint32_t)min(b - a, (uint64_t)0xFFFFFFFFu));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(PDR_FULL, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Dense compaction for host delivery, one chunk of events at a time: an
// exclusive scan of the chunk's per-event counts per collection, continuing
// from the running totals in carry[4] (single block per collection, chunked),
// then a gather into the dense arrays.  dense_off holds the four collections'
// offsets with a stride of `stride` entries.
__global__ void scan_counts_kernel(const uint32_t* __restrict__ counts, uint64_t n_events,
                                   uint64_t* __restrict__ dense_off, uint64_t stride,
                                   unsigned long long* __restrict__ carry) {
  const int c = blockIdx.x;  // collection
  __shared__ unsigned long long part[1024];
  uint64_t* out = dense_off + (uint64_t)c * stride;
  unsigned long long run = carry[c];
  for (uint64_t base = 0; base < n_events; base += blockDim.x) {
    const uint64_t e = base + threadIdx.x;
    const unsigned long long v = e < n_events ? counts[4 * e + c] : 0ull;
    part[threadIdx.x] = v;
    __syncthreads();
    for (unsigned o = 1; o < blockDim.x; o <<= 1) {
      const unsigned long long u = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
      __syncthreads();
      part[threadIdx.x] += u;
      __syncthreads();
    }
    if (e < n_events) out[e] = run + part[threadIdx.x] - v;
    const unsigned long long blk = part[blockDim.x - 1];
    __syncthreads();
    run += blk;
  }
  if (threadIdx.x == 0) {
    out[n_events] = run;
    carry[c] = run;
  }
}

__global__ void gather_dense_kernel(const uint64_t* __restrict__ offsets, uint64_t n_events,
                                    const uint32_t* __restrict__ counts,
                                    const uint64_t* __restrict__ dense_off, uint64_t stride, pdr_outputs src,
                                    pdr_outputs dst) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t e = warp; e < n_events; e += nwarps) {
    const uint64_t a = offsets[e];
    const uint32_t nt = counts[4 * e], nw = counts[4 * e + 1], nf = counts[4 * e + 2], nc = counts[4 * e + 3];
    const uint64_t dt = dense_off[e], dw = dense_off[stride + e];
    const uint64_t df = dense_off[2 * stride + e], dc = dense_off[3 * stride + e];
    for (uint32_t k = lane; k < nt; k += 32) dst.tracks[dt + k] = src.tracks[a + k];
    for (uint32_t k = lane; k < nw; k += 32) dst.towers[dw + k] = src.towers[a + k];
    for (uint32_t k = lane; k < nf; k += 32) dst.eflow[df + k] = src.eflow[a + k];
    for (uint32_t k = lane; k < nc; k += 32) {
      dst.cands[dc + k] = src.cands[a + k];
      dst.iso[dc + k] = src.iso[a + k];
    }
  }
}

// ------------------------------------------------------- launch helpers
// A kernel's dynamic shared-memory limit only ever grows (per device): a
// captured graph replays its launch with the shared memory it was captured
// with, which a later smaller launch must not take away.
template <int TEAM, int BLOCK, bool OVF, bool IP>
static cudaError_t allow_smem(size_t smem) {
  static std::mutex mu;
  static int allowed[PDR_MAX_DEVICES] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= PDR_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if ((int)smem <= allowed[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(fused_kernel<TEAM, BLOCK, OVF, IP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) allowed[dev] = (int)smem;
  return e;
}

template <int TEAM, int BLOCK, bool OVF, bool IP>
static cudaError_t launch_t(const KParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
  cudaError_t e = allow_smem<TEAM, BLOCK, OVF, IP>(smem);
  if (e != cudaSuccess) return e;
  fused_kernel<TEAM, BLOCK, OVF, IP><<<grid, BLOCK, smem, s>>>(p);
  return cudaGetLastError();
}

template <int TEAM, int BLOCK, bool OVF>
static cudaError_t occupancy_t(int* blocks, size_t smem) {
  cudaError_t e = allow_smem<TEAM, BLOCK, OVF, false>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fused_kernel<TEAM, BLOCK, OVF, false>, BLOCK, smem);
}

#define PDR_SHAPES(X) X(32, 128) X(32, 256) X(64, 256) X(128, 128) X(128, 256) X(256, 256) X(512, 512) X(1024, 1024)
// shapes also built with a shared table sized below the particle count (large events)
#define PDR_OVF_SHAPES(X) X(512, 512) X(1024, 1024)

bool shape_supported(uint32_t team, uint32_t block) {
#define PDR_SUP(T, B) if (team == T && block == B) return true;
  PDR_SHAPES(PDR_SUP)
#undef PDR_SUP
  return false;
}

bool shape_supports_overflow(uint32_t team, uint32_t block) {
#define PDR_SUP(T, B) if (team == T && block == B) return true;
  PDR_OVF_SHAPES(PDR_SUP)
#undef PDR_SUP
  return false;
}

// ip: the kernel that also writes the tracks' impact parameters (the
// parameter block's segments carry the ip arrays); its occupancy is taken
// to be the plain kernel's (same shared memory, same register cap).
cudaError_t launch_fused(uint32_t team, uint32_t block, const KParams& p, uint32_t grid, size_t smem,
                         cudaStream_t s, bool ip) {
  if (p.smem_may_overflow) {
#define PDR_LO(T, B) if (team == T && block == B) return ip ? launch_t<T, B, true, true>(p, grid, smem, s) \
                                                                : launch_t<T, B, true, false>(p, grid, smem, s);
    PDR_OVF_SHAPES(PDR_LO)
#undef PDR_LO
    return cudaErrorInvalidValue;
  }
#define PDR_L(T, B) if (team == T && block == B) return ip ? launch_t<T, B, false, true>(p, grid, smem, s) \
                                                           : launch_t<T, B, false, false>(p, grid, smem, s);
  PDR_SHAPES(PDR_L)
#undef PDR_L
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_fused_ovf(uint32_t team, uint32_t block, size_t smem, int* blocks) {
#define PDR_OO(T, B) if (team == T && block == B) return occupancy_t<T, B, true>(blocks, smem);
  PDR_OVF_SHAPES(PDR_OO)
#undef PDR_OO
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_fused(uint32_t team, uint32_t block, size_t smem, int* blocks) {
#define PDR_O(T, B) if (team == T && block == B) return occupancy_t<T, B, false>(blocks, smem);
  PDR_SHAPES(PDR_O)
#undef PDR_O
  return cudaErrorInvalidValue;
}

cudaError_t launch_max_event(const uint64_t* offsets, uint64_t n_events, uint32_t* out, uint32_t* err,
                             cudaStream_t s) {
  const uint64_t blocks = n_events / 256 + 1;
  max_event_kernel<<<(unsigned)(blocks < 1184 ? blocks : 1184), 256, 0, s>>>(offsets, n_events, out, err);
  return cudaGetLastError();
}

cudaError_t launch_dense(const uint64_t* offsets, uint64_t n_events, const uint32_t* counts,
                         uint64_t* dense_off, uint64_t stride, unsigned long long* carry,
                         const pdr_outputs& src, const pdr_outputs& dst, int n_sms, cudaStream_t s) {
  scan_counts_kernel<<<4, 1024, 0, s>>>(counts, n_events, dense_off, stride, carry);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gather_dense_kernel<<<n_sms * 8, 256, 0, s>>>(offsets, n_events, counts, dense_off, stride, src, dst);
  return cudaGetLastError();
}

}  // namespace pdr
