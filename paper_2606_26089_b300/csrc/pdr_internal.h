// Internal layouts of the CUDA library: the expanded device card and the
// kernel parameter block.  Shared by the kernels and the host runtime of the
// library only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pdr.h"

#define PDR_MAXRING 512      // eta rings per calorimeter (both sides)
#define PDR_MAXPHI 1024      // phi bins per ring
#define PDR_PHIPOOL (2 * PDR_MAXSEG * (2 * PDR_MAXPHI + 1))
#define PDR_FP_SCALE 68719476736.0f   // 2^36: fixed-point quantum of energy sums (GeV)
#define PDR_FP_INV 1.4551915228366852e-11f  // 2^-36
#define PDR_MAXQ 8           // |charge| handled by the precomputed reach constants
#define PDR_CMAX 32          // isolation candidates held in shared memory at once
#define PDR_EMPTY 0xFFFFFFFFu

#ifdef __CUDACC__
#define PDR_HD __host__ __device__
#else
#define PDR_HD
#endif

namespace pdr {

enum { CLS_E = 0, CLS_MU = 1, CLS_GAMMA = 2, CLS_CHAD = 3, CLS_NHAD = 4, CLS_INVIS = 5 };
enum { RES_TRACK = 0, RES_MUON = 1, RES_ECAL = 2, RES_HCAL = 3 };

// One calorimeter's tower grid, float32 where a decision is taken on it.
struct DevCalo {
  int32_t nring, ntowers, nseg, pad;
  float seg_lo[PDR_MAXSEG], seg_hi[PDR_MAXSEG], seg_scale[PDR_MAXSEG];  // |eta| segments (guess only)
  int32_t seg_n[PDR_MAXSEG], seg_first[PDR_MAXSEG];
  float edge[PDR_MAXRING + 1];   // signed ring edges, float32 (decisions)
  int32_t base[PDR_MAXRING];     // first tower id of each ring
  int32_t nphi[PDR_MAXRING];
  int32_t phioff[PDR_MAXRING];   // offset of the ring's phi table in DevCard::phi_pool
  float phi_scale[PDR_MAXRING];  // nphi / (2 pi), guess only
  float eta_c[PDR_MAXRING];      // ring centre (float32 of the double midpoint)
  float inv_cosh_c[PDR_MAXRING]; // 1 / cosh(eta_c) (float32 of the double value)
  int32_t resbin[PDR_MAXRING];   // resolution row of |eta_c|
  // ring groups: runs of rings with the same phi segmentation, in ring order
  // (tower id -> ring without a search: ring = first + (id - base) / nphi)
  int32_t ngroup, pad2[3];
  int32_t grp_first[2 * PDR_MAXSEG], grp_base[2 * PDR_MAXSEG], grp_nphi[2 * PDR_MAXSEG];
};

struct DevCard {
  DevCalo calo[2];
  // phi tables: for each distinct ring layout, nphi + 1 edges then nphi centres
  float phi_pool[PDR_PHIPOOL];
  // propagation
  float R, L;                    // float32 of the card values
  float L_lo;                    // L - float32(L)
  float kB, kB_lo;               // 0.299792458 |B|, split hi + lo
  int32_t Bsign, has_field, pad0;
  float cR_hi[PDR_MAXQ + 1], cR_lo[PDR_MAXQ + 1];  // c = 0.299792458 |q| |B| R, split hi + lo
  // tracking efficiency: pass iff (u64) w < T
  // small piecewise-constant tables: edges padded with +inf to PDR_MAXEDGE,
  // 16-byte aligned so a lookup is two vector loads
  int32_t trk_npt, trk_neta;
  alignas(16) float trk_pt_edges[PDR_MAXEDGE];
  alignas(16) float trk_eta_edges[PDR_MAXEDGE];
  unsigned long long trk_T[3][PDR_MAXEDGE][PDR_MAXEDGE];
  // resolutions, squared coefficients
  int32_t res_n[4];
  alignas(16) float res_edges[4][PDR_MAXEDGE];
  float res_a2[4][PDR_MAXEDGE], res_b2[4][PDR_MAXEDGE], res_c2[4][PDR_MAXEDGE], res_d2[4][PDR_MAXEDGE];
  // identification efficiency
  int32_t id_n, pad1;
  alignas(16) float id_edges[PDR_MAXEDGE];
  unsigned long long id_T[3][PDR_MAXEDGE];
  // thresholds and isolation (float32 of the card values; dr2 = float32(dr * dr))
  float e_min[2], s_min[2];
  float cand_ptmin, dr2max, dr2min, iso_ptmin, imax, pad2;
};

// The part of a card the kernel touches per particle and per tower, laid out
// compactly so each persistent CTA copies it once into shared memory.  A fixed
// header (below) is followed by `data_floats` floats: per calorimeter the ring
// edges (nring + 1), per eta segment its phi table (nphi + 1 edges, then nphi
// centres), and a 16-byte record per ring (eta_c, 1 / cosh(eta_c), first tower
// id, phi-table offset | nphi << 16 | resolution row << 27), so one vector
// load gives a ring's tower numbering, phi binning and smearing row.
struct HotSeg {
  float lo, hi, scale;      // |eta| range of the segment, n / (hi - lo) (guess only)
  int32_t n, first;         // rings in the segment; first ring counting from eta = 0
  int32_t nphi;
  int32_t base_pos, base_neg;  // tower id of the segment's lowest-index ring on each side
  int32_t phioff;           // offset (floats) of the phi table in the data part
  float phi_scale;          // nphi / (2 pi), guess only
  int32_t pad[2];
};

struct HotCalo {
  int32_t nring, m, nseg, edge_off;  // m = nring / 2; edge_off: offset of the ring edges
  int32_t ring_off, pad[3];          // offset of the per-ring records (4 words a ring, 16-byte aligned)
  HotSeg seg[PDR_MAXSEG];
};

struct alignas(16) HotCard {
  HotCalo calo[2];
  float R, L, kB, L_lo, kB_lo;    // L and 0.299792458 |B| as float32, and their float32 remainders
  int32_t Bsign, has_field, trk_npt, trk_neta, id_n;
  int32_t res_n[4];
  alignas(16) float trk_pt_edges[PDR_MAXEDGE];
  alignas(16) float trk_eta_edges[PDR_MAXEDGE];
  alignas(16) float id_edges[PDR_MAXEDGE];
  alignas(16) float res_edges[4][PDR_MAXEDGE];
  float4 res[4][PDR_MAXEDGE];       // (a^2, b^2, c^2, d^2) per resolution component and |eta| row
  float cR_hi[PDR_MAXQ + 1], cR_lo[PDR_MAXQ + 1];
  unsigned long long trk_T[3][PDR_MAXEDGE][PDR_MAXEDGE];
  unsigned long long id_T[3][PDR_MAXEDGE];
  float e_min[2], s_min[2];
  float cand_ptmin, dr2max, dr2min, iso_ptmin, imax;
  // isolation pre-selection: eta bins of width w >= 1.001 dR over [-8, 8]
  // (eta outside clamps to the end bins), so an object within the cone of a
  // candidate lies in the candidate's bin or a neighbouring one
  float iso_inv_w;
  int32_t iso_nbin;
  int32_t data_floats;
};

#define PDR_HOT_MAX_BYTES (40u * 1024u)   // shared-memory card cache limit

#define PDR_MAX_DEVICES 64   // device ordinals the library tracks per-device state for
#define PDR_LAUNCH_SEGS 32   // batches in one fused launch
#define PDR_LAUNCH_CARDS 4   // distinct cards in one fused launch

// Field and resolutions of the impact-parameter smearing.
struct IPConst {
  float kB;                          // 0.299792458 |B|
  int32_t bsign, has_field;
  float a_d0, b_d0, a_z0, b_z0;      // sigma = sqrt(a^2 + (b / pT)^2)
};

// One batch of a launch: its inputs, outputs, randomness and card.
struct KSeg {
  uint64_t event_start;              // first launch-wide event index of the batch
  uint64_t n_events;
  const uint64_t* offsets;
  const float *pt, *eta, *phi, *mass, *vz;
  const int32_t* pdg;
  const int8_t* charge;
  uint32_t seed_lo, seed_hi, event_base, card;  // card: slot of KParams::hot
  uint32_t rk[20];                   // Philox round keys of the seed: (k0, k1) of rounds 0..9
  pdr_track* tracks;
  pdr_tower* towers;
  pdr_eflow* eflow;
  pdr_cand* cands;
  pdr_iso* iso;
  uint32_t* counts;
  pdr_debug* debug;                  // null: no debug records
  // impact parameters of the tracks (kernels built for them only)
  pdr_ip* ip;
  const float *vx, *vy;              // transverse production vertex, or null (0)
  IPConst ipc;
};

// Philox4x32-10 round keys of a 64-bit seed: round r uses key (lo + r W0,
// hi + r W1) with the Weyl constants W0 = 0x9E3779B9, W1 = 0xBB67AE85.
PDR_HD inline void fill_round_keys(uint32_t* rk, uint64_t seed) {
  uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0;
    rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

PDR_HD inline void set_round_keys(KSeg& g, uint64_t seed) {
  g.seed_lo = (uint32_t)(seed & 0xFFFFFFFFu);
  g.seed_hi = (uint32_t)(seed >> 32);
  fill_round_keys(g.rk, seed);
}

// Pile-up merging: the hard batch, the minimum-bias pool, the Poisson
// thresholds, the vertex parameters and the outputs of both passes.
struct PuParams {
  uint64_t n_events, n_pool;
  const uint64_t* hoff;
  const float *hpt, *heta, *hphi, *hmass, *hvz;
  const int32_t* hpdg;
  const int8_t* hcharge;
  const uint64_t* poff;
  const float *ppt, *peta, *pphi, *pmass;
  const int32_t* ppdg;
  const int8_t* pcharge;
  const unsigned long long* T;       // Poisson CDF thresholds, K entries, T[K-1] = 2^32
  uint32_t K, event_base, smear_hs, pad;
  float sigma_z, max_z, sigma_t, max_t;
  uint32_t rk[20];
  uint64_t* counts;                  // first pass: merged size of each event
  const uint64_t* moff;              // second pass: merged offsets
  float *opt, *oeta, *ophi, *omass, *ovz, *ovt;  // ovt may be null
  int32_t* opdg;
  int8_t* ocharge;
  uint32_t* err;
};

// Post-processing (filter + event features): one condition, thresholds in
// the type the field is compared in.
struct PostCond {
  uint32_t field, op, abs, n;
  float fv[PDR_MAX_VALUES];
  int32_t iv[PDR_MAX_VALUES];
};

struct PostParams {
  uint64_t n_events;
  const uint64_t* offsets;
  const int32_t* pdg;
  const int8_t* charge;
  const float* mass;
  const float2* centres;             // (eta_c, phi_c) of ECAL tower ids, then HCAL ones
  uint32_t ntowers[2];
  pdr_track* tracks;
  pdr_tower* towers;
  pdr_eflow* eflow;
  pdr_cand* cands;
  pdr_iso* iso;
  uint32_t* counts;
  pdr_features* features;            // may be null
  uint32_t* err;
  uint32_t filtered, collection, combine, n_cond, compact, update_features;
  uint32_t need_gen;                 // a condition reads pdg or charge
  uint32_t need_mass;                // a track condition reads e
  PostCond cond[PDR_MAX_CONDITIONS];
};

// Track impact parameters.
struct IPParams {
  uint64_t n_events;
  const uint64_t* offsets;
  const float *pt, *eta, *phi, *vx, *vy, *vz;
  const int8_t* charge;
  const pdr_track* tracks;
  const uint32_t* counts;
  pdr_ip* ip;
  uint32_t* err;
  IPConst c;
  uint32_t event_base;
  uint32_t rk[20];                   // Philox round keys of the batch's seed
};

// Jet clustering.
struct JetParams {
  uint64_t n_events;
  const uint64_t* offsets;
  const float *pt, *eta, *phi, *mass;   // generated particles
  const int32_t* pdg;
  const pdr_track* tracks;              // PFlow
  const pdr_eflow* eflow;
  const uint32_t* counts;
  const float2* centres;
  uint32_t ntowers[2];
  uint32_t collection, nconst_min;
  uint32_t ee;                          // e+e- distances: energies and unit directions
  uint32_t cap;                         // objects per warp workspace (multiple of 32)
  uint32_t min_obj;                     // this launch clusters events with min_obj..cap objects
  uint32_t warps;                       // warps per block
  float p, R2, inv_R2, pt_min;
  int32_t nty, ntp;                     // rapidity x azimuth tiles, each at least R wide
  uint32_t ntiles;                      // nty * ntp
  float y0, inv_wy, inv_wp;
  pdr_jet* jets;
  uint32_t* jet_counts;
  uint32_t* err;
  double* scratch;                      // PDR_JET_SCRATCH_DOUBLES x cap doubles for each warp of the grid
  uint32_t* next_event;                 // work counter (zero at launch): warps take events in turn
};

// Bytes of one warp's shared-memory clustering workspace for `cap` objects
// (a multiple of 32) and `ntiles` tiles: float y, phi, pT^2p and distance,
// and for e+e- a third direction component (y, phi, nz then hold the unit
// direction); short nearest neighbour, tile, next-in-tile and a step's
// re-search list; then the heads of the tile lists and a counter.  (The
// double four-momenta, constituent counts and merge parents, touched once a
// step by one lane, live in global scratch.)
PDR_HD inline uint64_t jet_ws_bytes(uint32_t cap, bool ee, uint32_t ntiles) {
  return (uint64_t)cap * ((ee ? 5 : 4) * 4 + 4 * 2) + 2 * (uint64_t)((ntiles + 7u) & ~7u) + 16;
}
// Global scratch of one warp, in doubles per object: px, py, E + pz, E - pz,
// then float pT, y, phi of each object as loaded, int constituent count and
// short merge parent (50 of the 56 bytes).
constexpr uint32_t PDR_JET_SCRATCH_DOUBLES = 7;

// Kernel parameter block (passed by value, read through __grid_constant__).
struct KParams {
  uint64_t n_events;                 // all segments
  uint32_t n_segs, n_cards;
  const unsigned char* hot[PDR_LAUNCH_CARDS];   // card cache images (device)
  uint32_t hot_bytes[PDR_LAUNCH_CARDS];         // each a multiple of 16
  uint32_t hot_off[PDR_LAUNCH_CARDS];           // offset of each image in shared memory
  uint32_t hot_total;                // shared memory of all card images
  uint32_t table_slots;              // shared-memory table per team (multiple of 32)
  uint32_t nmax_smem;                // largest event handled in shared memory
  uint32_t g_slots, g_nmax;          // global-memory table per team for larger events
  unsigned char* gscratch;           // g_team_bytes per team, or null
  uint64_t g_team_bytes;
  uint32_t* err;                     // device error word (bit flags below)
  KSeg seg[PDR_LAUNCH_SEGS];
  uint32_t smem_may_overflow;        // 1: the shared table is sized below the particle count (an event
                                     // whose towers overflow it is redone with the global table)
  uint32_t* work;                    // (events handed out, teams done), zero at launch and reset by the
                                     // launch's last team; null: a fixed round-robin of events
};

#define PDR_WORK_STREAMS 1024   // streams per context with their own fused-launch work counter

enum : uint32_t {
  ERR_CSR = 1u,        // offsets not monotone
  ERR_OVERSIZE = 2u,   // event larger than any table available to the launch
  ERR_TABLE = 4u,      // tower table full (cannot happen when sized as documented)
  ERR_PILEUP = 8u,     // pile-up merge: an event's size differs from the offsets given
  ERR_VERTEX = 16u,    // pile-up merge: no vertex inside the truncation in 1024 draws
  ERR_JETS = 32u,      // jet clustering: more jets than the event's slots, or an inconsistent cell list
  ERR_BOUNDS = 64u,    // bounds-checking build (PDR_BOUNDS): an index out of its array; the access was skipped
};

// An event's CSR range [a, b) is usable iff a <= b <= end, end = offsets[n_events]
// (the particle and output arrays hold `end` entries).  Checking b < a alone
// is not enough: a non-monotone interior offset past the end gives an earlier
// event a range that reads and writes beyond the arrays.
PDR_HD inline bool csr_ok(uint64_t a, uint64_t b, uint64_t end) { return a <= b && b <= end; }

#define PDR_PART_BYTES 8     // per particle: info word, smearing-job entry
#define PDR_ISO_BINS 64      // eta bins of the isolation pre-selection

// Bytes of a team's event workspace: the tower table (keys, owner, esum, etrk
// per slot), then per particle an info word and a smearing-job entry
// (16-byte multiple).
PDR_HD inline uint64_t table_bytes(uint32_t slots, uint32_t nmax) {
  const uint64_t b = (uint64_t)slots * (4 + 4 + 8 + 8) + (uint64_t)nmax * PDR_PART_BYTES;
  return (b + 15) & ~15ull;
}

// A team's shared scratch after its table: scan buffers (double-buffered),
// the staged isolation candidates (eta, phi, pT', particle index; own tower
// key; record info word; fixed-point cone sums) and their eta-bin masks.
struct TeamTail {
  uint32_t next[4];                  // the team's next events, double-buffered (work counter)
  uint32_t wbuf[2 * 32];
  float4 cf[PDR_CMAX];
  uint32_t ckey[PDR_CMAX];
  uint32_t cinfo[PDR_CMAX];
  unsigned long long csum[PDR_CMAX];
  uint32_t binmask[PDR_ISO_BINS];    // bit c: staged candidate c lies in this eta bin or a neighbour
};

PDR_HD inline uint64_t tail_bytes(uint32_t) { return (sizeof(TeamTail) + 15) & ~15ull; }

// Shared-memory bytes needed by one team of a launch shape (the card cache is
// counted separately, once per CTA).
PDR_HD inline uint64_t team_smem_bytes(uint32_t team, uint32_t slots, uint32_t nmax) {
  return table_bytes(slots, nmax) + tail_bytes(team);
}

PDR_HD inline uint64_t global_team_bytes(uint32_t slots, uint32_t nmax) {
  return (table_bytes(slots, nmax) + 255) & ~255ull;
}

}  // namespace pdr
