/*
 * pdr.h - parametric detector response on one GPU: the C ABI.
 *
 * The library applies a Delphes-style parametric detector response to every
 * truth particle of every event in a batch: the TorchDelphes module chain of
 * the paper (Sec. 2.2 "parametric backend"; App. D.1): particle propagation in
 * the solenoid field, tracking / lepton / photon efficiencies, momentum and
 * energy smearing, ECAL/HCAL eta-phi towers with smearing and thresholds,
 * energy-flow track subtraction (Towers and EFlowObjects), and the cone
 * isolation of electrons, muons and photons (Sec. 2.4, Eq. 1).
 *
 * Everything on the data path runs in the library's CUDA kernels.  All entry
 * points are plain C: pointers, sizes and status codes; no C++ types and no
 * PyTorch types cross this boundary.  Pointers are DEVICE pointers unless an
 * entry point says HOST.  Streams are passed as `void*` holding a
 * `cudaStream_t` (NULL = the legacy default stream).
 *
 * Errors: every entry point returns a pdr_status.  Nothing is thrown across
 * the ABI.  On failure `pdr_last_error(ctx)` gives a message for the calling
 * thread.  A device-side error (an overflowed table, a bounded wait that ran
 * out) is recorded in a device error word that `pdr_check` / `pdr_wait` read.
 *
 * Randomness: counter-based Philox4x32-10 keyed by (seed low, seed high) with
 * counter (slot, event, purpose, 0), where event = event_index_base + e for
 * the e-th event of a batch, slot = the particle's index inside its event
 * (purposes 1 tracking, 2 identification) or the tower id (purposes 3 ECAL,
 * 4 HCAL tower smearing).  A result therefore depends only on the event's
 * particles, the card, the seed and the event's index - not on batching,
 * launch shape or which other events share the batch.
 */
#ifndef PDR_H
#define PDR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDR_ABI_VERSION 1

typedef enum {
  PDR_OK = 0,
  PDR_EINVAL = -1,     /* bad argument (null pointer, malformed CSR, bad size)      */
  PDR_ENOMEM = -2,     /* device or pool memory exhausted                           */
  PDR_ECARD = -3,      /* malformed card (non-monotone edges, efficiency outside [0,1]) */
  PDR_ETIMEDOUT = -4,  /* a bounded wait ran out                                    */
  PDR_EDEVICE = -5,    /* CUDA error, or a device-side error word was set           */
  PDR_EBUSY = -6,      /* too many tickets in flight / serving loop busy            */
  PDR_ENOTFOUND = -7,  /* unknown card id or ticket                                 */
  PDR_EOVERFLOW = -8   /* an event exceeds the size the launch configuration allows */
} pdr_status;

/* ---------------------------------------------------------------- cards -- */
#define PDR_MAXSEG 4   /* eta segments per calorimeter side           */
#define PDR_MAXEDGE 8  /* edges per axis of a piecewise-constant table */

/* Calorimeters and classes (also used in output keys and flags). */
#define PDR_ECAL 0
#define PDR_HCAL 1
#define PDR_CAND_E 0
#define PDR_CAND_MU 1
#define PDR_CAND_GAMMA 2

/*
 * Detector card: raw parameters (GeV, m, T), as the paper's cards give the
 * per-module parameters (App. D.1).  The library expands them into device
 * tables at pdr_card_load; the caller keeps ownership of the struct.
 *
 * Calorimeter grids: each side of eta = 0 is cut into nseg segments; segment
 * s spans [eta_hi[s-1], eta_hi[s]] (eta_hi[-1] = 0) in neta[s] rings of
 * nphi[s] towers.  Ring edges inside a segment are lo + ((hi - lo) * k) / n
 * (double precision), segment ends exact; phi edges are -pi + (2 pi k) / nphi.
 * Tower id = (rings below) + phi bin; tower key = calo << 24 | id.
 * Piecewise-constant tables use bins [edge_k, edge_k+1) with an open last bin.
 */
typedef struct pdr_card {
  double B, R, L;                        /* field (T), calorimeter radius and half-length (m) */
  int32_t nseg[2];
  double seg_eta_hi[2][PDR_MAXSEG];
  int32_t seg_neta[2][PDR_MAXSEG];
  int32_t seg_nphi[2][PDR_MAXSEG];
  int32_t trk_npt, trk_neta;             /* tracking efficiency table axes       */
  double trk_pt_edges[PDR_MAXEDGE];
  double trk_eta_edges[PDR_MAXEDGE];     /* |eta| edges                          */
  double trk_eff[3][PDR_MAXEDGE][PDR_MAXEDGE]; /* [hadron, electron, muon][pT bin][|eta| bin] */
  int32_t res_n[4];                      /* resolution tables: track, muon, ECAL, HCAL */
  double res_edges[4][PDR_MAXEDGE];      /* |eta| edges                          */
  double res_abcd[4][PDR_MAXEDGE][4];    /* sigma/x = sqrt(a^2/x + b^2/x^2 + c^2 + d^2 x^2) */
  int32_t id_n;                          /* identification efficiency table      */
  double id_edges[PDR_MAXEDGE];          /* |eta| edges                          */
  double id_eff[3][PDR_MAXEDGE];         /* [electron, muon, photon][|eta| bin]  */
  double e_min[2], s_min[2];             /* tower / EFlow thresholds: E > e_min, E/sigma > s_min */
  double cand_ptmin;                     /* e/mu/gamma candidates need truth pT > cand_ptmin */
  double iso_dr, iso_drmin, iso_ptmin, iso_imax; /* isolation cone, inner cone, object pT floor, I_max */
} pdr_card;

/* ---------------------------------------------------------- output records -- */
/* All output collections are written per event into slots starting at the
 * event's INPUT offset (offsets[e]); event e's k-th record of a collection is
 * at [offsets[e] + k], and counts[4 e + c] says how many there are (c = 0
 * tracks, 1 towers, 2 EFlow neutrals, 3 candidates).  Every collection has at
 * most as many records as the event has particles, so buffers of n_particles
 * records always suffice.  Records within an event are ordered by particle
 * index (towers and EFlow neutrals: by the lowest index depositing in them). */
typedef struct { float pt, eta, phi; uint32_t idx; } pdr_track;     /* smeared pT, momentum direction, particle index */
typedef struct { uint32_t key; float e, et; } pdr_tower;            /* key = calo << 24 | tower id; E', E'/cosh(eta_c) */
typedef struct { uint32_t key; float e, et; } pdr_eflow;            /* EFlow neutral at the tower centre: dE, dE/cosh(eta_c) */
typedef struct { float pt, eta, phi; uint32_t info; } pdr_cand;     /* info = idx | class << 28 | isolated << 31 */
typedef struct { float sum, rel; } pdr_iso;                         /* cone pT sum and sum / pT */
typedef struct { uint32_t key; float eta_pos, phi_pos; uint32_t flags; } pdr_debug; /* per particle */

#define PDR_CAND_IDX(info) ((info) & 0x0FFFFFFFu)
#define PDR_CAND_CLASS(info) (((info) >> 28) & 0x3u)
#define PDR_CAND_ISOLATED(info) ((info) >> 31)

/* pdr_debug.flags bits */
#define PDR_F_REACH 0x01u    /* reached the calorimeter surface     */
#define PDR_F_BARREL 0x02u   /* hit the barrel (else the endcap)      */
#define PDR_F_TRACKED 0x04u  /* accepted by the tracking efficiency   */
#define PDR_F_CAND 0x08u     /* accepted e/mu/gamma candidate         */
#define PDR_F_ECAL 0x10u     /* deposited in ECAL                     */
#define PDR_F_HCAL 0x20u     /* deposited in HCAL                     */
#define PDR_NO_KEY 0xFFFFFFFFu

/* ---------------------------------------------------------------- batches -- */
/* A ragged CSR batch in SoA layout (DEVICE pointers unless PDR_BATCH_HOST).
 * offsets[n_events + 1] is non-decreasing with offsets[0] = 0; particle
 * arrays hold offsets[n_events] entries; vz may be NULL (all vertices at 0). */
#define PDR_BATCH_DEBUG 0x1u      /* also write pdr_debug records             */
typedef struct pdr_batch {
  uint64_t n_events;
  const uint64_t* offsets;
  const float* pt;            /* GeV                          */
  const float* eta;           /* momentum pseudorapidity      */
  const float* phi;           /* momentum azimuth, [-pi, pi)  */
  const float* mass;          /* GeV                          */
  const int32_t* pdg;         /* PDG id                       */
  const int8_t* charge;       /* units of e                   */
  const float* vz;            /* vertex z (m) or NULL         */
  uint64_t seed;
  uint32_t event_index_base;
  uint32_t card_id;
  uint32_t max_event_size;    /* largest event (particles); 0 = let the library find it */
  uint32_t flags;             /* PDR_BATCH_* */
} pdr_batch;

/* Caller-owned DEVICE output buffers, each with room for offsets[n_events]
 * records (counts: 4 * n_events words; debug may be NULL). */
typedef struct pdr_outputs {
  pdr_track* tracks;
  pdr_tower* towers;
  pdr_eflow* eflow;
  pdr_cand* cands;
  pdr_iso* iso;
  uint32_t* counts;
  pdr_debug* debug;
} pdr_outputs;

/* Launch shape of the fused kernel: `team` threads work on one event (32 =
 * warp per event ... 1024 = block per event), `block` threads per CTA (a
 * multiple of team), `table_slots` shared-memory tower-table slots per team
 * (rounded up to a multiple of 32; events with more than 3/4 x table_slots
 * particles use a global-memory table), `grid` CTAs (0 = fill the GPU,
 * persistent). */
typedef struct pdr_launch {
  uint32_t team, block, table_slots, grid;
} pdr_launch;

/* ---------------------------------------------------------------- context -- */
typedef struct pdr_ctx pdr_ctx;

typedef struct pdr_options {
  uint64_t pool_bytes;    /* device pool for submit() results and scratch (0: 1 GiB) */
  uint32_t max_tickets;   /* outstanding submit() tickets (0: 64)                    */
  uint32_t flags;         /* reserved, 0                                             */
} pdr_options;

/* Create a context on CUDA device `cuda_device` (made current by the call).
 * opt may be NULL.  On success *out owns device memory until pdr_destroy. */
int pdr_create(pdr_ctx** out, int cuda_device, const pdr_options* opt);
/* Destroy a context after synchronising its work.  Frees every card, ticket,
 * graph and pool it owns.  NULL is accepted. */
int pdr_destroy(pdr_ctx* ctx);
/* Thread-local message for the calling thread's last failure in ctx. */
const char* pdr_last_error(pdr_ctx* ctx);
/* Version of this ABI (PDR_ABI_VERSION). */
int pdr_abi_version(void);

/* Validate a card (monotone edges, efficiencies in [0, 1], positive R, L,
 * table sizes in range), expand it and copy the tables to the device.  The
 * struct is HOST memory and stays the caller's.  *card_id names it. */
int pdr_card_load(pdr_ctx* ctx, const pdr_card* card, uint32_t* card_id);
/* Free a card's device tables (after synchronising). */
int pdr_card_unload(pdr_ctx* ctx, uint32_t card_id);
/* Number of towers of a card's calorimeter (PDR_ECAL / PDR_HCAL) via *n. */
int pdr_card_towers(pdr_ctx* ctx, uint32_t card_id, int calo, uint32_t* n);

/* ------------------------------------------------------------ batched path -- */
/* Enqueue the whole detector response for a batch on `stream` (one persistent
 * fused launch), writing into caller-owned device buffers.  Asynchronous: the
 * caller must keep inputs and outputs alive until the stream has finished.
 * launch may be NULL (the context's tuned or default shape is used).  Events
 * larger than the launch's shared-memory table use a global-memory table from
 * the context pool (allocated on first need, outside any stream capture);
 * launches of one context that use it share it, so do not overlap such
 * launches on different streams.
 * Returns PDR_EINVAL for malformed arguments (checked on the host: non-null
 * pointers, n_events < 2^31; the CSR itself is checked on the device and a bad
 * one sets the device error word).  The launch hands events to its teams
 * from a work counter that the context keeps per stream (launches on one
 * stream run in order, and each leaves its counter at zero): a launch
 * captured into a graph keeps the counter of the stream it was captured on,
 * so do not run two replays of it, or a replay and a launch on that stream,
 * at the same time; likewise let a stream's launches finish before
 * destroying it if a new stream might receive the same handle. */
int pdr_run(pdr_ctx* ctx, const pdr_batch* batch, const pdr_outputs* out,
            const pdr_launch* launch, void* stream);

/* Several batches (up to 32 per launch, each with its own card among up to 4
 * distinct cards per launch, its own seed, event-index base and outputs) in one
 * fused persistent launch; larger sets are split into consecutive launches.
 * Each batch's results are those pdr_run gives it alone (same bits).  The
 * launch shape is sized for the largest event of all batches; launch may be
 * NULL (the tuned shape of batches[0]'s card, else the default). */
int pdr_run_multi(pdr_ctx* ctx, const pdr_batch* batches, uint32_t n, const pdr_outputs* outs,
                  const pdr_launch* launch, void* stream);

/* The plain per-event form: one launch per event (team = block per event),
 * for comparison with pdr_run.  Same outputs, same bits. */
int pdr_run_per_event(pdr_ctx* ctx, const pdr_batch* batch, const pdr_outputs* out,
                      void* stream);

/* End-to-end call with HOST buffers (pinned memory gives overlapped copies):
 * the batch (HOST pointers) goes to device memory from the context pool in
 * chunks of whole events (about 2 M particles each), each chunk runs as soon
 * as its inputs have arrived, and its records come back while later chunks
 * are copied in and computed.  Outputs are HOST buffers with the pdr_outputs
 * record types, DENSE: all tracks of event 0, then of event 1, ... without
 * gaps, likewise towers, eflow, cands and iso (one iso record per candidate);
 * counts[4e .. 4e + 3] gives each event's share.  Each record buffer needs
 * room for n_particles records, counts for n_events; debug is ignored.  The
 * results are those of pdr_run on the same batch (same bits).  Blocking; the
 * kernels run on `stream`, the copies on two streams of the context; calls
 * on one context are serialised. */
int pdr_run_host(pdr_ctx* ctx, const pdr_batch* host_batch, const pdr_outputs* host_out,
                 const pdr_launch* launch, void* stream);

/* Time the candidate launch shapes on this batch (each once after a warm-up)
 * and remember the fastest for batches of this card and size class; *best
 * (may be NULL) receives it.  The outputs are scratch for the trial runs.
 * Synchronises the stream. */
int pdr_autotune(pdr_ctx* ctx, const pdr_batch* batch, const pdr_outputs* scratch_out,
                 void* stream, pdr_launch* best);

/* Largest event (particles) of a batch, computed on the device (synchronous
 * on `stream`). */
int pdr_max_event_size(pdr_ctx* ctx, const pdr_batch* batch, void* stream, uint32_t* out);

/* Read and clear the device error word after synchronising `stream`.
 * PDR_OK, or PDR_EDEVICE with the reason in pdr_last_error. */
int pdr_check(pdr_ctx* ctx, void* stream);

/* ------------------------------------------------------------ pile-up merging -- */
/* Sec. 2.2: with a pile-up block, the parametric path first merges
 * minimum-bias interactions with each hard-scatter event, then applies the
 * detector card; the block gives the mean number of interactions, the Gaussian
 * vertex-z width and its truncation, and whether the hard-scatter vertex is
 * smeared too.  Per hard event e (event index event_index_base + e, the hard
 * batch's seed; Philox purposes 5 to 8, disjoint from the response's 1-4):
 *   - N ~ Poisson(mean) by inversion: the smallest k with w0 < T[k], where
 *     T[k] = floor(P(N <= k) 2^32) from the CDF summed in double from
 *     P(N = 0) = exp(-mean) by P(N = k) = P(N = k-1) mean / k, the first entry
 *     at or above 2^32 - 1 becoming 2^32 (w0: counter (0, event, 5, 0));
 *   - interaction k < N takes pool event floor(w0 n_pool / 2^32) (w0: counter
 *     (k, event, 6, 0)) at vertex z = sigma_z x (Box-Muller normal of words 1
 *     and 2 of counter (k, event, 6, a)), a the first attempt with
 *     |z| <= max_z in float32 (a truncated Gaussian);
 *   - its vertex time is t = sigma_t x (the normal of words 1 and 2 of
 *     counter (k, event, 7, a)), a the first attempt with |t| <= max_t;
 *   - the hard vertex shift z_hs and time t_hs are drawn likewise from
 *     counters (0, event, 5, a) and (0, event, 8, a) if smear_hs, else 0;
 *   - the merged event holds the hard particles (vertex z = own vz, or 0, plus
 *     z_hs; time t_hs) followed by the pool events of interactions 0..N-1 in
 *     that order, each particle at its interaction's z and t; pool particles
 *     are copied as stored (no rotation, no transverse vertex offset).
 * The pool is a CSR batch in DEVICE memory and stays owned by the caller. */
typedef struct pdr_pileup {
  uint64_t n_pool;                /* minimum-bias events in the pool (>= 1)        */
  const uint64_t* offsets;        /* [n_pool + 1]                                  */
  const float *pt, *eta, *phi, *mass;
  const int32_t* pdg;
  const int8_t* charge;
  double mean;                    /* mean interactions per hard event (>= 0)       */
  double sigma_z;                 /* vertex-z width (m)                            */
  double max_z;                   /* vertex-z truncation |z| <= max_z (m, > 0)     */
  double sigma_t;                 /* vertex-time width (s; the paper's default 160e-12) */
  double max_t;                   /* vertex-time truncation (s, > 0; default 800e-12)   */
  uint32_t smear_hs;              /* 1: shift the hard-scatter vertex as well      */
  uint32_t pad;
} pdr_pileup;

/* DEVICE arrays of a merged batch, each with room for the merged particle
 * count that pdr_pileup_offsets returns.  vt (vertex time, seconds) may be
 * NULL: the times are then not written. */
typedef struct pdr_particles {
  float *pt, *eta, *phi, *mass, *vz, *vt;
  int32_t* pdg;
  int8_t* charge;
} pdr_particles;

/* First pass: the merged CSR offsets [n_events + 1] (DEVICE, caller-owned)
 * and their total *total (HOST); synchronises `stream`.  The hard batch's
 * card_id and flags are ignored.  PDR_EINVAL for bad arguments, PDR_EOVERFLOW
 * if mean is too large for the Poisson table (mean > 4000), PDR_ENOMEM if the
 * context pool has no room for the per-event counts (8 B an event). */
int pdr_pileup_offsets(pdr_ctx* ctx, const pdr_batch* hard, const pdr_pileup* pu, uint64_t* merged_offsets,
                       uint64_t* total, void* stream);

/* Second pass: fill `out` from the same hard batch and pool.  Every event
 * recomputes its merged size and, if it differs from merged_offsets (a call
 * with other arguments than the first pass), writes nothing and sets the
 * device error word (pdr_check reports it).  Asynchronous on `stream`; the
 * result is a batch for pdr_run with merged_offsets and these arrays.
 * Events whose hard or drawn pool offsets decrease, or that draw a pool
 * event of 2^32 particles or more, are skipped in both passes and reported
 * as malformed offsets by pdr_check. */
int pdr_pileup_merge(pdr_ctx* ctx, const pdr_batch* hard, const pdr_pileup* pu, const uint64_t* merged_offsets,
                     const pdr_particles* out, void* stream);

/* ------------------------------------------- filter and event features -- */
/* Sec. 2.4: a filter drops entries of a collection in place by per-field
 * conditions combined with "all" (AND) or "any" (OR); the event features H_T
 * and missing E_T are recomputed from the survivors.  The paper defines
 * neither feature; here the PFlow collection is the energy-flow tracks plus
 * the energy-flow neutrals, H_T = sum of their pT and missing E_T = minus the
 * vector sum of their transverse momenta.  Object fields per collection:
 *   tracks    pt = smeared pT, eta/phi = momentum direction,
 *             e = sqrt(pT^2 cosh^2(eta) + m^2), et = pt, pdg/charge of the
 *             generated particle;
 *   neutrals  (EFlow) pt = et = dE / cosh(eta_c), e = dE, eta/phi = tower
 *             centre, pdg 22 (ECAL) or 130 (HCAL), charge 0;
 *   towers    pt = et = E' / cosh(eta_c), e = E', tower centre, pdg 0, charge 0;
 *   cands     pt, eta, phi as reconstructed, e = pt cosh(eta), et = pt,
 *             pdg/charge of the generated particle.
 * A float field is compared in float32 (the threshold rounded to float32), an
 * integer field (pdg, charge) as an integer; abs compares the magnitude;
 * PDR_OP_IN / PDR_OP_NOT_IN test membership in values[0..n_values).  No
 * conditions keep everything.  PFLOW filters tracks and neutrals alike. */
#define PDR_COLL_PFLOW 0
#define PDR_COLL_TRACK 1
#define PDR_COLL_NEUTRAL 2
#define PDR_COLL_TOWER 3
#define PDR_COLL_CAND 4

#define PDR_FIELD_PT 0
#define PDR_FIELD_ETA 1
#define PDR_FIELD_PHI 2
#define PDR_FIELD_E 3
#define PDR_FIELD_ET 4
#define PDR_FIELD_PDG 5
#define PDR_FIELD_CHARGE 6

#define PDR_OP_GT 0
#define PDR_OP_GE 1
#define PDR_OP_LT 2
#define PDR_OP_LE 3
#define PDR_OP_EQ 4
#define PDR_OP_NE 5
#define PDR_OP_IN 6
#define PDR_OP_NOT_IN 7

#define PDR_COMBINE_ALL 0
#define PDR_COMBINE_ANY 1

#define PDR_MAX_CONDITIONS 8
#define PDR_MAX_VALUES 8

typedef struct pdr_condition {
  uint32_t field, op;
  uint32_t abs;                   /* 1: compare |field|                              */
  uint32_t n_values;              /* 1 for comparisons; 1..PDR_MAX_VALUES for in/not in */
  double values[PDR_MAX_VALUES];  /* integral for pdg and charge                     */
} pdr_condition;

typedef struct pdr_filter {
  uint32_t collection;            /* PDR_COLL_*                                      */
  uint32_t combine;               /* PDR_COMBINE_*                                   */
  uint32_t n_conditions;          /* 0..PDR_MAX_CONDITIONS                           */
  uint32_t compact;               /* 1: drop the failing records in place            */
  uint32_t update_features;       /* 1: features from the survivors, 0: from all     */
  uint32_t pad;
  pdr_condition cond[PDR_MAX_CONDITIONS];
} pdr_filter;

typedef struct pdr_features {
  float ht;                       /* GeV */
  float met_x, met_y, met;        /* missing E_T vector and magnitude (GeV) */
} pdr_features;

/* Post-processing of pdr_run's outputs (all DEVICE, slot layout): `batch` is
 * the batch that produced `out` (its offsets, pdg, charge, mass and card are
 * read).  With a filter and compact = 1 the target collection's surviving
 * records are moved down in order (candidates together with their isolation
 * records) and counts are updated; with compact = 0 nothing in `out` changes.
 * filter may be NULL (no filter).  features [n_events] (DEVICE) may be NULL.
 * Sums are exact 64-bit fixed-point (quantum 2^-24 GeV) over float32 terms,
 * so results do not depend on the launch.  Asynchronous on `stream`; events
 * whose counts exceed their multiplicity are skipped and reported as
 * malformed by pdr_check.  PDR_EINVAL for a bad filter or track records that
 * are not 16-byte aligned, PDR_ENOTFOUND for an unknown card. */
int pdr_postprocess(pdr_ctx* ctx, const pdr_batch* batch, const pdr_outputs* out, const pdr_filter* filter,
                    pdr_features* features, void* stream);

/* ------------------------------------------------ track impact parameters -- */
/* The paper's output table (Sec. 2.5) lists d0, z0 and their errors for
 * charged particles.  For every track record of pdr_run's outputs, from the
 * generated particle it came from (pT, eta, phi, charge at its vertex
 * (vx, vy, vz)) and the card's field:
 *   - the point of closest approach (pca) to the beam axis of the particle's
 *     helix (straight line if B = 0), reached the shorter way along the helix;
 *   - d0 = (p_hat x pca)_z (signed transverse distance, p_hat the momentum
 *     direction at the pca), z0 = vz + s sinh(eta), s the signed transverse
 *     path from the vertex to the pca;
 *   - errors sigma = sqrt(a^2 + (b / pT)^2) per parameter; the record holds
 *     d0 + sigma_d0 n1 and z0 + sigma_z0 n2, n1 / n2 the Box-Muller normals of
 *     words (0, 1) / (2, 3) of Philox counter (particle index, event, 9, 0)
 *     under the batch's seed.
 * Transverse vertex offsets (vx, vy) enter only here: the detector response
 * propagates every particle from (0, 0, vz). */
typedef struct pdr_ip_params {
  double a_d0, b_d0;              /* m, m GeV */
  double a_z0, b_z0;              /* m, m GeV */
  const float* vx;                /* [n_particles] DEVICE, m, or NULL (0) */
  const float* vy;                /* [n_particles] DEVICE, m, or NULL (0) */
} pdr_ip_params;

typedef struct { float d0, z0, sigma_d0, sigma_z0; } pdr_ip;   /* m */

/* ip (DEVICE, slot layout parallel to out->tracks: event e's k-th track's
 * record at [offsets[e] + k]) for the tracks that pdr_run wrote into `out`
 * from `batch` (same seed and event_index_base).  Asynchronous on `stream`;
 * PDR_EINVAL for negative resolutions or null arrays, PDR_ENOTFOUND for an
 * unknown card; events whose track count exceeds their multiplicity are
 * skipped and reported by pdr_check. */
int pdr_track_ip(pdr_ctx* ctx, const pdr_batch* batch, const pdr_outputs* out, const pdr_ip_params* params,
                 pdr_ip* ip, void* stream);

/* pdr_run with the tracks' impact parameters computed in the same fused
 * launch: each accepted track's pdr_ip record is written beside its track
 * record, from the generated particle the smearing job already holds (ip:
 * DEVICE, slot layout parallel to out->tracks, like pdr_track_ip).  The
 * results are those of pdr_run followed by pdr_track_ip, bit for bit, without
 * a second pass over the generated particles.  Same launch shapes, errors
 * and asynchrony as pdr_run, plus PDR_EINVAL for a null ip or negative
 * resolutions. */
int pdr_run_ip(pdr_ctx* ctx, const pdr_batch* batch, const pdr_outputs* out, const pdr_ip_params* params,
               pdr_ip* ip, const pdr_launch* launch, void* stream);

/* ---------------------------------------------------------- jet clustering -- */
/* Sec. 2.4: jets from the PFlow (or truth) collection with the generalized-kT
 * family (anti-kT p = -1 by default, Cambridge/Aachen p = 0, kT p = 1, any
 * p), jet radius R, and cuts pT >= pt_min and at least nconst_min
 * constituents.  Sequential recombination: repeatedly the smallest of
 * d_iB = pT_i^(2p) and d_ij = min(pT_i^(2p), pT_j^(2p)) dR_ij^2 / R^2
 * (dR in rapidity and azimuth) over the remaining objects; a pair merges by
 * four-momentum addition, a beam distance makes a jet.  Jets are ordered by
 * decreasing pT.  The e+e- generalized kT (ee = 1) takes energies and
 * opening angles instead: d_iB = E_i^(2p), d_ij = min(E_i^(2p), E_j^(2p))
 * (1 - cos theta_ij) / (1 - cos R).  Substructure (the output table of Sec. 2.5): with the
 * energy correlation functions of the jet's constituents
 * e2 = sum_{i<j} z_i z_j dR_ij and e3 = sum_{i<j<k} z_i z_j z_k dR_ij dR_ik dR_jk
 * (z = pT / sum pT of the constituents, angular exponent 1), C2 = e3 / e2^2
 * and D2 = e3 / e2^3 (0 when e2 = 0).  PFlow objects are the energy-flow tracks (smeared pT,
 * momentum direction, the generated particle's mass) and the energy-flow
 * neutrals (massless, E = dE at the tower centre); truth objects are the
 * generated particles except neutrinos (|pdg| 12, 14, 16). */
#define PDR_JETS_PFLOW 0
#define PDR_JETS_TRUTH 1

typedef struct pdr_jet_params {
  uint32_t collection;            /* PDR_JETS_*                               */
  uint32_t nconst_min;            /* keep jets with at least this many objects */
  double p;                       /* -1 anti-kT, 0 Cambridge/Aachen, 1 kT      */
  double R;                       /* jet radius (> 0, <= 10; e+e-: <= pi)      */
  double pt_min;                  /* GeV                                       */
  uint32_t ee;                    /* 1: the e+e- generalized kT (below)        */
  uint32_t pad;
} pdr_jet_params;

typedef struct {
  float pt, eta, phi, mass;       /* GeV, pseudorapidity, azimuth, GeV          */
  float e;                        /* GeV                                        */
  uint32_t nconst;
  float c2, d2;                   /* substructure (below)                       */
} pdr_jet;

/* Clusters every event of `batch` (for PDR_JETS_PFLOW: the outputs `out` that
 * pdr_run wrote from it; out may be NULL for truth).  jets: DEVICE, slot
 * layout (event e's k-th jet at [offsets[e] + k]; at most as many jets as
 * the event has particles); jet_counts [n_events] DEVICE.  Each event is
 * clustered by one warp with its objects in shared memory; PDR_EOVERFLOW if
 * an event has more objects than fit (about 9,600; 8,200 for e+e-).  Synchronises `stream`
 * once to size the shared memory, then runs asynchronously.  Calls on one
 * context share its clustering scratch (four-momenta in device memory, grown
 * on demand): do not overlap two clusterings of one context on different
 * streams. */
int pdr_cluster_jets(pdr_ctx* ctx, const pdr_batch* batch, const pdr_outputs* out, const pdr_jet_params* params,
                     pdr_jet* jets, uint32_t* jet_counts, void* stream);

/* ----------------------------------------------------------- diagnostics -- */
/* The paper has no counterpart to this entry point: it exposes, for tests, the
 * single-precision function approximations the kernels use in place of the
 * library calls (each with an error bound stated in the library's source),
 * evaluated element-wise on DEVICE arrays: y[k] = f(x[k]) (PDR_FN_NORMAL:
 * the Box-Muller deviate of the words whose bits x[k] and x2[k] carry;
 * PDR_FN_U01: the uniform of the word whose bits x[k] carries).
 * Asynchronous on `stream`; PDR_EINVAL for an unknown function or a null array. */
#define PDR_FN_ASIN_HALF 0      /* asin(x), x in [0, 1/2]                      */
#define PDR_FN_SIN_HALF_TURN 1  /* sin(x), x in [0, pi]                        */
#define PDR_FN_LN_UNIT 2        /* ln(u), u in (0, 1)                          */
#define PDR_FN_LOG1P_POS 3      /* ln(1 + x), x >= 0                           */
#define PDR_FN_COS_TWO_PI 4     /* cos(2 pi u), u in (0, 1)                    */
#define PDR_FN_COSH 5           /* cosh(x)                                     */
#define PDR_FN_SINH 6           /* sinh(x)                                     */
#define PDR_FN_ASINH 7          /* asinh(x)                                    */
#define PDR_FN_U01 8            /* (2k + 1) / 2^24 for the top 23 bits k       */
#define PDR_FN_NORMAL 9         /* sqrt(-2 ln u01(a)) cos(2 pi u01(b))         */
#define PDR_FN_RCP 10           /* 1 / x                                       */
#define PDR_FN_SQRT 11          /* sqrt(x)                                     */
#define PDR_FN_EXP_FF_HI 12     /* e^x, x in [0, 88], float-float: hi part     */
#define PDR_FN_EXP_FF_LO 13     /*   ... and lo part (e^x ~ hi + lo)           */
#define PDR_FN_SINH_FF_HI 14    /* sinh(x), x >= 0, float-float: hi part       */
#define PDR_FN_SINH_FF_LO 15    /*   ... and lo part                           */
#define PDR_FN_COUNT 16
int pdr_math_eval(int fn, const float* x, const float* x2, float* y, uint64_t n, void* stream);

/* ------------------------------------------------------- allocation-free run -- */
/* The paper has no counterpart to this entry point; it exists for callers of
 * this library that may not allocate device memory when they run the response:
 * applications that hand out all device memory through their own fixed-budget
 * allocator and forbid allocations after start-up, or latency-critical paths
 * that cannot afford an allocation's implicit synchronisation.  The caller
 * passes HOST card and DEVICE inputs/outputs exactly as for pdr_run (the
 * batch's card_id is ignored); the library allocates nothing.  Everything else
 * the kernel needs - the expanded card, an error word, and the global-memory
 * tower tables for events larger than the shared-memory table - lives in one
 * static device array of PDR_NOALLOC_SCRATCH_BYTES compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *
 * The first call on a device looks up that array's device address (a one-time
 * set-up with the device current).  With CUDA's lazy module loading (the
 * default) the array's device memory is committed at that first call, not
 * when the library is loaded (CUDA_MODULE_LOADING=EAGER commits it at load):
 * a caller that gives the remaining device memory to its own allocator makes
 * one warm-up call first - a batch with n_events = 0 does the set-up and
 * nothing else.  Calls share the array and it keeps the previous call's
 * contents: each call re-stages the card, clears the error word and
 * re-initialises the tables it uses, but calls whose work overlaps on the GPU
 * race and must not be issued.  Every call copies the error word back and
 * synchronises `stream` before it returns, so it cannot be issued on a stream
 * that is being captured into a CUDA graph.  Device-side errors are reported
 * directly: PDR_EDEVICE for malformed CSR offsets, PDR_EOVERFLOW when an
 * event has more than 49152 particles or its tower tables do not fit in the
 * static array, PDR_EINVAL / PDR_ECARD for bad arguments or cards.  No context
 * is needed; messages go to pdr_last_error(NULL). */
#define PDR_NOALLOC_SCRATCH_BYTES (32ull << 20)
int pdr_run_noalloc(const pdr_card* card, const pdr_batch* batch, const pdr_outputs* out, void* stream);

/* ------------------------------------------------------- library-owned results -- */
/* Result view returned by pdr_fetch: DEVICE pointers owned by the library
 * until pdr_release(ticket); layouts as pdr_outputs. */
typedef struct pdr_result {
  uint64_t n_events, n_particles;
  const uint64_t* offsets;    /* = the batch's offsets (slot bases), copied into the pool */
  const uint32_t* counts;
  const pdr_track* tracks;
  const pdr_tower* towers;
  const pdr_eflow* eflow;
  const pdr_cand* cands;
  const pdr_iso* iso;
  const pdr_debug* debug;     /* NULL unless PDR_BATCH_DEBUG */
} pdr_result;

/* Allocate result buffers from the pool, enqueue the batch on `stream` and
 * return a ticket.  The caller keeps the batch's inputs alive until pdr_wait
 * returns PDR_OK.  PDR_ENOMEM when the pool has no room (admission by free
 * device memory); PDR_EBUSY when max_tickets are outstanding. */
int pdr_submit(pdr_ctx* ctx, const pdr_batch* batch, void* stream, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: no limit) for a ticket; PDR_ETIMEDOUT if it is
 * still running (the wait never hangs), PDR_EDEVICE on a device error. */
int pdr_wait(pdr_ctx* ctx, uint64_t ticket, int timeout_ms);
/* Result view of a finished ticket. */
int pdr_fetch(pdr_ctx* ctx, uint64_t ticket, pdr_result* r);
/* Return a ticket's buffers to the pool. */
int pdr_release(pdr_ctx* ctx, uint64_t ticket);

/* ---------------------------------------------------------------- serving -- */
/* A request loop on the device's behalf: requests (HOST batches) are admitted
 * in arrival order as soon as the context pool has room for their inputs and
 * results (admission by free device memory), their inputs are copied on a copy
 * stream, and admitted requests are grouped into waves - one fused launch of
 * up to 32 requests and 4 cards, replayed from a captured CUDA graph per launch
 * shape - while up to max_inflight_waves waves run, so requests that arrive
 * while others are on the GPU join the next wave (continuous batching).  Card
 * tables stay on the device; random numbers are counter-based, so a request's
 * results are the bits it gets alone (pdr_run with the same batch).  Tickets
 * are the same as pdr_submit's: pdr_wait / pdr_fetch (device results in the
 * slot layout of pdr_outputs) / pdr_release (which returns the memory used by
 * admission). */
typedef struct pdr_serve_options {
  uint32_t max_inflight_waves;   /* waves on the device at once (0: 2)            */
  uint32_t max_wave_requests;    /* requests in one wave (0 or > 32: 32)          */
  uint64_t max_wave_particles;   /* particles in one wave (0: 64M)                */
  uint32_t use_graphs;           /* 1: replay captured graphs, 0: plain launches  */
  uint32_t flags;                /* reserved, 0                                   */
} pdr_serve_options;

typedef struct pdr_serve_stats {
  uint64_t requests_done, events_done, particles_done, waves, admission_waits, graph_launches;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> results complete on the device */
  double span_s;                           /* first submit -> last completion          */
} pdr_serve_stats;

/* Start the loop (one per context).  opt may be NULL. */
int pdr_serve_start(pdr_ctx* ctx, const pdr_serve_options* opt);
/* Queue a request: HOST pointers (pinned memory copies fastest) that the caller
 * keeps alive and unchanged until pdr_wait returns PDR_OK.  Returns at once. */
int pdr_serve_submit(pdr_ctx* ctx, const pdr_batch* host_batch, uint64_t* ticket);
/* Latency and throughput of the requests completed so far. */
int pdr_serve_stats_get(pdr_ctx* ctx, pdr_serve_stats* out);
/* Finish queued and running requests, then stop the loop. */
int pdr_serve_stop(pdr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PDR_H */
