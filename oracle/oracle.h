/*
 * FP64 CPU oracle for the parametric detector response (TEST INFRASTRUCTURE).
 *
 * This is the plain, slow, obviously-correct reference that the CUDA path is
 * checked against.  Only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table
 * or constant generator with the CUDA library: it expands the detector card
 * itself, implements its own Philox4x32-10, and computes every step in double
 * precision in the order the method defines.
 *
 * The method is the paper's parametric backend (TorchDelphes, Sec. 2.2 and
 * App. D.1): particle propagation in the solenoid field, tracking efficiency,
 * momentum smearing, calorimeter response (towers), energy-flow merging, and
 * the lepton isolation of Sec. 2.4 (Eq. 1).  The paper prints no formulas for
 * the TorchDelphes modules; the readings used here (helix geometry, log-normal
 * smearing, tower centres, thresholds, counter-based random numbers) are the
 * project's and are listed in the design notes.
 *
 * Decisions taken on floating-point values (a tower index, a threshold, a cone
 * edge) are taken in float32, the CUDA kernel's precision: the double value is
 * rounded to float and compared with the float32 threshold or edge.  Every such
 * decision whose double value lies within a relative band g of its threshold is
 * reported as "marginal", and a caller may ask the oracle to take the other
 * branch of a marginal decision (a "flip").  The oracle refuses flips of
 * decisions that are not marginal.  This lets a test accept either outcome of a
 * decision that float32 rounding can legitimately change, and still check
 * everything downstream of it exactly.
 */
#ifndef PDR_ORACLE_H
#define PDR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXSEG 4      /* eta segments per calorimeter (per side)        */
#define OR_MAXEDGE 8     /* edges per piecewise-constant table axis         */
#define OR_MAXRING 512   /* eta rings per calorimeter (both sides)          */

/* Particle classes (from |pdg| and charge). */
enum { OR_CLS_E = 0, OR_CLS_MU = 1, OR_CLS_GAMMA = 2, OR_CLS_CHAD = 3,
       OR_CLS_NHAD = 4, OR_CLS_INVIS = 5 };
/* Calorimeters. */
enum { OR_ECAL = 0, OR_HCAL = 1 };
/* Resolution components. */
enum { OR_RES_TRACK = 0, OR_RES_MUON = 1, OR_RES_ECAL = 2, OR_RES_HCAL = 3 };
/* Random-number purposes (third Philox counter word). */
enum { OR_PURPOSE_TRACK = 1, OR_PURPOSE_ID = 2, OR_PURPOSE_TOWER_ECAL = 3,
       OR_PURPOSE_TOWER_HCAL = 4 };

/* Decision kinds (for marginal reports and flips). */
enum {
  OR_K_BARREL = 1,    /* id = particle: |z at barrel| <= L                    */
  OR_K_LOOP = 2,      /* id = particle: endcap turning angle psi < 2 pi         */
  OR_K_ETA = 3,       /* id = particle, aux = calo: eta-ring lookup           */
  OR_K_PHI = 4,       /* id = particle, aux = calo: phi-bin lookup            */
  OR_K_TWR_E = 5,     /* id = tower key: E' > E_min                           */
  OR_K_TWR_S = 6,     /* id = tower key: E'/sigma(E') > S_min                 */
  OR_K_EF_E = 7,      /* id = tower key: dE > E_min                           */
  OR_K_EF_S = 8,      /* id = tower key: dE/sigma(E') > S_min                 */
  OR_K_ISO_PT = 9,    /* id = object (track: particle, neutral: key), aux = 0 track / 1 neutral */
  OR_K_ISO_DR = 10,   /* id = candidate particle, aux = object id, aux2 = object type: dR^2 < dR_max^2 */
  OR_K_ISO_DRMIN = 11,/* same ids: dR^2 >= dR_min^2                            */
  OR_K_ISOLATED = 12  /* id = candidate particle: I < I_max                    */
};

/* Particle flag bits (per-particle debug record). */
#define OR_F_REACH   0x01u  /* reached the calorimeter surface                */
#define OR_F_BARREL  0x02u  /* hit the barrel (else endcap)                     */
#define OR_F_TRACKED 0x04u  /* accepted by the tracking efficiency              */
#define OR_F_CAND    0x08u  /* e/mu/gamma candidate accepted by its ID efficiency */
#define OR_F_ECAL    0x10u  /* deposited in ECAL                                */
#define OR_F_HCAL    0x20u  /* deposited in HCAL                                */

#define OR_NO_KEY 0xFFFFFFFFu

/* Raw detector card (the JSON card's numbers; units GeV, m, T). */
typedef struct {
  double B, R, L;
  int32_t nseg[2];
  double seg_eta_hi[2][OR_MAXSEG];
  int32_t seg_neta[2][OR_MAXSEG];
  int32_t seg_nphi[2][OR_MAXSEG];
  int32_t trk_npt, trk_neta;
  double trk_pt_edges[OR_MAXEDGE];
  double trk_eta_edges[OR_MAXEDGE];
  double trk_eff[3][OR_MAXEDGE][OR_MAXEDGE];  /* [hadron, electron, muon][pt bin][|eta| bin] */
  int32_t res_n[4];
  double res_edges[4][OR_MAXEDGE];
  double res_abcd[4][OR_MAXEDGE][4];         /* [component][|eta| bin][a, b, c, d] */
  int32_t id_n;
  double id_edges[OR_MAXEDGE];
  double id_eff[3][OR_MAXEDGE];              /* [electron, muon, photon][|eta| bin] */
  double e_min[2], s_min[2];
  double cand_ptmin, iso_dr, iso_drmin, iso_ptmin, iso_imax;
} oracle_card;

/* Per-particle record. */
typedef struct {
  double eta_pos, phi_pos;   /* position on the calorimeter surface (if reached) */
  double e;                  /* truth energy                                   */
  double cond;               /* |d eta_pos / d ln(psi)|: conditioning of eta_pos
                                on the turning angle (endcap helices; else 0)  */
  uint32_t key;              /* tower key deposited into, or OR_NO_KEY          */
  uint32_t flags;            /* OR_F_* bits                                    */
  uint32_t cls;              /* OR_CLS_*                                       */
  uint32_t pad;
} or_particle;

typedef struct {
  double pt, eta, phi, e;    /* smeared pT, momentum direction, track energy  */
  uint32_t idx, pad;         /* particle index in the event                    */
} or_track;

typedef struct {
  double esum, etrk;         /* pre-smearing deposit sum, sum of track energies */
  double e, et, sigma;       /* smeared energy, E'/cosh(eta_c), sigma(E')       */
  double eflow_e, eflow_et;  /* dE = E' - etrk and dE/cosh(eta_c)               */
  double eta_c, phi_c;       /* tower centre                                    */
  uint32_t key, owner;       /* tower key; lowest depositing particle index     */
  uint32_t kept, eflow_kept;
} or_tower;

typedef struct {
  double pt, eta, phi;       /* smeared pT, momentum direction                 */
  double iso_sum, iso_rel;   /* cone sum and I = sum / pT                       */
  uint32_t idx, cls;         /* particle index, 0 e / 1 mu / 2 gamma            */
  uint32_t isolated, pad;
} or_cand;

typedef struct {
  uint32_t kind, id, aux, aux2;
  double v, t;               /* decision value and threshold (double)          */
  double w;                  /* pair decisions: the object's pT contribution   */
  int32_t taken, alt;        /* branch taken; alternative (lookups: other bin) */
} or_marginal;

typedef struct { uint32_t kind, id, aux, aux2; } or_flip;

typedef struct {
  int32_t n_trk, n_twr, n_twr_kept, n_eflow, n_cand, n_marg, err, pad;
} or_counts;

/* ---- building blocks (exposed for the pin tests) ---- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double oracle_u01(uint32_t w);
double oracle_normal(uint32_t wa, uint32_t wb);
double oracle_lognormal(double x, double rel, double z);
double oracle_rel_resolution(const oracle_card* c, int comp, double abseta, double x);
uint64_t oracle_eff_threshold(double eff);
int oracle_classify(int32_t pdg, int32_t charge);
/* Propagation of one particle; returns reach (0/1).  barrel/eta_pos/phi_pos out. */
int oracle_propagate(const oracle_card* c, double pt, double eta, double phi, int32_t q,
                     double vz, int32_t* barrel, double* eta_pos, double* phi_pos);
/* Tower key of a position in a calorimeter, or OR_NO_KEY if outside coverage. */
uint32_t oracle_tower_key(const oracle_card* c, int calo, double eta_pos, double phi_pos);
/* Centre of a tower; returns 0 on success. */
int oracle_tower_centre(const oracle_card* c, uint32_t key, double* eta_c, double* phi_c,
                        int32_t* ring, int32_t* iphi);
int oracle_n_towers(const oracle_card* c, int calo);
/* Array forms for the statistical pins (element-wise, n elements). */
void oracle_philox_n(int64_t n, const uint32_t* ctr4, const uint32_t key[2], uint32_t* out4);
void oracle_normal_n(int64_t n, const uint32_t* wa, const uint32_t* wb, double* out);
void oracle_lognormal_n(int64_t n, double x, double rel, const double* z, double* out);

/* ---- one event, with decision reports and flips ----
 * Outputs are caller-allocated with room for n records each (marg: marg_cap).
 * Towers are returned in ascending key order, all of them (kept or not).
 * Returns 0, or a negative code: -1 bad argument, -2 a flip named a decision
 * that is not marginal, -3 marginal list overflow. */
int oracle_run_event(const oracle_card* c, int64_t n, const float* pt, const float* eta,
                     const float* phi, const float* mass, const int32_t* pdg,
                     const int8_t* charge, const float* vz, uint64_t seed, uint32_t event,
                     double g, const or_flip* flips, int32_t n_flips,
                     or_particle* part, or_track* trk, or_tower* twr, or_cand* cand,
                     or_marginal* marg, int32_t marg_cap, or_counts* counts);

/* ---- a whole CSR batch on nthreads host threads (CPU baseline) ----
 * counts_out[e*4 + {0,1,2,3}] = tracks, kept towers, EFlow neutrals, candidates.
 * Returns 0 or a negative code. */
int oracle_run_batch(const oracle_card* c, int64_t n_events, const uint64_t* offsets,
                     const float* pt, const float* eta, const float* phi, const float* mass,
                     const int32_t* pdg, const int8_t* charge, const float* vz,
                     uint64_t seed, uint32_t event_base, int32_t nthreads,
                     uint32_t* counts_out);

/* ---- pile-up merging (Sec. 2.2: with a pile-up block, the parametric path
 * first merges minimum-bias interactions with the hard-scatter event; the
 * block's parameters are listed with the generator configuration: mean
 * pile-up, vertex-z width sigma_z and truncation max_z_spread, and whether the
 * hard-scatter vertex is smeared).  Readings of what the paper leaves open:
 *   - N ~ Poisson(mean) interactions per hard event, drawn by inversion: N is
 *     the smallest k with w0 < T[k] (thresholds below), w0 from Philox counter
 *     (0, event, 5, 0);
 *   - interaction k (0 <= k < N) takes minimum-bias event floor(w0 * n_pool / 2^32)
 *     of the pool, w0 from counter (k, event, 6, 0), at vertex z = sigma_z * z
 *     with z the Box-Muller normal of (w1, w2) of counter (k, event, 6, a), a the
 *     first attempt with |z sigma_z| <= max_z (a truncated Gaussian);
 *   - its vertex time is t = sigma_t * (the normal of (w1, w2) of counter
 *     (k, event, 7, a)), a the first attempt with |t| <= max_t;
 *   - the hard-scatter vertex, if smeared, is z_hs from counter (0, event, 5, a)
 *     and t_hs from counter (0, event, 8, a) likewise; its particles keep
 *     their own z plus z_hs and have time t_hs;
 *   - the pool event's particles are used as stored (no rotation, no
 *     transverse vertex offset: the pile-up block has no x/y spread).
 * Each truncation is a decision on a float32 value; a draw whose |v| lies
 * within g max(|v|, bound) of its bound is counted as marginal. */
typedef struct oracle_pileup {
  double mean, sigma_z, max_z, sigma_t, max_t;
  int32_t smear_hs, pad;
} oracle_pileup;

/* Thresholds T[0..K-1] of the Poisson(mean) CDF: T[k] = floor(P(N <= k) 2^32),
 * the CDF summed in double from P(N = 0) = exp(-mean) by P(N = k) = P(N = k-1)
 * mean / k; the first entry at or above 2^32 - 1 is the last and becomes 2^32.
 * Returns K, or -1 if kmax entries do not reach it. */
int32_t oracle_poisson_thresholds(double mean, uint64_t* T, int32_t kmax);

/* The draws of one hard event: *n interactions (at most cap are written) with
 * pool indices idx[], vertex z[] (metres) and vertex times t[] (seconds), and
 * the hard vertex shift *z_hs and time *t_hs (0 unless smeared).  Returns the
 * number of marginal truncation decisions, or -1 if n exceeds cap. */
int32_t oracle_pileup_draws(const oracle_pileup* p, const uint64_t* T, int32_t K, uint64_t n_pool,
                            uint64_t seed, uint32_t event, double g, int32_t* n, uint32_t* idx,
                            double* z, double* t, int32_t cap, double* z_hs, double* t_hs);

/* The same with the parity protocol's forced branches: each (purpose, slot,
 * attempt) triple of flips[3 n_flips] names a truncation decision (purpose 5
 * hard vertex z, 8 hard vertex time, 6 interaction z, 7 interaction time;
 * slot the interaction; attempt the draw's counter word 3) to be taken the
 * other way.  Every listed decision must occur and be marginal, else the
 * call refuses and returns -2.  The triples of this run's marginal decisions
 * go to marg_out[3 marg_cap] (may be NULL). */
int32_t oracle_pileup_draws_forced(const oracle_pileup* p, const uint64_t* T, int32_t K, uint64_t n_pool,
                                   uint64_t seed, uint32_t event, double g, int32_t* n, uint32_t* idx,
                                   double* z, double* t, int32_t cap, double* z_hs, double* t_hs,
                                   const uint32_t* flips, int32_t n_flips, uint32_t* marg_out, int32_t marg_cap);

/* ---- track impact parameters (the paper's output table: d0, z0 and their
 * errors for charged particles; Sec. 2.5) ----
 * Readings (the paper gives no formula):
 *   - the track is the helix of the generated particle (pT, eta, phi at its
 *     production vertex (x0, y0, z0), charge q) in the card's field B along z:
 *     radius r = pT / (0.299792458 |q B|), its momentum azimuth turning by
 *     -h s / r with h = sign(q B), s the transverse path; a straight line if
 *     B = 0;
 *   - the point of closest approach (pca) is the point of that circle (line)
 *     in the transverse plane nearest to the beam axis (x = y = 0), reached
 *     by the shorter way along the helix (forward or backward, |turn| <= pi);
 *     if the axis is the circle's centre the pca is the vertex;
 *   - d0 = (p_hat x pca)_z = pca_y cos(phi_pca) - pca_x sin(phi_pca), with
 *     phi_pca the momentum azimuth at the pca; z0 = z0_vertex + s sinh(eta),
 *     s the signed transverse path from the vertex to the pca;
 *   - errors sigma = sqrt(a^2 + (b / pT)^2) with (a, b) per parameter, and the
 *     reconstructed values d0 + sigma_d0 n1, z0 + sigma_z0 n2 with n1 the
 *     Box-Muller normal of words 0, 1 and n2 of words 2, 3 of Philox counter
 *     (particle index, event, 9, 0). */
typedef struct oracle_ip_params {
  double a_d0, b_d0, a_z0, b_z0;   /* metres, metres x GeV */
} oracle_ip_params;

/* True d0 and z0 of one particle; *s_out (may be NULL) the signed path. */
void oracle_track_ip(const oracle_card* c, double pt, double eta, double phi, int32_t q, double x0, double y0,
                     double z0, double* d0, double* zz0, double* s_out);
/* The smeared pair and the errors: out[4] = d0', z0', sigma_d0, sigma_z0. */
void oracle_track_ip_smeared(const oracle_card* c, const oracle_ip_params* ip, double pt, double eta, double phi,
                             int32_t q, double x0, double y0, double z0, uint64_t seed, uint32_t event,
                             uint32_t idx, double out[4]);

/* ---- jet clustering (Sec. 2.4: FastJet's generalized-kT family on the
 * PFlow or truth collection; jet pT and constituent-count cuts) ----
 * The sequential recombination written out (FastJet's algorithm is not
 * copied; its definitions are textbook):
 *   - objects i carry four-momenta (px, py, pz, E), rapidity
 *     y = 0.5 ln((E + pz) / (E - pz)) and azimuth phi;
 *   - d_iB = pt_i^(2p), d_ij = min(pt_i^(2p), pt_j^(2p)) dR_ij^2 / R^2 with
 *     dR^2 = (y_i - y_j)^2 + dphi^2 (dphi wrapped into [-pi, pi]);
 *     p = -1 anti-kT, 0 Cambridge/Aachen, 1 kT;
 *   - repeatedly the smallest of all d_ij and d_iB over the active objects:
 *     a d_ij merges i and j (E-scheme: four-momenta added), a d_iB makes i a
 *     jet; ties go to the beam distance, then to the lower indices;
 *   - jets with pT >= pt_min and at least nconst_min constituents are kept,
 *     ordered by decreasing pT;
 *   - substructure (the output table of Sec. 2.5: D2 and C2): with the
 *     energy correlation functions of the jet's constituents
 *     e2 = sum_{i<j} z_i z_j dR_ij and e3 = sum_{i<j<k} z_i z_j z_k dR_ij dR_ik dR_jk
 *     (z_i = pT_i / sum pT, dR in rapidity and azimuth, angular exponent
 *     beta = 1), C2 = e3 / e2^2 and D2 = e3 / e2^3 (both 0 when e2 = 0).
 * With ee set (the e+e- generalized kT of the same family): d_iB = E_i^(2p),
 * d_ij = min(E_i^(2p), E_j^(2p)) (1 - cos theta_ij) / (1 - cos R), R <= pi,
 * with 1 - cos theta = |n_i - n_j|^2 / 2 for the unit directions n; pT cuts,
 * ordering and substructure as above.
 * A step is marginal when the runner-up distance (a different decision) lies
 * within the float32 uncertainty of the two distances: 1e-6 relative, plus for
 * pair distances min(pt^(2p)) (2 |dy| eps_y + 2 |dphi| eps_phi) / R^2 with
 * eps_y = 2^-23 max(|y_i|, |y_j|, 1) and eps_phi = 2^-23 pi (ee: the pair term
 * min(E^2p) 4 |n_i - n_j| 2^-22 / (2 (1 - cos R))). */
typedef struct or_jet {
  double px, py, pz, e;
  double pt, eta, phi, mass;
  double e2, e3, c2, d2;
  int32_t nconst, pad;
} or_jet;

/* Cluster n objects (four-momenta px, py, pz, e).  Writes the kept jets
 * (at most n) and returns their number, or -1 for bad arguments; *n_marg
 * counts the marginal steps. */
int32_t oracle_cluster(int64_t n, const double* px, const double* py, const double* pz, const double* e,
                       double p, double R, double pt_min, int32_t nconst_min, int32_t ee, or_jet* jets,
                       int32_t* n_marg);

/* The same, with the parity protocol's forced branches: at every step whose
 * index (0, 1, ... in recombination order) is listed in flips[n_flips] the
 * runner-up decision is taken instead of the smallest distance - only where
 * that step is marginal and exists (else the call refuses and returns -2).  The indices of
 * the marginal steps of this run go to marg_steps (up to marg_cap of them). */
int32_t oracle_cluster_forced(int64_t n, const double* px, const double* py, const double* pz, const double* e,
                              double p, double R, double pt_min, int32_t nconst_min, int32_t ee, or_jet* jets,
                              int32_t* n_marg, const int32_t* flips, int32_t n_flips, int32_t* marg_steps,
                              int32_t marg_cap);

#ifdef __cplusplus
}
#endif
#endif
