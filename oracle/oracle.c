/*
 * FP64 CPU oracle for the parametric detector response (TEST INFRASTRUCTURE).
 *
 * Only the tests, the package smoke check and the benchmark's CPU-baseline leg
 * may load this library; the product path never does.  See oracle.h for the
 * contract.  Every function below names the part of the method it follows:
 *
 *   Sec. 2.2 / App. D.1  TorchDelphes module chain: propagation, tracking
 *                        efficiency, momentum smearing, calorimeter response,
 *                        energy-flow merging (Towers, EFlowObjects).
 *   App. D.2             PropagatedParticle (deterministic intermediate).
 *   Sec. 2.4, Eq. 1      lepton isolation: cone sum of charged, neutral and
 *                        photon pT, excluding the lepton itself, over pT.
 *
 * The paper gives the module list but no module formulas; the readings coded
 * here are the project's (documented with the design): a helix in a uniform
 * solenoid field, Delphes-style piecewise-constant efficiencies, resolutions
 * sigma/x = a/sqrt(x) (+) b/x (+) c (+) d x, log-normal smearing with mean x and
 * standard deviation sigma, tower energy placed at the tower centre, strict
 * thresholds on energy and significance, and counter-based Philox4x32-10
 * random numbers keyed by (seed, event, slot, purpose).
 *
 * Everything is computed in double precision, plainly and in the order the
 * method defines; there is no blocking or reordering.  Tower sums add the
 * deposits in ascending particle index.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define TWO_PI (2.0 * M_PI)
#define C_LIGHT_GEV_PER_TM 0.299792458 /* pT[GeV] = 0.299792458 * |q| * B[T] * r[m] */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds; each round multiplies counter words */
/* 0 and 2 by the two Philox multipliers, xors the high halves into words 1   */
/* and 3 together with the round key, and permutes; the key is bumped by the  */
/* Weyl constants between rounds.                                             */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(uint64_t seed, uint32_t slot, uint32_t event, uint32_t purpose, uint32_t w[4]) {
  uint32_t ctr[4] = {slot, event, purpose, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, w);
}

/* Uniform in (0, 1): the top 23 bits k of w give (2k + 1) / 2^24, a value that
 * float32 represents exactly (24-bit odd integer over a power of two). */
double oracle_u01(uint32_t w) {
  return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Standard normal by the Box-Muller transform (cosine branch). */
double oracle_normal(uint32_t wa, uint32_t wb) {
  double u1 = oracle_u01(wa), u2 = oracle_u01(wb);
  return sqrt(-2.0 * log(u1)) * cos(TWO_PI * u2);
}

/* Log-normal variate with mean x and standard deviation rel * x (reading of
 * the smearing modules): s^2 = log(1 + rel^2), x' = x exp(-s^2/2 + s z). */
double oracle_lognormal(double x, double rel, double z) {
  double s2 = log1p(rel * rel);
  double s = sqrt(s2);
  return x * exp(-0.5 * s2 + s * z);
}

void oracle_philox_n(int64_t n, const uint32_t* ctr4, const uint32_t key[2], uint32_t* out4) {
  for (int64_t i = 0; i < n; ++i) oracle_philox4x32_10(ctr4 + 4 * i, key, out4 + 4 * i);
}

void oracle_normal_n(int64_t n, const uint32_t* wa, const uint32_t* wb, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = oracle_normal(wa[i], wb[i]);
}

void oracle_lognormal_n(int64_t n, double x, double rel, const double* z, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = oracle_lognormal(x, rel, z[i]);
}

/* Efficiency as a 32-bit acceptance threshold: pass iff (u32 draw) < T. */
uint64_t oracle_eff_threshold(double eff) {
  if (eff >= 1.0) return 4294967296ull;
  if (!(eff > 0.0)) return 0ull;
  return (uint64_t)floor(eff * 4294967296.0);
}

/* Largest k with float(edges[k]) <= float(x); -1 if x lies below edges[0]. */
static int lookup_f32(const double* edges, int n, double x) {
  float xf = (float)x;
  int k = -1;
  for (int j = 0; j < n; ++j)
    if ((float)edges[j] <= xf) k = j;
  return k;
}

/* sigma(x)/x = sqrt(a^2/x + b^2/x^2 + c^2 + d^2 x^2), coefficients chosen by
 * the |eta| bin of the component's table. */
double oracle_rel_resolution(const oracle_card* c, int comp, double abseta, double x) {
  int k = lookup_f32(c->res_edges[comp], c->res_n[comp], abseta);
  if (k < 0) k = 0;
  double a = c->res_abcd[comp][k][0], b = c->res_abcd[comp][k][1];
  double cc = c->res_abcd[comp][k][2], d = c->res_abcd[comp][k][3];
  return sqrt(a * a / x + b * b / (x * x) + cc * cc + d * d * x * x);
}

int oracle_classify(int32_t pdg, int32_t charge) {
  int32_t a = pdg < 0 ? -pdg : pdg;
  if (a == 11) return OR_CLS_E;
  if (a == 13) return OR_CLS_MU;
  if (a == 22) return OR_CLS_GAMMA;
  if (a == 12 || a == 14 || a == 16) return OR_CLS_INVIS;
  return charge != 0 ? OR_CLS_CHAD : OR_CLS_NHAD;
}

/* ------------------------------------------------------------------------ */
/* Calorimeter grid expanded from the card.  Each side of eta = 0 is cut into */
/* segments; segment s covers [lo_s, hi_s] in n_s rings with n_phi_s towers   */
/* per ring.  Ring edges inside a segment are lo + ((hi - lo) * k) / n for     */
/* 0 < k < n, with the segment ends exactly lo and hi.  Rings are numbered     */
/* from the most negative eta upward; ring r spans [edge[r], edge[r+1]).       */
/* Tower id = base[ring] + phi bin; phi bin edges are -pi + (2 pi k) / n_phi   */
/* for 0 < k < n_phi, with ends -pi and pi.  Key = calo << 24 | id.            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nring;
  double edge[OR_MAXRING + 1];
  int nphi[OR_MAXRING];
  int base[OR_MAXRING];
  int ntowers;
} or_grid;

static int build_grid(const oracle_card* c, int calo, or_grid* g) {
  double p[OR_MAXRING / 2 + 1];
  int pn[OR_MAXRING / 2];
  int m = 0;
  double lo = 0.0;
  p[0] = 0.0;
  for (int s = 0; s < c->nseg[calo]; ++s) {
    double hi = c->seg_eta_hi[calo][s];
    int n = c->seg_neta[calo][s];
    if (n <= 0 || m + n > OR_MAXRING / 2) return -1;
    for (int k = 1; k <= n; ++k) {
      p[m + k] = (k == n) ? hi : lo + ((hi - lo) * (double)k) / (double)n;
      pn[m + k - 1] = c->seg_nphi[calo][s];
    }
    m += n;
    lo = hi;
  }
  g->nring = 2 * m;
  for (int j = 0; j <= m; ++j) {
    g->edge[m + j] = p[j];
    g->edge[m - j] = -p[j];
  }
  g->edge[m] = 0.0;
  for (int r = 0; r < m; ++r) {
    g->nphi[m + r] = pn[r];
    g->nphi[m - 1 - r] = pn[r];
  }
  int base = 0;
  for (int r = 0; r < g->nring; ++r) {
    g->base[r] = base;
    base += g->nphi[r];
  }
  g->ntowers = base;
  return 0;
}

static double phi_edge(int nphi, int k) {
  if (k <= 0) return -M_PI;
  if (k >= nphi) return M_PI;
  return -M_PI + (TWO_PI * (double)k) / (double)nphi;
}

/* ------------------------------------------------------------------------ */
/* Decisions.  v is compared with t in float32; a decision is marginal when   */
/* |v - t| <= g * max(|v|, |t|, scale).                                       */
/* ------------------------------------------------------------------------ */
enum { OP_GT = 0, OP_LT = 1, OP_LE = 2, OP_GE = 3 };

typedef struct {
  const or_flip* flips;
  int nflips;
  or_marginal* marg;
  int nmarg, cap; /* cap < 0: do not record */
  int overflow;
  double g;
  int err;
} or_dctx;

static int find_flip(const or_dctx* d, uint32_t kind, uint32_t id, uint32_t aux, uint32_t aux2) {
  for (int i = 0; i < d->nflips; ++i)
    if (d->flips[i].kind == kind && d->flips[i].id == id && d->flips[i].aux == aux &&
        d->flips[i].aux2 == aux2)
      return 1;
  return 0;
}

static void record(or_dctx* d, uint32_t kind, uint32_t id, uint32_t aux, uint32_t aux2,
                   double v, double t, double w, int taken, int alt) {
  if (d->cap < 0) return;
  if (d->nmarg >= d->cap) { d->overflow = 1; return; }
  or_marginal* m = &d->marg[d->nmarg++];
  m->kind = kind; m->id = id; m->aux = aux; m->aux2 = aux2;
  m->v = v; m->t = t; m->w = w; m->taken = taken; m->alt = alt;
}

static int decide(or_dctx* d, uint32_t kind, uint32_t id, uint32_t aux, uint32_t aux2,
                  int op, double v, double t, double scale, double w) {
  float vf = (float)v, tf = (float)t;
  int res;
  switch (op) {
    case OP_GT: res = vf > tf; break;
    case OP_LT: res = vf < tf; break;
    case OP_LE: res = vf <= tf; break;
    default: res = vf >= tf; break;
  }
  double band = d->g * fmax(fmax(fabs(v), fabs(t)), scale);
  int marginal = isfinite(v) && fabs(v - t) <= band;
  if (d->nflips > 0 && find_flip(d, kind, id, aux, aux2)) {
    if (!marginal) d->err = -2;
    else res = !res;
  }
  if (marginal) record(d, kind, id, aux, aux2, v, t, w, res, !res);
  return res;
}

/* Eta-ring lookup with decision report: ring index, or -1 outside coverage. */
static int ring_decide(or_dctx* d, uint32_t id, int calo, const or_grid* g, double v) {
  int m = g->nring;
  float vf = (float)v;
  int k = -1;
  for (int j = 0; j <= m; ++j)
    if ((float)g->edge[j] <= vf) k = j;
  int ring = (k >= 0 && k < m) ? k : -1;
  int jn = 0;
  double dn = INFINITY;
  for (int j = 0; j <= m; ++j) {
    double dd = fabs(v - (double)(float)g->edge[j]);
    if (dd < dn) { dn = dd; jn = j; }
  }
  int below = jn - 1 >= 0 ? jn - 1 : -1;
  int above = jn < m ? jn : -1;
  int marginal = isfinite(v) && dn <= d->g * fmax(fabs(v), 1.0) &&
                 (ring == below || ring == above);
  int alt = (ring == above) ? below : above;
  if (d->nflips > 0 && find_flip(d, OR_K_ETA, id, (uint32_t)calo, 0)) {
    if (!marginal) d->err = -2;
    else { int t = ring; ring = alt; alt = t; }
  }
  if (marginal)
    record(d, OR_K_ETA, id, (uint32_t)calo, 0, v, (double)(float)g->edge[jn], 0.0, ring, alt);
  return ring;
}

/* Phi-bin lookup with decision report (clamped to [0, nphi - 1]). */
static int phi_decide(or_dctx* d, uint32_t id, int calo, int nphi, double v) {
  float vf = (float)v;
  int k = 0;
  for (int j = 0; j <= nphi; ++j)
    if ((float)phi_edge(nphi, j) <= vf) k = j;
  if (k > nphi - 1) k = nphi - 1;
  int jn = 0;
  double dn = INFINITY;
  for (int j = 0; j <= nphi; ++j) {
    double dd = fabs(v - (double)(float)phi_edge(nphi, j));
    if (dd < dn) { dn = dd; jn = j; }
  }
  int below = (jn - 1 + nphi) % nphi;
  int above = jn % nphi;
  int marginal = isfinite(v) && dn <= d->g * M_PI && (k == below || k == above);
  int alt = (k == above) ? below : above;
  if (d->nflips > 0 && find_flip(d, OR_K_PHI, id, (uint32_t)calo, 0)) {
    if (!marginal) d->err = -2;
    else { int t = k; k = alt; alt = t; }
  }
  if (marginal)
    record(d, OR_K_PHI, id, (uint32_t)calo, 0, v, (double)(float)phi_edge(nphi, jn), 0.0, k, alt);
  return k;
}

/* ------------------------------------------------------------------------ */
/* Propagation to the calorimeter cylinder (radius R, half-length L) in a     */
/* uniform field B along z (App. D.2 PropagatedParticle).  The particle starts */
/* at (0, 0, vz).  Neutral particles (or B = 0) move on a straight line.       */
/* Charged ones move on a helix of radius r = pT / (0.299792458 |q| |B|); the  */
/* momentum azimuth turns by -h s / r over transverse arc length s, with        */
/* h = sign(q B), and the distance from the axis is rho(s) = 2 r |sin(s/2r)|.   */
/* The barrel is reached iff 2 r >= R, first at s = 2 r asin(R / 2r), where the */
/* position azimuth is phi - h asin(R / 2r).  Otherwise, or if |z| > L there,   */
/* the endcap z = sign(pz) L is hit after turning angle psi = s_z / r, with     */
/* rho = 2 r |sin(psi/2)| and position azimuth phi - h psi / 2, unless psi is   */
/* at least 2 pi (a looper, dropped).  eta_pos = asinh(z / rho).               */
/* ------------------------------------------------------------------------ */
static int propagate_dec(const oracle_card* c, or_dctx* d, uint32_t id, double pt, double eta,
                         double phi, int q, double vz, int* barrel, double* eta_pos,
                         double* phi_pos, double* cond) {
  const double L = c->L, R = c->R, B = c->B;
  *barrel = 0;
  *eta_pos = 0.0;
  *phi_pos = 0.0;
  *cond = 0.0;
  if (!((float)fabs(vz) <= (float)L)) return 0; /* produced outside the detector */
  double sh = sinh(eta);                          /* pz / pT */
  if (q == 0 || B == 0.0) {
    if (vz == 0.0) {
      /* From the axis origin a straight line keeps its direction exactly. */
      *barrel = decide(d, OR_K_BARREL, id, 0, 0, OP_LE, fabs(R * sh), L, L, 0.0);
      *eta_pos = eta;
      *phi_pos = phi;
      return 1;
    }
    double z = vz + R * sh;
    *barrel = decide(d, OR_K_BARREL, id, 0, 0, OP_LE, fabs(z), L, L, 0.0);
    if (*barrel) {
      *eta_pos = asinh(z / R);
    } else {
      double ze = sh > 0.0 ? L : -L;
      double rho = (ze - vz) / sh;
      *eta_pos = asinh(ze / rho);
    }
    *phi_pos = phi;
    return 1;
  }
  double kq = C_LIGHT_GEV_PER_TM * fabs((double)q) * fabs(B);
  double r = pt / kq;
  double h = ((q > 0) == (B > 0.0)) ? 1.0 : -1.0;
  double cR = kq * R; /* R / (2 r) = cR / (2 pT) */
  int reach_barrel = (float)(2.0 * pt) >= (float)cR;
  double a = 0.0, z = 0.0, pphi;
  if (reach_barrel) {
    double x = cR / (2.0 * pt);
    if (x > 1.0) x = 1.0;
    a = asin(x);
    z = vz + 2.0 * r * a * sh;
    *barrel = decide(d, OR_K_BARREL, id, 0, 0, OP_LE, fabs(z), L, L, 0.0);
  }
  if (*barrel) {
    *eta_pos = asinh(z / R);
    pphi = phi - h * a;
  } else {
    if (sh == 0.0) return 0; /* pz = 0 and the barrel is out of reach */
    double ze = sh > 0.0 ? L : -L;
    double sz = (ze - vz) / sh;
    double psi = sz / r;
    if (!decide(d, OR_K_LOOP, id, 0, 0, OP_LT, psi, TWO_PI, TWO_PI, 0.0)) return 0;
    double rho = 2.0 * r * fabs(sin(0.5 * psi));
    *eta_pos = asinh(ze / rho);
    pphi = phi - h * 0.5 * psi;
    /* d eta_pos / d ln psi = -(L/rho)/sqrt(1 + (L/rho)^2) * (psi/2) cot(psi/2):
     * large when the helix has nearly closed (psi -> 2 pi, rho -> 0). */
    double lr = fabs(ze) / rho;
    *cond = lr / sqrt(1.0 + lr * lr) * fabs(0.5 * psi * cos(0.5 * psi) / sin(0.5 * psi));
  }
  if (pphi < -M_PI) pphi += TWO_PI;
  else if (pphi >= M_PI) pphi -= TWO_PI;
  *phi_pos = pphi;
  return 1;
}

int oracle_propagate(const oracle_card* c, double pt, double eta, double phi, int32_t q,
                     double vz, int32_t* barrel, double* eta_pos, double* phi_pos) {
  or_dctx d;
  memset(&d, 0, sizeof d);
  d.cap = -1;
  int b = 0;
  double cond = 0.0;
  int reach = propagate_dec(c, &d, 0, pt, eta, phi, q, vz, &b, eta_pos, phi_pos, &cond);
  *barrel = b;
  return reach;
}

uint32_t oracle_tower_key(const oracle_card* c, int calo, double eta_pos, double phi_pos) {
  or_grid g;
  if (build_grid(c, calo, &g)) return OR_NO_KEY;
  or_dctx d;
  memset(&d, 0, sizeof d);
  d.cap = -1;
  int ring = ring_decide(&d, 0, calo, &g, eta_pos);
  if (ring < 0) return OR_NO_KEY;
  int iphi = phi_decide(&d, 0, calo, g.nphi[ring], phi_pos);
  return ((uint32_t)calo << 24) | (uint32_t)(g.base[ring] + iphi);
}

static int centre_of(const or_grid* g, uint32_t key, double* eta_c, double* phi_c, int* ring,
                     int* iphi) {
  int id = (int)(key & 0xFFFFFFu);
  if (id < 0 || id >= g->ntowers) return -1;
  int r = 0;
  for (int j = 0; j < g->nring; ++j)
    if (g->base[j] <= id) r = j;
  int k = id - g->base[r];
  *ring = r;
  *iphi = k;
  *eta_c = 0.5 * (g->edge[r] + g->edge[r + 1]);
  *phi_c = 0.5 * (phi_edge(g->nphi[r], k) + phi_edge(g->nphi[r], k + 1));
  return 0;
}

int oracle_tower_centre(const oracle_card* c, uint32_t key, double* eta_c, double* phi_c,
                        int32_t* ring, int32_t* iphi) {
  int calo = (int)(key >> 24);
  if (calo < 0 || calo > 1) return -1;
  or_grid g;
  if (build_grid(c, calo, &g)) return -1;
  int r, k;
  if (centre_of(&g, key, eta_c, phi_c, &r, &k)) return -1;
  *ring = r;
  *iphi = k;
  return 0;
}

int oracle_n_towers(const oracle_card* c, int calo) {
  or_grid g;
  if (build_grid(c, calo, &g)) return -1;
  return g.ntowers;
}

/* ------------------------------------------------------------------------ */
/* One event.                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t key, idx;
  double e, etrk;
} or_deposit;

static int cmp_deposit(const void* a, const void* b) {
  const or_deposit* x = (const or_deposit*)a;
  const or_deposit* y = (const or_deposit*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

static double wrap_dphi(double dphi) {
  if (dphi >= M_PI) dphi -= TWO_PI;
  else if (dphi < -M_PI) dphi += TWO_PI;
  return dphi;
}

static int run_event_impl(const oracle_card* c, const or_grid grid[2], int64_t n,
                          const float* pt, const float* eta, const float* phi,
                          const float* mass, const int32_t* pdg, const int8_t* charge,
                          const float* vz, uint64_t seed, uint32_t event, or_dctx* d,
                          or_particle* part, or_track* trk, or_tower* twr, or_cand* cand,
                          or_deposit* dep, uint32_t* cand_key, or_counts* counts) {
  int n_trk = 0, n_cand = 0, nd = 0;
  for (int64_t ii = 0; ii < n; ++ii) {
    uint32_t i = (uint32_t)ii;
    or_particle* P = &part[ii];
    memset(P, 0, sizeof *P);
    P->key = OR_NO_KEY;
    const double PT = pt[ii], ETA = eta[ii], PHI = phi[ii], M = mass[ii];
    const int q = charge[ii];
    const double VZ = vz ? (double)vz[ii] : 0.0;
    const int cls = oracle_classify(pdg[ii], q);
    P->cls = (uint32_t)cls;
    const double cosh_eta = cosh(ETA);
    const double pcosh = PT * cosh_eta; /* |p| */
    const double E = sqrt(pcosh * pcosh + M * M);
    P->e = E;
    if (cls == OR_CLS_INVIS) continue;

    /* S1: propagation */
    int barrel = 0;
    double ep = 0.0, pp = 0.0, cond = 0.0;
    if (!propagate_dec(c, d, i, PT, ETA, PHI, q, VZ, &barrel, &ep, &pp, &cond)) continue;
    P->flags |= OR_F_REACH | (barrel ? OR_F_BARREL : 0u);
    P->eta_pos = ep;
    P->phi_pos = pp;
    P->cond = cond;

    /* S5: which calorimeter tower receives the deposit.  e/gamma go to ECAL,
     * or to HCAL where ECAL does not cover; hadrons to HCAL; mu/nu to none. */
    int calo = -1, ring = -1;
    if (cls == OR_CLS_E || cls == OR_CLS_GAMMA) {
      ring = ring_decide(d, i, OR_ECAL, &grid[OR_ECAL], ep);
      if (ring >= 0) calo = OR_ECAL;
      else {
        ring = ring_decide(d, i, OR_HCAL, &grid[OR_HCAL], ep);
        if (ring >= 0) calo = OR_HCAL;
      }
    } else if (cls == OR_CLS_CHAD || cls == OR_CLS_NHAD) {
      ring = ring_decide(d, i, OR_HCAL, &grid[OR_HCAL], ep);
      if (ring >= 0) calo = OR_HCAL;
    }
    uint32_t key = OR_NO_KEY;
    if (calo >= 0) {
      int iphi = phi_decide(d, i, calo, grid[calo].nphi[ring], pp);
      key = ((uint32_t)calo << 24) | (uint32_t)(grid[calo].base[ring] + iphi);
      P->key = key;
      P->flags |= calo == OR_ECAL ? OR_F_ECAL : OR_F_HCAL;
    }

    /* S2, S3: tracking efficiency and momentum smearing (charged, reached). */
    int tracked = 0;
    double etrk = 0.0;
    if (q != 0) {
      int tc = cls == OR_CLS_E ? 1 : (cls == OR_CLS_MU ? 2 : 0);
      int kp = lookup_f32(c->trk_pt_edges, c->trk_npt, PT);
      int ke = lookup_f32(c->trk_eta_edges, c->trk_neta, fabs(ETA));
      double eff = (kp >= 0 && ke >= 0) ? c->trk_eff[tc][kp][ke] : 0.0;
      uint32_t w[4];
      draw(seed, i, event, OR_PURPOSE_TRACK, w);
      if ((uint64_t)w[0] < oracle_eff_threshold(eff)) {
        tracked = 1;
        double z = oracle_normal(w[1], w[2]);
        double rel = oracle_rel_resolution(c, OR_RES_TRACK, fabs(ETA), PT);
        double ptp = oracle_lognormal(PT, rel, z);
        double pc = ptp * cosh_eta;
        etrk = sqrt(pc * pc + M * M);
        or_track* T = &trk[n_trk++];
        T->pt = ptp; T->eta = ETA; T->phi = PHI; T->e = etrk; T->idx = i; T->pad = 0;
        P->flags |= OR_F_TRACKED;
      }
    }

    /* S4: electron, muon and photon candidates: identification efficiency
     * and energy (e, gamma: ECAL resolution) or momentum (mu) smearing. */
    int cc = -1;
    if (cls == OR_CLS_E && tracked) cc = 0;
    else if (cls == OR_CLS_MU && tracked) cc = 1;
    else if (cls == OR_CLS_GAMMA && calo == OR_ECAL) cc = 2;
    if (cc >= 0 && (float)PT > (float)c->cand_ptmin) {
      int ke = lookup_f32(c->id_edges, c->id_n, fabs(ETA));
      double eff = ke >= 0 ? c->id_eff[cc][ke] : 0.0;
      uint32_t w[4];
      draw(seed, i, event, OR_PURPOSE_ID, w);
      if ((uint64_t)w[0] < oracle_eff_threshold(eff)) {
        double z = oracle_normal(w[1], w[2]);
        double ptp;
        if (cc != 1) {
          double rel = oracle_rel_resolution(c, OR_RES_ECAL, fabs(ETA), E);
          ptp = oracle_lognormal(E, rel, z) / cosh_eta;
        } else {
          double rel = oracle_rel_resolution(c, OR_RES_MUON, fabs(ETA), PT);
          ptp = oracle_lognormal(PT, rel, z);
        }
        cand_key[n_cand] = key;
        or_cand* C = &cand[n_cand++];
        memset(C, 0, sizeof *C);
        C->pt = ptp; C->eta = ETA; C->phi = PHI; C->idx = i; C->cls = (uint32_t)cc;
        P->flags |= OR_F_CAND;
      }
    }

    /* S5: the deposit (and, for tracked e and hadrons, the track energy that
     * energy flow will subtract from the same tower). */
    if (calo >= 0) {
      or_deposit* D = &dep[nd++];
      D->key = key; D->idx = i; D->e = E; D->etrk = tracked ? etrk : 0.0;
    }
  }

  /* S5: per-tower sums in ascending particle index. */
  qsort(dep, (size_t)nd, sizeof(or_deposit), cmp_deposit);
  int nt = 0, n_kept = 0, n_eflow = 0;
  for (int j = 0; j < nd;) {
    uint32_t key = dep[j].key;
    double esum = 0.0, etrk = 0.0;
    uint32_t owner = dep[j].idx;
    for (; j < nd && dep[j].key == key; ++j) {
      esum += dep[j].e;
      etrk += dep[j].etrk;
    }
    or_tower* T = &twr[nt++];
    memset(T, 0, sizeof *T);
    T->key = key; T->owner = owner; T->esum = esum; T->etrk = etrk;
    int calo = (int)(key >> 24), r, k;
    centre_of(&grid[calo], key, &T->eta_c, &T->phi_c, &r, &k);
    int comp = calo == OR_ECAL ? OR_RES_ECAL : OR_RES_HCAL;
    /* S6: tower smearing, keyed by the tower id, and thresholds. */
    uint32_t w[4];
    draw(seed, key & 0xFFFFFFu, event,
         calo == OR_ECAL ? OR_PURPOSE_TOWER_ECAL : OR_PURPOSE_TOWER_HCAL, w);
    double z = oracle_normal(w[0], w[1]);
    double ae = fabs(T->eta_c);
    double e1 = oracle_lognormal(esum, oracle_rel_resolution(c, comp, ae, esum), z);
    double sigma = e1 * oracle_rel_resolution(c, comp, ae, e1);
    double cosh_c = cosh(T->eta_c);
    T->e = e1; T->sigma = sigma; T->et = e1 / cosh_c;
    int k1 = decide(d, OR_K_TWR_E, key, 0, 0, OP_GT, e1, c->e_min[calo], 0.0, 0.0);
    int k2 = decide(d, OR_K_TWR_S, key, 0, 0, OP_GT, e1 / sigma, c->s_min[calo], 0.0, 0.0);
    T->kept = (uint32_t)(k1 && k2);
    /* S7: energy flow: the excess over the matched track energy becomes a
     * neutral (photon for ECAL, neutral hadron for HCAL) at the tower centre. */
    double de = e1 - etrk;
    T->eflow_e = de; T->eflow_et = de / cosh_c;
    int f1 = decide(d, OR_K_EF_E, key, 0, 0, OP_GT, de, c->e_min[calo], 0.0, 0.0);
    int f2 = decide(d, OR_K_EF_S, key, 0, 0, OP_GT, de / sigma, c->s_min[calo], 0.0, 0.0);
    T->eflow_kept = (uint32_t)(f1 && f2);
    n_kept += (int)T->kept;
    n_eflow += (int)T->eflow_kept;
  }

  /* S8: isolation (Sec. 2.4, Eq. 1).  Objects are the energy-flow tracks and
   * neutrals above the pT floor; the candidate's own track and the neutral of
   * the tower it deposited into are the lepton itself and are excluded, as are
   * objects closer than dR_min. */
  if (n_cand > 0) {
    unsigned char* tpass = (unsigned char*)calloc((size_t)(n_trk + nt + 1), 1);
    unsigned char* npass = tpass + n_trk;
    for (int t = 0; t < n_trk; ++t)
      tpass[t] = (unsigned char)decide(d, OR_K_ISO_PT, trk[t].idx, 0, 0, OP_GT, trk[t].pt,
                                       c->iso_ptmin, 0.0, 0.0);
    for (int t = 0; t < nt; ++t)
      npass[t] = twr[t].eflow_kept
                     ? (unsigned char)decide(d, OR_K_ISO_PT, twr[t].key, 1, 0, OP_GT,
                                             twr[t].eflow_et, c->iso_ptmin, 0.0, 0.0)
                     : 0;
    const double dr2max = c->iso_dr * c->iso_dr, dr2min = c->iso_drmin * c->iso_drmin;
    for (int ci = 0; ci < n_cand; ++ci) {
      or_cand* C = &cand[ci];
      double sum = 0.0;
      for (int t = 0; t < n_trk; ++t) {
        if (!tpass[t] || trk[t].idx == C->idx) continue;
        double deta = trk[t].eta - C->eta, dphi = wrap_dphi(trk[t].phi - C->phi);
        double dr2 = deta * deta + dphi * dphi;
        int in1 = decide(d, OR_K_ISO_DR, C->idx, trk[t].idx, 0, OP_LT, dr2, dr2max, 0.0, trk[t].pt);
        int in2 = decide(d, OR_K_ISO_DRMIN, C->idx, trk[t].idx, 0, OP_GE, dr2, dr2min, 0.0, trk[t].pt);
        if (in1 && in2) sum += trk[t].pt;
      }
      for (int t = 0; t < nt; ++t) {
        if (!npass[t] || twr[t].key == cand_key[ci]) continue;
        double deta = twr[t].eta_c - C->eta, dphi = wrap_dphi(twr[t].phi_c - C->phi);
        double dr2 = deta * deta + dphi * dphi;
        int in1 = decide(d, OR_K_ISO_DR, C->idx, twr[t].key, 1, OP_LT, dr2, dr2max, 0.0, twr[t].eflow_et);
        int in2 = decide(d, OR_K_ISO_DRMIN, C->idx, twr[t].key, 1, OP_GE, dr2, dr2min, 0.0, twr[t].eflow_et);
        if (in1 && in2) sum += twr[t].eflow_et;
      }
      C->iso_sum = sum;
      C->iso_rel = sum / C->pt;
      C->isolated = (uint32_t)decide(d, OR_K_ISOLATED, C->idx, 0, 0, OP_LT, C->iso_rel,
                                     c->iso_imax, 0.0, 0.0);
    }
    free(tpass);
  }
  counts->n_trk = n_trk;
  counts->n_twr = nt;
  counts->n_twr_kept = n_kept;
  counts->n_eflow = n_eflow;
  counts->n_cand = n_cand;
  return 0;
}

int oracle_run_event(const oracle_card* c, int64_t n, const float* pt, const float* eta,
                     const float* phi, const float* mass, const int32_t* pdg,
                     const int8_t* charge, const float* vz, uint64_t seed, uint32_t event,
                     double g, const or_flip* flips, int32_t n_flips, or_particle* part,
                     or_track* trk, or_tower* twr, or_cand* cand, or_marginal* marg,
                     int32_t marg_cap, or_counts* counts) {
  if (!c || n < 0 || !counts || (n > 0 && (!pt || !eta || !phi || !mass || !pdg || !charge ||
                                             !part || !trk || !twr || !cand)))
    return -1;
  memset(counts, 0, sizeof *counts);
  or_grid grid[2];
  if (build_grid(c, OR_ECAL, &grid[0]) || build_grid(c, OR_HCAL, &grid[1])) return -1;
  or_dctx d;
  memset(&d, 0, sizeof d);
  d.flips = flips;
  d.nflips = flips ? n_flips : 0;
  d.marg = marg;
  d.cap = marg ? marg_cap : -1;
  d.g = g;
  or_deposit* dep = (or_deposit*)malloc(sizeof(or_deposit) * (size_t)(n + 1));
  uint32_t* cand_key = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  int rc = run_event_impl(c, grid, n, pt, eta, phi, mass, pdg, charge, vz, seed, event, &d,
                          part, trk, twr, cand, dep, cand_key, counts);
  free(dep);
  free(cand_key);
  counts->n_marg = d.nmarg;
  counts->err = d.err;
  if (rc) return rc;
  if (d.err) return d.err;
  if (d.overflow) return -3;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole batch on host threads (the CPU baseline).                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  const oracle_card* c;
  const or_grid* grid;
  int64_t n_events;
  const uint64_t* offsets;
  const float *pt, *eta, *phi, *mass, *vz;
  const int32_t* pdg;
  const int8_t* charge;
  uint64_t seed;
  uint32_t event_base;
  int nthreads, tid;
  uint32_t* counts_out;
  int rc;
} or_job;

static void* batch_worker(void* arg) {
  or_job* J = (or_job*)arg;
  int64_t nmax = 0;
  for (int64_t e = J->tid; e < J->n_events; e += J->nthreads) {
    int64_t n = (int64_t)(J->offsets[e + 1] - J->offsets[e]);
    if (n > nmax) nmax = n;
  }
  size_t cap = (size_t)nmax + 1;
  or_particle* part = (or_particle*)malloc(sizeof(or_particle) * cap);
  or_track* trk = (or_track*)malloc(sizeof(or_track) * cap);
  or_tower* twr = (or_tower*)malloc(sizeof(or_tower) * cap);
  or_cand* cand = (or_cand*)malloc(sizeof(or_cand) * cap);
  or_deposit* dep = (or_deposit*)malloc(sizeof(or_deposit) * cap);
  uint32_t* cand_key = (uint32_t*)malloc(sizeof(uint32_t) * cap);
  if (!part || !trk || !twr || !cand || !dep || !cand_key) J->rc = -4;
  for (int64_t e = J->tid; J->rc == 0 && e < J->n_events; e += J->nthreads) {
    uint64_t a = J->offsets[e], b = J->offsets[e + 1];
    or_dctx d;
    memset(&d, 0, sizeof d);
    d.cap = -1;
    d.g = 0.0;
    or_counts cnt;
    memset(&cnt, 0, sizeof cnt);
    run_event_impl(J->c, J->grid, (int64_t)(b - a), J->pt + a, J->eta + a, J->phi + a,
                   J->mass + a, J->pdg + a, J->charge + a, J->vz ? J->vz + a : NULL, J->seed,
                   J->event_base + (uint32_t)e, &d, part, trk, twr, cand, dep, cand_key, &cnt);
    J->counts_out[e * 4 + 0] = (uint32_t)cnt.n_trk;
    J->counts_out[e * 4 + 1] = (uint32_t)cnt.n_twr_kept;
    J->counts_out[e * 4 + 2] = (uint32_t)cnt.n_eflow;
    J->counts_out[e * 4 + 3] = (uint32_t)cnt.n_cand;
  }
  free(part); free(trk); free(twr); free(cand); free(dep); free(cand_key);
  return NULL;
}

int oracle_run_batch(const oracle_card* c, int64_t n_events, const uint64_t* offsets,
                     const float* pt, const float* eta, const float* phi, const float* mass,
                     const int32_t* pdg, const int8_t* charge, const float* vz,
                     uint64_t seed, uint32_t event_base, int32_t nthreads,
                     uint32_t* counts_out) {
  if (!c || n_events < 0 || !offsets || !counts_out) return -1;
  if (nthreads < 1) nthreads = 1;
  or_grid grid[2];
  if (build_grid(c, OR_ECAL, &grid[0]) || build_grid(c, OR_HCAL, &grid[1])) return -1;
  or_job* jobs = (or_job*)calloc((size_t)nthreads, sizeof(or_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    or_job* J = &jobs[t];
    J->c = c; J->grid = grid; J->n_events = n_events; J->offsets = offsets;
    J->pt = pt; J->eta = eta; J->phi = phi; J->mass = mass; J->vz = vz;
    J->pdg = pdg; J->charge = charge; J->seed = seed; J->event_base = event_base;
    J->nthreads = nthreads; J->tid = t; J->counts_out = counts_out; J->rc = 0;
    pthread_create(&th[t], NULL, batch_worker, J);
  }
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].rc) rc = jobs[t].rc;
  }
  free(jobs);
  free(th);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Pile-up merging (Sec. 2.2; parameters of the pile-up block).  See oracle.h */
/* for the readings: Poisson(mean) interactions by inversion of the CDF on    */
/* integer thresholds, uniform pool events, truncated-Gaussian vertex z and t.*/
/* ------------------------------------------------------------------------ */
int32_t oracle_poisson_thresholds(double mean, uint64_t* T, int32_t kmax) {
  double p = exp(-mean), cdf = p;  /* P(N = 0), P(N <= 0) */
  for (int32_t k = 0; k < kmax; ++k) {
    if (k > 0) {
      p = p * mean / (double)k;  /* P(N = k) = P(N = k-1) mean / k */
      cdf = cdf + p;
    }
    /* the CDF summed in double may stop short of 1: the entry that reaches
     * 2^32 - 1 is the last one and becomes 2^32 (a change below 2^-32) */
    double t = floor(cdf * 4294967296.0);
    if (t >= 4294967295.0) {
      T[k] = 4294967296ull;
      return k + 1;
    }
    T[k] = (uint64_t)t;
  }
  return -1;
}

/* sigma times a standard normal, redrawn until |v| <= bound (decided on the
 * float32 value): a Gaussian truncated at +-bound.  *marg counts decisions
 * within the band g of the bound. */
/* The parity protocol's forced branches of the truncation decisions: a
 * decision (purpose, slot, attempt) listed in fl is taken the other way -
 * only if it is marginal (else *refused is set).  Marginal decisions are
 * recorded as (purpose, slot, attempt) triples in mo (up to mcap of them). */
typedef struct pu_force {
  const uint32_t* fl;
  int32_t nfl;
  uint32_t* mo;
  int32_t mcap;
  int32_t used;   /* forced decisions met */
  int refused;
} pu_force;

static int pu_listed(const pu_force* f, uint32_t purpose, uint32_t slot, uint32_t a) {
  for (int32_t k = 0; f && k < f->nfl; ++k)
    if (f->fl[3 * k] == purpose && f->fl[3 * k + 1] == slot && f->fl[3 * k + 2] == a) return 1;
  return 0;
}

static double truncated_normal(double sigma, double bound, uint64_t seed, uint32_t slot, uint32_t event,
                               uint32_t purpose, double g, int32_t* marg, pu_force* f) {
  for (uint32_t a = 0;; ++a) {
    uint32_t w[4];
    uint32_t ctr[4] = {slot, event, purpose, a};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, w);
    double v = sigma * oracle_normal(w[1], w[2]);
    const int marginal = fabs(fabs(v) - bound) <= g * fmax(fabs(v), bound);
    if (marginal) {
      if (f && *marg < f->mcap) {
        f->mo[3 * *marg] = purpose;
        f->mo[3 * *marg + 1] = slot;
        f->mo[3 * *marg + 2] = a;
      }
      ++*marg;
    }
    int accept = fabsf((float)v) <= (float)bound;
    if (pu_listed(f, purpose, slot, a)) {
      if (!marginal) f->refused = 1;
      accept = !accept;
      ++f->used;
    }
    if (accept) return v;
  }
}

int32_t oracle_pileup_draws(const oracle_pileup* p, const uint64_t* T, int32_t K, uint64_t n_pool,
                            uint64_t seed, uint32_t event, double g, int32_t* n, uint32_t* idx,
                            double* z, double* t, int32_t cap, double* z_hs, double* t_hs) {
  return oracle_pileup_draws_forced(p, T, K, n_pool, seed, event, g, n, idx, z, t, cap, z_hs, t_hs,
                                    NULL, 0, NULL, 0);
}

int32_t oracle_pileup_draws_forced(const oracle_pileup* p, const uint64_t* T, int32_t K, uint64_t n_pool,
                                   uint64_t seed, uint32_t event, double g, int32_t* n, uint32_t* idx,
                                   double* z, double* t, int32_t cap, double* z_hs, double* t_hs,
                                   const uint32_t* flips, int32_t n_flips, uint32_t* marg_out, int32_t marg_cap) {
  int32_t marg = 0;
  pu_force force = {flips, n_flips, marg_out, marg_out ? marg_cap : 0, 0, 0};
  pu_force* f = (flips || marg_out) ? &force : NULL;
  uint32_t w[4];
  draw(seed, 0u, event, 5u, w);
  int32_t N = 0;
  while (N < K - 1 && (uint64_t)w[0] >= T[N]) ++N;  /* smallest N with w0 < T[N] */
  *n = N;
  *z_hs = p->smear_hs ? truncated_normal(p->sigma_z, p->max_z, seed, 0u, event, 5u, g, &marg, f) : 0.0;
  *t_hs = p->smear_hs ? truncated_normal(p->sigma_t, p->max_t, seed, 0u, event, 8u, g, &marg, f) : 0.0;
  if (N > cap) return -1;
  for (int32_t k = 0; k < N; ++k) {
    draw(seed, (uint32_t)k, event, 6u, w);
    idx[k] = (uint32_t)(((uint64_t)w[0] * n_pool) >> 32);
    z[k] = truncated_normal(p->sigma_z, p->max_z, seed, (uint32_t)k, event, 6u, g, &marg, f);
    t[k] = truncated_normal(p->sigma_t, p->max_t, seed, (uint32_t)k, event, 7u, g, &marg, f);
  }
  /* every forced decision must be met, and be marginal */
  if (f && (force.refused || force.used != n_flips)) return -2;
  return marg;
}

/* ------------------------------------------------------------------------ */
/* Track impact parameters (see oracle.h for the readings).                  */
/* ------------------------------------------------------------------------ */
void oracle_track_ip(const oracle_card* c, double pt, double eta, double phi, int32_t q, double x0, double y0,
                     double z0, double* d0, double* zz0, double* s_out) {
  const double cp = cos(phi), sp = sin(phi);
  double s;
  if (c->B == 0.0 || q == 0) {
    /* straight line x = v0 + s p_hat: nearest to the axis at s = -(v0 . p_hat) */
    s = -(x0 * cp + y0 * sp);
    const double px = x0 + s * cp, py = y0 + s * sp;
    *d0 = py * cp - px * sp;
  } else {
    const double h = (q > 0) == (c->B > 0) ? 1.0 : -1.0;
    const double r = pt / (0.299792458 * fabs((double)q * c->B));
    /* centre: to the right of the momentum when the track turns clockwise */
    const double cx = x0 + h * r * sp, cy = y0 - h * r * cp;
    const double dc = hypot(cx, cy);
    /* position angles on the circle (measured at the centre) */
    const double a0 = atan2(y0 - cy, x0 - cx);
    double px, py, ap;
    if (dc == 0.0) {
      px = x0; py = y0; ap = a0;
    } else {
      px = cx - r * cx / dc;
      py = cy - r * cy / dc;
      ap = atan2(py - cy, px - cx);
    }
    /* turning angle from the vertex to the pca, the shorter way */
    double da = ap - a0;
    while (da > M_PI) da -= 2.0 * M_PI;
    while (da <= -M_PI) da += 2.0 * M_PI;
    /* the position angle decreases by h s / r along the motion */
    s = -h * r * da;
    /* momentum direction at the pca: tangent, in the direction of motion */
    const double phip = ap - h * 0.5 * M_PI;
    *d0 = py * cos(phip) - px * sin(phip);
  }
  *zz0 = z0 + s * sinh(eta);
  if (s_out) *s_out = s;
}

void oracle_track_ip_smeared(const oracle_card* c, const oracle_ip_params* ip, double pt, double eta, double phi,
                             int32_t q, double x0, double y0, double z0, uint64_t seed, uint32_t event,
                             uint32_t idx, double out[4]) {
  double d0, zz0;
  oracle_track_ip(c, pt, eta, phi, q, x0, y0, z0, &d0, &zz0, NULL);
  const double sd = sqrt(ip->a_d0 * ip->a_d0 + (ip->b_d0 / pt) * (ip->b_d0 / pt));
  const double sz = sqrt(ip->a_z0 * ip->a_z0 + (ip->b_z0 / pt) * (ip->b_z0 / pt));
  uint32_t w[4];
  draw(seed, idx, event, 9u, w);
  out[0] = d0 + sd * oracle_normal(w[0], w[1]);
  out[1] = zz0 + sz * oracle_normal(w[2], w[3]);
  out[2] = sd;
  out[3] = sz;
}

/* ------------------------------------------------------------------------ */
/* Jet clustering: sequential recombination of the generalized-kT family   */
/* (see oracle.h).  O(n^3): every step scans all active pairs.             */
/* ------------------------------------------------------------------------ */
typedef struct {
  double px, py, pz, e, y, phi, kt2p;
  double nx, ny, nz;      /* unit direction (e+e- distances) */
  double pt0, y0, phi0;   /* the object as loaded (a constituent) */
  int32_t nconst, active, parent;
} cl_obj;

static void cl_derive(cl_obj* o, double p, int32_t ee) {
  const double pt2 = o->px * o->px + o->py * o->py;
  o->phi = atan2(o->py, o->px);
  o->y = 0.5 * log((o->e + o->pz) / (o->e - o->pz));
  const double pm = sqrt(pt2 + o->pz * o->pz);
  o->nx = o->px / pm; o->ny = o->py / pm; o->nz = o->pz / pm;
  /* pp: (pt^2)^p = pt^(2p); e+e-: E^(2p) */
  o->kt2p = ee ? pow(o->e * o->e, p) : pow(pt2, p);
}

static double cl_dphi(double a, double b) {
  double d = a - b;
  while (d > M_PI) d -= 2.0 * M_PI;
  while (d < -M_PI) d += 2.0 * M_PI;
  return d;
}

int32_t oracle_cluster(int64_t n, const double* px, const double* py, const double* pz, const double* e,
                       double p, double R, double pt_min, int32_t nconst_min, int32_t ee, or_jet* jets,
                       int32_t* n_marg) {
  return oracle_cluster_forced(n, px, py, pz, e, p, R, pt_min, nconst_min, ee, jets, n_marg, NULL, 0, NULL, 0);
}

static int cl_listed(const int32_t* v, int32_t nv, int32_t x) {
  for (int32_t k = 0; k < nv; ++k)
    if (v[k] == x) return 1;
  return 0;
}

int32_t oracle_cluster_forced(int64_t n, const double* px, const double* py, const double* pz, const double* e,
                              double p, double R, double pt_min, int32_t nconst_min, int32_t ee, or_jet* jets,
                              int32_t* n_marg, const int32_t* flips, int32_t n_flips, int32_t* marg_steps,
                              int32_t marg_cap) {
  if (n < 0 || !(R > 0.0) || (ee && !(R <= M_PI))) return -1;
  *n_marg = 0;
  if (n == 0) return 0;
  cl_obj* o = (cl_obj*)calloc((size_t)n, sizeof(cl_obj));
  if (!o) return -1;
  for (int64_t i = 0; i < n; ++i) {
    o[i].px = px[i]; o[i].py = py[i]; o[i].pz = pz[i]; o[i].e = e[i];
    o[i].nconst = 1; o[i].active = 1; o[i].parent = -1;
    cl_derive(&o[i], p, ee);
    o[i].pt0 = hypot(px[i], py[i]);
    o[i].y0 = o[i].y;
    o[i].phi0 = o[i].phi;
  }
  int64_t* jet_of = (int64_t*)malloc((size_t)n * sizeof(int64_t)); /* object -> jet slot, or -1 */
  if (!jet_of) { free(o); return -1; }
  for (int64_t i = 0; i < n; ++i) jet_of[i] = -1;
  /* the distance normalisation: R^2, or 2 (1 - cos R) for e+e- (|n_i - n_j|^2 = 2 (1 - cos theta)) */
  const double R2 = ee ? 2.0 * (1.0 - cos(R)) : R * R, eps = 1.0 / 8388608.0; /* 2^-23 */
  int32_t nj = 0;
  int32_t step = 0;
  for (int64_t left = n; left > 0; ++step) {
    /* smallest distance; best / second: value, uncertainty and decision
     * (object i with object j, or with the beam: j = -1) */
    double b = INFINITY, bu = 0.0, s2 = INFINITY, su = 0.0;
    int64_t bi = -1, bj = -1, si = -1, sj = -1;
    for (int64_t i = 0; i < n; ++i) {
      if (!o[i].active) continue;
      const double diB = o[i].kt2p, uiB = 1e-6 * diB;
      /* the beam distance first: it wins ties (the first active object's is
       * taken even when infinite, so that objects whose every distance is
       * infinite - pT = 0 with p < 0 - leave as jets in index order) */
      if (bi < 0 || diB < b) { s2 = b; su = bu; si = bi; sj = bj; b = diB; bu = uiB; bi = i; bj = -1; }
      else if (diB < s2) { s2 = diB; su = uiB; si = i; sj = -1; }
      for (int64_t j = i + 1; j < n; ++j) {
        if (!o[j].active) continue;
        const double kmin = fmin(o[i].kt2p, o[j].kt2p);
        double d, u;
        if (ee) {
          const double ax = o[i].nx - o[j].nx, ay = o[i].ny - o[j].ny, az = o[i].nz - o[j].nz;
          const double dn2 = ax * ax + ay * ay + az * az;
          d = kmin * dn2 / R2;
          u = 1e-6 * d + kmin * 4.0 * sqrt(dn2) * (2.0 * eps) / R2;
        } else {
          const double dy = o[i].y - o[j].y, dp = cl_dphi(o[i].phi, o[j].phi);
          d = kmin * (dy * dy + dp * dp) / R2;
          const double ey = eps * fmax(fmax(fabs(o[i].y), fabs(o[j].y)), 1.0), ep = eps * M_PI;
          u = 1e-6 * d + kmin * (2.0 * fabs(dy) * ey + 2.0 * fabs(dp) * ep) / R2;
        }
        if (d < b) { s2 = b; su = bu; si = bi; sj = bj; b = d; bu = u; bi = i; bj = j; }
        else if (d < s2) { s2 = d; su = u; si = i; sj = j; }
      }
    }
    const int marginal = s2 - b <= bu + su;
    if (marginal) {
      if (*n_marg < marg_cap && marg_steps) marg_steps[*n_marg] = step;
      ++*n_marg;
    }
    if (flips && cl_listed(flips, n_flips, step)) {
      /* take the runner-up decision: only at a marginal step */
      if (!marginal || si < 0) { free(jet_of); free(o); return -2; }
      bi = si;
      bj = sj;
    }
    if (bj < 0) {
      /* i becomes a jet */
      cl_obj* q = &o[bi];
      q->active = 0;
      --left;
      const double pt = hypot(q->px, q->py);
      if (pt >= pt_min && q->nconst >= nconst_min) {
        jet_of[bi] = nj;
        or_jet* J = &jets[nj++];
        J->px = q->px; J->py = q->py; J->pz = q->pz; J->e = q->e;
        J->pt = pt;
        J->eta = asinh(q->pz / pt);
        J->phi = atan2(q->py, q->px);
        const double m2 = q->e * q->e - (q->px * q->px + q->py * q->py + q->pz * q->pz);
        J->mass = m2 > 0.0 ? sqrt(m2) : 0.0;
        J->nconst = q->nconst;
        J->pad = 0;
      }
    } else {
      /* merge j into i (E-scheme) */
      cl_obj* a = &o[bi];
      cl_obj* c = &o[bj];
      a->px += c->px; a->py += c->py; a->pz += c->pz; a->e += c->e;
      a->nconst += c->nconst;
      c->active = 0;
      c->parent = (int32_t)bi; /* j was merged into i */
      --left;
      cl_derive(a, p, ee);
    }
  }
  /* a forced step that never came is refused too */
  for (int32_t k = 0; flips && k < n_flips; ++k)
    if (flips[k] < 0 || flips[k] >= step) { free(jet_of); free(o); return -2; }
  /* substructure: each constituent's jet is the end of its chain of merges */
  for (int32_t k = 0; k < nj; ++k) { jets[k].e2 = jets[k].e3 = jets[k].c2 = jets[k].d2 = 0.0; }
  int64_t* root = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!root) { free(jet_of); free(o); return -1; }
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = i;
    while (o[r].parent >= 0) r = o[r].parent;
    root[i] = jet_of[r];
  }
  for (int32_t k = 0; k < nj; ++k) {
    double spt = 0.0;
    for (int64_t i = 0; i < n; ++i) if (root[i] == k) spt += o[i].pt0;
    double e2 = 0.0, e3 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (root[i] != k) continue;
      for (int64_t j = i + 1; j < n; ++j) {
        if (root[j] != k) continue;
        const double dij = hypot(o[i].y0 - o[j].y0, cl_dphi(o[i].phi0, o[j].phi0));
        e2 += o[i].pt0 * o[j].pt0 / (spt * spt) * dij;
        for (int64_t l = j + 1; l < n; ++l) {
          if (root[l] != k) continue;
          const double dil = hypot(o[i].y0 - o[l].y0, cl_dphi(o[i].phi0, o[l].phi0));
          const double djl = hypot(o[j].y0 - o[l].y0, cl_dphi(o[j].phi0, o[l].phi0));
          e3 += o[i].pt0 * o[j].pt0 * o[l].pt0 / (spt * spt * spt) * dij * dil * djl;
        }
      }
    }
    jets[k].e2 = e2;
    jets[k].e3 = e3;
    jets[k].c2 = e2 > 0.0 ? e3 / (e2 * e2) : 0.0;
    jets[k].d2 = e2 > 0.0 ? e3 / (e2 * e2 * e2) : 0.0;
  }
  free(root);
  free(jet_of);
  free(o);
  /* decreasing pT (insertion sort: stable, small counts) */
  for (int32_t i = 1; i < nj; ++i) {
    or_jet t = jets[i];
    int32_t k = i - 1;
    while (k >= 0 && jets[k].pt < t.pt) { jets[k + 1] = jets[k]; --k; }
    jets[k + 1] = t;
  }
  return nj;
}
