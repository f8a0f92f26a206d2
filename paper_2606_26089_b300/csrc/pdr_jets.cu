// Jet clustering (sm_103a; Sec. 2.4): the generalized-kT family by
// sequential recombination, one warp per event with the event's objects in
// shared memory.  The definitions are documented with pdr_cluster_jets in
// the C header.
//
// Search: the smallest d_ij over all pairs is always reached at a pair whose
// second member is a geometric nearest neighbour (in dR) of the first (if i's
// nearest neighbour m is closer than j, then d_im <= pT_i^2p dR_im^2 / R^2 <
// d_ij whenever pT_i^2p <= pT_j^2p), and a pair at dR >= R never beats the
// beam distance of its member with the smaller pT^2p.  So each object keeps
// its nearest neighbour within R and the distance min(d_iB, d_i,nn); a step
// takes the smallest of those (a warp argmin), merges or makes a jet, and
// re-searches only the objects whose neighbour was involved.
//
// Precision: four-momenta are kept as double (px, py, E + pz, E - pz; in
// global scratch, read and written once a step by one lane); the
// light-cone components are sums of positive terms, so the rapidity
// y = ln((E + pz) / (E - pz)) / 2 of a merged object carries no cancellation
// even far forward.  Distances are float32.
//
// Occupancy: a step is a serial chain of dependent shared-memory accesses, so
// the time follows the number of events (warps) an SM holds, which the
// shared workspace limits.  It holds per object only what the step chain
// reads (24 bytes: y, phi, pT^2p, the distance, and 16-bit neighbour, tile,
// list and work-list entries); an object's neighbour dR^2 is recomputed from
// the two positions when needed (bitwise the value the search found), and the
// constituent counts and merge parents live in global scratch with the
// four-momenta.  A warp takes its next event from a work counter when it
// becomes free, as clustering times vary with the event.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "pdr_internal.h"
#include "pdr_math.cuh"

namespace pdr {

namespace {

// dist holds, besides the distances (non-negative or +inf), these bit
// patterns; as unsigned keys all of them order after every distance
constexpr uint32_t KEY_MERGED = 0xFFFFFFFFu;   // merged away
constexpr uint32_t KEY_JET = 0xFFFFFFFEu;      // a jet (removed with its beam distance)
constexpr uint32_t KEY_TODO = 0xBF800000u;     // (-1.0f) listed for a re-search this step

struct WS {
  // global scratch
  double *px, *py, *ap, *am;
  float *pt0, *y0, *phi0;        // each object as loaded (the jets' constituents)
  int32_t* nc;                   // constituents of each object
  int16_t* parent;               // the object a merged-away object went into, or -1
  // shared
  float *y, *phi, *k2p, *dist;
  float* nz;                     // e+e-: (y, phi, nz) hold the unit direction instead
  int16_t* nn;                   // nearest neighbour within R, or -1
  int16_t *tile, *next, *head;   // tile lists of the active objects
  int16_t* todo;                 // a step's objects to re-search
  int32_t* ntodo;
};

__device__ __forceinline__ WS carve(unsigned char* base, double* mom, uint32_t cap, bool ee, uint32_t ntiles) {
  WS w;
  w.px = mom;
  w.py = mom + cap;
  w.ap = mom + 2 * cap;
  w.am = mom + 3 * cap;
  float* g = reinterpret_cast<float*>(mom + 4 * cap);
  w.pt0 = g;
  w.y0 = g + cap;
  w.phi0 = g + 2 * cap;
  w.nc = reinterpret_cast<int32_t*>(g + 3 * cap);
  w.parent = reinterpret_cast<int16_t*>(w.nc + cap);
  float* f = reinterpret_cast<float*>(base);
  w.y = f;
  w.phi = f + cap;
  w.k2p = f + 2 * cap;
  w.dist = f + 3 * cap;
  w.nz = ee ? f + 4 * cap : nullptr;
  int16_t* h = reinterpret_cast<int16_t*>(f + (ee ? 5 : 4) * cap);
  w.nn = h;
  w.tile = h + cap;
  w.next = h + 2 * cap;
  w.todo = h + 3 * cap;
  w.head = h + 4 * cap;
  w.ntodo = reinterpret_cast<int32_t*>(w.head + ((ntiles + 7u) & ~7u));
  return w;
}

__device__ __forceinline__ float kt2p_of(float pt2, float p) {
  if (p == -1.0f) return 1.0f / pt2;
  if (p == 0.0f) return 1.0f;
  if (p == 1.0f) return pt2;
  return powf(pt2, p);
}

__device__ __forceinline__ float dr2(const WS& w, uint32_t i, float yk, float pk) {
  const float dy = w.y[i] - yk;
  float dp = fabsf(w.phi[i] - pk);
  if (dp > 3.14159265f) dp = 6.28318531f - dp;
  return fmaf(dy, dy, dp * dp);
}

// The pair metric of the clustering: dR^2 in (y, phi), or for e+e-
// |n_i - n_j|^2 = 2 (1 - cos theta) of the unit directions.
__device__ __forceinline__ float metric(const WS& w, bool ee, uint32_t i, float a, float b, float c) {
  if (ee) {
    const float dx = w.y[i] - a, dy = w.phi[i] - b, dz = w.nz[i] - c;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  }
  return dr2(w, i, a, b);
}

__device__ __forceinline__ float dr2_between(float y1, float p1, float y2, float p2) {
  const float dy = y1 - y2;
  float dp = fabsf(p1 - p2);
  if (dp > 3.14159265f) dp = 6.28318531f - dp;
  return fmaf(dy, dy, dp * dp);
}

// min(d_iB, d_i,nn) of an object with beam distance dB, neighbour m (or -1)
// at pair metric r2 (NaN read as +inf, so that every comparison below is a
// total order).
__device__ __forceinline__ float dist_of(const WS& w, float dB, int32_t m, float r2, float inv_R2) {
  float d = dB;
  if (m >= 0) {
    const float dJ = fminf(dB, w.k2p[m]) * r2 * inv_R2;
    d = dJ < dB ? dJ : dB;
  }
  return d <= INFINITY ? d : INFINITY;
}

// ---- tiles: nty x ntp cells in (rapidity, azimuth), each at least R wide,
// so that every object within R of another lies in its cell or an adjacent
// one (rapidity clamped at the ends, azimuth periodic; a single azimuth
// column when 2 pi / R < 3).  A tile is ty << 5 | tp (both < 32).
__device__ __forceinline__ int tile_of(const JetParams& p, float y, float phi) {
  int ty = (int)floorf((y - p.y0) * p.inv_wy);
  ty = min(max(ty, 0), p.nty - 1);
  int tp = (int)floorf((phi + 3.14159265f) * p.inv_wp);
  tp = min(max(tp, 0), p.ntp - 1);
  return (ty << 5) | tp;
}

// The list head of tile t (heads stored densely, nty x ntp).
__device__ __forceinline__ int16_t& head(const JetParams& p, const WS& w, int t) {
  return w.head[(t >> 5) * p.ntp + (t & 31)];
}

// Neighbour l (0..8) of tile t, or -1.
__device__ __forceinline__ int neighbour(const JetParams& p, int t, int l) {
  const int y2 = (t >> 5) + l / 3 - 1, dp = l % 3 - 1;
  if (y2 < 0 || y2 >= p.nty) return -1;
  int tp = t & 31;
  if (p.ntp < 3) return dp == 0 ? (y2 << 5) | tp : -1;
  tp += dp;
  tp = tp < 0 ? tp + p.ntp : (tp >= p.ntp ? tp - p.ntp : tp);
  return (y2 << 5) | tp;
}

__device__ __forceinline__ void push(const JetParams& p, const WS& w, int t, uint32_t k) {
  int16_t& h = head(p, w, t);
  w.next[k] = h;
  h = (int16_t)k;
  w.tile[k] = (int16_t)t;
}

// Unlinks k from its tile list (at most cap steps; a missing k sets the error word).
__device__ __forceinline__ void unlink(const JetParams& p, const WS& w, uint32_t k, uint32_t* err) {
  int16_t& h = head(p, w, w.tile[k]);
  int q = h;
  if (q == (int)k) {
    h = w.next[k];
    return;
  }
  for (uint32_t it = 0; it < p.cap && q >= 0; ++it) {
    const int nx = w.next[q];
    if (nx == (int)k) {
      w.next[q] = w.next[k];
      return;
    }
    q = nx;
  }
  atomicOr(err, ERR_JETS);
}

// Nearest neighbour within R of object k among the active objects of the
// nine surrounding tiles (lanes 0..8 walk one tile each), as (dR^2, index).
__device__ __forceinline__ void search(const JetParams& p, const WS& w, uint32_t k, uint32_t lane, float& best,
                                       int32_t& bi) {
  best = p.R2;
  bi = -1;
  const bool ee = p.ee != 0;
  const float yk = w.y[k], pk = w.phi[k], zk = ee ? w.nz[k] : 0.0f;
  if (lane < 9u) {
    const int t = neighbour(p, w.tile[k], (int)lane);
    if (t >= 0) {
      int q = head(p, w, t);
      for (uint32_t it = 0; it < p.cap && q >= 0; ++it) {
        if (q != (int)k) {
          const float d = metric(w, ee, (uint32_t)q, yk, pk, zk);
          if (d < best || (d == best && q < bi)) { best = d; bi = q; }
        }
        q = w.next[q];
      }
    }
  }
  // (dR^2, index) minimum: non-negative floats order as their bit patterns
  const uint32_t key = bi < 0 ? 0xFFFFFFFFu : __float_as_uint(best);
  const uint32_t mkey = __reduce_min_sync(PDR_FULL, key);
  const uint32_t mi = __reduce_min_sync(PDR_FULL, key == mkey && bi >= 0 ? (uint32_t)bi : 0xFFFFFFFFu);
  bi = mi == 0xFFFFFFFFu ? -1 : (int32_t)mi;
  best = bi < 0 ? p.R2 : __uint_as_float(mkey);
}

// Square root by the PTX approximate instruction (relative error about one
// float32 ulp; the substructure's tolerance is far coarser); sqrt(0) = 0.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The warp's (key, index) minimum over the lanes' candidates (a lane without
// one holds index -1); returns the index, the key in *mkey.
__device__ __forceinline__ int32_t warp_argmin(uint32_t key, int32_t k, uint32_t* mkey) {
  key = k < 0 ? 0xFFFFFFFFu : key;
  *mkey = __reduce_min_sync(PDR_FULL, key);
  const uint32_t mi = __reduce_min_sync(PDR_FULL, key == *mkey && k >= 0 ? (uint32_t)k : 0xFFFFFFFFu);
  return mi == 0xFFFFFFFFu ? -1 : (int32_t)mi;
}

// The current pair metric of object q and its neighbour m (or R^2 without
// one): recomputed from the two positions in the operand order the searches
// use, so it is bitwise the value the search found (neither object has
// moved since, or q would have been re-searched).
__device__ __forceinline__ float nn_metric(const JetParams& p, const WS& w, uint32_t q, int32_t m) {
  if (m < 0) return p.R2;
  const bool ee = p.ee != 0;
  return metric(w, ee, (uint32_t)m, w.y[q], w.phi[q], ee ? w.nz[q] : 0.0f);
}

// Loads the event's objects into the workspace; returns their number.
__device__ __forceinline__ uint32_t load_objects(const JetParams& p, const WS& w, uint64_t a, uint64_t n_part,
                                                 uint32_t c0, uint32_t c2, uint32_t lane) {
  uint32_t n = 0;
  auto put = [&](uint32_t k, float pt, float eta, float phi, float m) {
    float sp, cp;
    sincosf(phi, &sp, &cp);
    const float mt = m > 0.0f ? sqrtf(fmaf(pt, pt, m * m)) : pt;
    const float y = m > 0.0f ? asinhf(pt * sinhf(eta) / mt) : eta;
    w.px[k] = (double)(pt * cp);
    w.py[k] = (double)(pt * sp);
    w.ap[k] = (double)(mt * expf(y));
    w.am[k] = (double)(mt * expf(-y));
    w.y[k] = y;
    w.phi[k] = phi;
    w.pt0[k] = pt;
    w.y0[k] = y;
    w.phi0[k] = phi;
    w.parent[k] = -1;
    w.nc[k] = 1;
    if (p.ee) {
      // unit direction of the momentum and E^2p
      const float ch = coshf(eta), ic = 1.0f / ch;
      w.y[k] = cp * ic;
      w.phi[k] = sp * ic;
      w.nz[k] = tanhf(eta);
      const float pc = pt * ch;
      w.k2p[k] = kt2p_of(fmaf(pc, pc, m * m), p.p);
    } else {
      w.k2p[k] = kt2p_of(pt * pt, p.p);
    }
  };
  if (p.collection == PDR_JETS_PFLOW) {
    n = c0 + c2;
    for (uint32_t k = lane; k < n; k += 32u) {
      if (k < c0) {
        const pdr_track t = p.tracks[a + k];
        const float m = t.idx < n_part ? __ldg(p.mass + a + t.idx) : 0.0f;
        put(k, t.pt, t.eta, t.phi, m);
      } else {
        const pdr_eflow f = p.eflow[a + (k - c0)];
        const uint32_t calo = f.key >> 24, id = f.key & 0x00FFFFFFu;
        float2 c = make_float2(0.0f, 0.0f);
        if (calo <= 1 && id < p.ntowers[calo]) c = __ldg(p.centres + (calo ? p.ntowers[0] : 0u) + id);
        else atomicOr(p.err, ERR_CSR);
        put(k, f.et, c.x, c.y, 0.0f);
      }
    }
  } else {
    // generated particles except neutrinos, compacted in input order
    for (uint64_t b = 0; b < n_part; b += 32u) {
      const uint64_t i = b + lane;
      bool vis = false;
      if (i < n_part) {
        const int32_t id = abs(__ldg(p.pdg + a + i));
        vis = id != 12 && id != 14 && id != 16;
      }
      const uint32_t m = __ballot_sync(PDR_FULL, vis);
      if (vis) {
        const uint32_t k = n + __popc(m & ((1u << lane) - 1u));
        put(k, __ldg(p.pt + a + i), __ldg(p.eta + a + i), __ldg(p.phi + a + i), __ldg(p.mass + a + i));
      }
      n += __popc(m);
    }
  }
  return n;
}

__global__ void __launch_bounds__(512) cluster_kernel(const __grid_constant__ JetParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const uint64_t w0 = (uint64_t)blockIdx.x * p.warps + wib;
  const bool ee = p.ee != 0;
  const WS w = carve(smem + (uint64_t)wib * jet_ws_bytes(p.cap, ee, p.ntiles),
                     p.scratch + w0 * (uint64_t)PDR_JET_SCRATCH_DOUBLES * p.cap, p.cap, ee, p.ntiles);
  const float inv_R2 = p.inv_R2;
  // events are taken from a work counter as warps become free (their
  // clustering times vary), not in a fixed round-robin
  for (;;) {
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(p.next_event, 1u);
    const uint64_t e = __shfl_sync(PDR_FULL, next, 0);
    if (e >= p.n_events) break;
    const uint64_t a = p.offsets[e], b = p.offsets[e + 1];
    uint32_t c0 = 0, c2 = 0;
    if (p.collection == PDR_JETS_PFLOW) {
      c0 = p.counts[4 * e];
      c2 = p.counts[4 * e + 2];
    }
    const uint64_t n_part = b - a;
    const uint64_t n_obj = p.collection == PDR_JETS_PFLOW ? (uint64_t)c0 + c2 : n_part;
    if (!csr_ok(a, b, p.offsets[p.n_events]) || c0 > n_part || c2 > n_part) {
      if (lane == 0 && p.min_obj == 0) {
        atomicOr(p.err, ERR_CSR);
        p.jet_counts[e] = 0;
      }
      continue;
    }
    if (n_obj < p.min_obj || n_obj > p.cap) continue;   // another launch's event
    const uint32_t n = load_objects(p, w, a, n_part, c0, c2, lane);
    for (uint32_t t = lane; t < p.ntiles; t += 32u) w.head[t] = -1;
    __syncwarp();
    if (lane == 0)
      for (uint32_t k = 0; k < n; ++k) push(p, w, tile_of(p, w.y[k], w.phi[k]), k);
    __syncwarp();
    // initial nearest neighbours and distances: each lane walks the cells
    // around its own objects (ties: the lower index, as in the warp search)
    uint32_t bkey = 0xFFFFFFFFu;
    int32_t bk = -1;
    for (uint32_t k = lane; k < n; k += 32u) {
      const float yk = w.y[k], pk = w.phi[k], zk = ee ? w.nz[k] : 0.0f;
      const int tk = w.tile[k];
      float best = p.R2;
      int32_t bi = -1;
      for (int l = 0; l < 9; ++l) {
        const int t = neighbour(p, tk, l);
        if (t < 0) continue;
        int q = head(p, w, t);
        for (uint32_t it = 0; it < p.cap && q >= 0; ++it) {
          if (q != (int)k) {
            const float d = metric(w, ee, (uint32_t)q, yk, pk, zk);
            if (d < best || (d == best && q < bi)) { best = d; bi = q; }
          }
          q = w.next[q];
        }
      }
      w.nn[k] = (int16_t)bi;
      const float d = dist_of(w, w.k2p[k], bi, best, inv_R2);
      w.dist[k] = d;
      if (__float_as_uint(d) < bkey) { bkey = __float_as_uint(d); bk = (int32_t)k; }
    }
    __syncwarp();
    for (uint32_t left = n; left > 0; --left) {
      // the smallest distance (ties: the lower index)
      uint32_t mkey;
      bk = warp_argmin(bkey, bk, &mkey);
      const uint32_t i = (uint32_t)bk;
      const int32_t j = w.nn[i];
      const float dB = w.k2p[i];
      // (d_i,j < d_iB exactly when the distance taken is the pair's)
      const bool merge = j >= 0 && __uint_as_float(mkey) < dB;
      const uint32_t ma = merge ? min(i, (uint32_t)j) : i, mb = merge ? max(i, (uint32_t)j) : i;
      const int ti = w.tile[i], tj = merge ? w.tile[j] : -1;   // cells before the step
      if (lane == 0) *w.ntodo = 0;
      __syncwarp();
      if (lane == 0) {
        if (merge) {
          unlink(p, w, mb, p.err);
          unlink(p, w, ma, p.err);
          const double px = w.px[ma] + w.px[mb], py = w.py[ma] + w.py[mb];
          const double ap = w.ap[ma] + w.ap[mb], am = w.am[ma] + w.am[mb];
          w.px[ma] = px;
          w.py[ma] = py;
          w.ap[ma] = ap;
          w.am[ma] = am;
          w.nc[ma] += w.nc[mb];
          w.parent[mb] = (int16_t)ma;
          w.dist[mb] = __uint_as_float(KEY_MERGED);
          const float fx = (float)px, fy = (float)py;
          if (ee) {
            const double pz = 0.5 * (ap - am), en = 0.5 * (ap + am);
            const float fz = (float)pz;
            const float ip = rsqrtf(fmaf(fx, fx, fmaf(fy, fy, fz * fz)));
            w.y[ma] = fx * ip;
            w.phi[ma] = fy * ip;
            w.nz[ma] = fz * ip;
            const float fe = (float)en;
            w.k2p[ma] = kt2p_of(fe * fe, p.p);
          } else {
            const float ym = 0.5f * logf((float)ap / (float)am), pm = atan2f(fy, fx);
            w.y[ma] = ym;
            w.phi[ma] = pm;
            w.k2p[ma] = kt2p_of(fmaf(fx, fx, fy * fy), p.p);
          }
          push(p, w, tile_of(p, w.y[ma], w.phi[ma]), ma);
        } else {
          unlink(p, w, i, p.err);
          w.dist[i] = __uint_as_float(KEY_JET);
        }
      }
      __syncwarp();
      if (left == 1) break;
      // neighbour records.  Every object's neighbour lies within R of it, so
      // the objects whose neighbour was i or j are in the cells around i's and
      // j's cells, and those the merged object may now be nearest to are in
      // the cells around its new cell: lanes 0-26 walk those 27 cells, listing
      // (once each) the objects to re-search and offering the merged object
      // to the others; then the listed objects are re-searched
      const int ta = w.tile[ma];
      const float ya = w.y[ma], pa = w.phi[ma], za = ee ? w.nz[ma] : 0.0f;
      const int grp = (int)(lane / 9u);
      if (lane < 27u && (grp == 0 || merge)) {
        const int t = neighbour(p, grp == 0 ? ti : (grp == 1 ? tj : ta), (int)(lane - 9u * grp));
        if (t >= 0) {
          int q = head(p, w, t);
          for (uint32_t it = 0; it < p.cap && q >= 0; ++it) {
            const int32_t m = w.nn[q];
            if (m == (int32_t)i || (merge && (m == j || q == (int)ma))) {
              const uint32_t prev = atomicExch(reinterpret_cast<unsigned int*>(w.dist + q), KEY_TODO);
              if (prev != KEY_TODO) w.todo[atomicAdd(w.ntodo, 1)] = (int16_t)q;
            } else if (grp == 2) {
              const float d = metric(w, ee, (uint32_t)q, ya, pa, za);
              if (d < p.R2) {   // (a neighbour record's metric is below R^2, or R^2 without one)
                const float r = nn_metric(p, w, (uint32_t)q, m);
                if (d < r || (d == r && (int32_t)ma < m)) {
                  w.nn[q] = (int16_t)ma;
                  w.dist[q] = dist_of(w, w.k2p[q], (int32_t)ma, d, inv_R2);
                }
              }
            }
            q = w.next[q];
          }
        }
      }
      __syncwarp();
      const int32_t nt = *w.ntodo;
      for (int32_t c = 0; c < nt; ++c) {
        const uint32_t kk = (uint32_t)w.todo[c];
        float best;
        int32_t bi;
        search(p, w, kk, lane, best, bi);
        if (lane == 0) {
          w.nn[kk] = (int16_t)bi;
          w.dist[kk] = dist_of(w, w.k2p[kk], bi, best, inv_R2);
        }
        __syncwarp();
      }
      bkey = 0xFFFFFFFFu;
      bk = -1;
#pragma unroll 4
      for (uint32_t k = lane; k < n; k += 32u) {
        const uint32_t kk = __float_as_uint(w.dist[k]);
        if (kk < bkey) { bkey = kk; bk = (int32_t)k; }
      }
    }
    // jets: the objects removed with their beam distance, cut, ordered by
    // decreasing pT.  The pair arrays are free now: nn holds the jet list,
    // k2p the jets' pT
    uint32_t m = 0;
    for (uint32_t t = 0; t < n; t += 32u) {
      const uint32_t k = t + lane;
      bool keep = false;
      float pt = 0.0f;
      if (k < n && __float_as_uint(w.dist[k]) == KEY_JET) {
        const double px = w.px[k], py = w.py[k];
        pt = (float)sqrt(px * px + py * py);
        keep = pt >= p.pt_min && (uint32_t)w.nc[k] >= p.nconst_min;
      }
      const uint32_t mask = __ballot_sync(PDR_FULL, keep);
      __syncwarp();
      if (keep) {
        const uint32_t slot = m + __popc(mask & ((1u << lane) - 1u));
        w.nn[slot] = (int16_t)k;
        w.k2p[slot] = pt;
      }
      m += __popc(mask);
      __syncwarp();
    }
    __syncwarp();
    // substructure of the kept jets: each object's jet is the end of its chain
    // of merges (the jet list's slot, or -1)
    for (uint32_t k = lane; k < n; k += 32u) {
      w.next[k] = -1;
      w.todo[k] = w.parent[k];   // the merge parents, into shared memory
    }
    __syncwarp();
    for (uint32_t s2 = lane; s2 < m; s2 += 32u) w.next[w.nn[s2]] = (int16_t)s2;
    __syncwarp();
    for (uint32_t k = lane; k < n; k += 32u) {
      int r = (int)k;
      for (uint32_t it = 0; it < n && w.todo[r] >= 0; ++it) r = w.todo[r];
      w.tile[k] = w.next[r];   // the tile array is free now: the object's jet slot
    }
    __syncwarp();
    // the kept jets' records, in decreasing pT (C2 and D2 are added below)
    for (uint32_t s = lane; s < m; s += 32u) {
      const float pts = w.k2p[s];
      uint32_t rank = 0;
      for (uint32_t o = 0; o < m; ++o) {
        const float po = w.k2p[o];
        rank += (po > pts || (po == pts && o < s)) ? 1u : 0u;
      }
      const uint32_t k = (uint32_t)w.nn[s];
      const double px = w.px[k], py = w.py[k], ap = w.ap[k], am = w.am[k];
      const double pt = sqrt(px * px + py * py), pz = 0.5 * (ap - am), en = 0.5 * (ap + am);
      const double m2 = ap * am - pt * pt;
      pdr_jet J;
      J.pt = (float)pt;
      J.eta = (float)asinh(pz / pt);
      J.phi = atan2f((float)py, (float)px);
      J.mass = m2 > 0.0 ? (float)sqrt(m2) : 0.0f;
      J.e = (float)en;
      J.nconst = (uint32_t)w.nc[k];
      J.c2 = 0.0f;
      J.d2 = 0.0f;
      if (rank < n_part) p.jets[a + rank] = J;   // the event's slots hold n_part records
      w.todo[s] = (int16_t)min(rank, 32767u);     // (the parents' copy is free now)
    }
    __syncwarp();
    // then the energy correlation functions e2, e3 (angular exponent 1) over
    // each jet's constituents, staged as (y, phi, pT) in the free y, phi and
    // pT^2p arrays.  Distances in float (relative error ~1e-7; the triples'
    // by the approximate square root), the innermost sums (at most one term a
    // constituent, all positive) in float, the pair terms in double
    float* sy = w.y;
    float* sf = w.phi;
    float* sz = w.k2p;
    for (uint32_t s2 = 0; s2 < m; ++s2) {
      uint32_t c = 0;
      double spt = 0.0;
      for (uint32_t t = 0; t < n; t += 32u) {
        const uint32_t k = t + lane;
        const bool in = k < n && w.tile[k] == (int16_t)s2;
        const uint32_t mask = __ballot_sync(PDR_FULL, in);
        if (in) {
          const uint32_t x = c + __popc(mask & ((1u << lane) - 1u));
          const float z = w.pt0[k];
          sy[x] = w.y0[k];
          sf[x] = w.phi0[k];
          sz[x] = z;
          spt += (double)z;
        }
        c += __popc(mask);
      }
      __syncwarp();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) spt += __shfl_xor_sync(PDR_FULL, spt, o);
      double e2 = 0.0, e3 = 0.0;
      for (uint32_t u = lane; u < c; u += 32u) {
        const float zi = sz[u], yi = sy[u], fi = sf[u];
        for (uint32_t v = u + 1; v < c; ++v) {
          const float zij = zi * sz[v];
          const float yj = sy[v], fj = sf[v];
          const float dij = sqrtf(dr2_between(yi, fi, yj, fj));
          e2 += (double)(zij * dij);
          float s3 = 0.0f;
          for (uint32_t x = v + 1; x < c; ++x) {
            const float yl = sy[x], fl = sf[x];
            s3 = fmaf(sz[x] * sqrt_approx(dr2_between(yi, fi, yl, fl)), sqrt_approx(dr2_between(yj, fj, yl, fl)), s3);
          }
          e3 += (double)(zij * dij) * (double)s3;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_xor_sync(PDR_FULL, e2, o);
        e3 += __shfl_xor_sync(PDR_FULL, e3, o);
      }
      if (lane == 0) {
        const uint32_t rank = (uint32_t)w.todo[s2];
        e2 /= spt * spt;
        e3 /= spt * spt * spt;
        if (rank < n_part) {
          p.jets[a + rank].c2 = e2 > 0.0 ? (float)(e3 / (e2 * e2)) : 0.0f;
          p.jets[a + rank].d2 = e2 > 0.0 ? (float)(e3 / (e2 * e2 * e2)) : 0.0f;
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      if (m > n_part) atomicOr(p.err, ERR_JETS);
      p.jet_counts[e] = (uint32_t)min((uint64_t)m, n_part);
    }
    __syncwarp();
  }
}

// Largest number of clustering objects of an event.
__global__ void jet_max_objects_kernel(JetParams p, uint32_t* out) {
  uint32_t mx = 0;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < p.n_events;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = p.offsets[e], b = p.offsets[e + 1];
    const uint64_t n = csr_ok(a, b, p.offsets[p.n_events]) ? b - a : 0;  // bad ranges are flagged by the clustering
    const uint64_t v = p.collection == PDR_JETS_PFLOW ? (uint64_t)p.counts[4 * e] + p.counts[4 * e + 2] : n;
    mx = max(mx, (uint32_t)min(v, (uint64_t)0xFFFFFFFFu));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(PDR_FULL, mx, o));
  if ((threadIdx.x & 31u) == 0) atomicMax(out, mx);
}

}  // namespace

cudaError_t launch_jet_max_objects(const JetParams& p, uint32_t* out, cudaStream_t s) {
  const uint64_t blocks = p.n_events / 256 + 1;
  jet_max_objects_kernel<<<(unsigned)(blocks < 1184 ? blocks : 1184), 256, 0, s>>>(p, out);
  return cudaGetLastError();
}

// The kernel's dynamic shared-memory limit only ever grows (per device), so
// calls from other threads or contexts never lower it under a launch.
static cudaError_t allow_cluster_smem(size_t smem) {
  static std::mutex mu;
  static int allowed[PDR_MAX_DEVICES] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= PDR_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if ((int)smem <= allowed[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) allowed[dev] = (int)smem;
  return e;
}

cudaError_t occupancy_cluster(uint32_t threads, size_t smem, int* blocks) {
  cudaError_t e = allow_cluster_smem(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, cluster_kernel, (int)threads, smem);
}

cudaError_t launch_cluster(const JetParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
  cudaError_t e = allow_cluster_smem(smem);
  if (e != cudaSuccess) return e;
  cluster_kernel<<<grid, p.warps * 32u, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pdr
