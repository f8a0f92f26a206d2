// Post-processing of the detector response (sm_103a; Sec. 2.4): the filter
// pipeline (per-field conditions on a collection, combined with all / any,
// survivors moved down in place) and the event features H_T and missing E_T
// of the PFlow collection (energy-flow tracks and neutrals).  The object
// fields and the definitions of the features are documented with
// pdr_postprocess in the C header.
//
// One warp per event, 32 records at a time (the PFlow tracks and neutrals in
// one index space): each lane evaluates one record's conditions, the warp
// compacts the survivors with a ballot (a record only
// ever moves down, and all lanes hold their record before a warp barrier that
// precedes any move, so the in-place move is safe), and the feature sums are
// exact 64-bit fixed-point integers (quantum 2^-24 GeV), so they do not depend
// on the order of the terms or the launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdr_internal.h"
#include "pdr_math.cuh"

namespace pdr {

namespace {

constexpr float PDR_FEAT_Q = 16777216.0f;   // 2^24 per GeV

// One record's fields (the float ones; pdg and charge separately).
struct Obj {
  float pt, eta, phi, e, et;
  int32_t pdg, q;
};

// Tower centre of a key: one load from the card's table of centres (float32
// of the double ring and phi-bin centres, the values the response uses).
// A key outside the card's towers sets the error word and gives (0, 0).
__device__ __forceinline__ void centre_of(const PostParams& p, uint32_t key, float& eta_c, float& phi_c) {
  const uint32_t calo = key >> 24, id = key & 0x00FFFFFFu;
  if (calo > 1 || id >= p.ntowers[calo]) {
    atomicOr(p.err, ERR_CSR);
    eta_c = phi_c = 0.0f;
    return;
  }
  const float2 c = __ldg(p.centres + (calo ? p.ntowers[0] : 0u) + id);
  eta_c = c.x;
  phi_c = c.y;
}

__device__ __forceinline__ bool cmp_f(uint32_t op, float v, const PostCond& c) {
  switch (op) {
    case PDR_OP_GT: return v > c.fv[0];
    case PDR_OP_GE: return v >= c.fv[0];
    case PDR_OP_LT: return v < c.fv[0];
    case PDR_OP_LE: return v <= c.fv[0];
    case PDR_OP_EQ: return v == c.fv[0];
    case PDR_OP_NE: return v != c.fv[0];
    default: {
      bool in = false;
#pragma unroll
      for (uint32_t k = 0; k < PDR_MAX_VALUES; ++k) in |= k < c.n && v == c.fv[k];
      return op == PDR_OP_IN ? in : !in;
    }
  }
}

__device__ __forceinline__ bool cmp_i(uint32_t op, int32_t v, const PostCond& c) {
  switch (op) {
    case PDR_OP_GT: return v > c.iv[0];
    case PDR_OP_GE: return v >= c.iv[0];
    case PDR_OP_LT: return v < c.iv[0];
    case PDR_OP_LE: return v <= c.iv[0];
    case PDR_OP_EQ: return v == c.iv[0];
    case PDR_OP_NE: return v != c.iv[0];
    default: {
      bool in = false;
#pragma unroll
      for (uint32_t k = 0; k < PDR_MAX_VALUES; ++k) in |= k < c.n && v == c.iv[k];
      return op == PDR_OP_IN ? in : !in;
    }
  }
}

// The filter's verdict on one object (conditions are warp-uniform; the loops
// are unrolled so that every condition field is a constant-bank operand).
__device__ __forceinline__ bool passes(const PostParams& p, const Obj& o) {
  if (p.n_cond == 0) return true;
  bool all = true, any = false;
#pragma unroll
  for (uint32_t k = 0; k < PDR_MAX_CONDITIONS; ++k) {
    if (k >= p.n_cond) break;
    const PostCond& c = p.cond[k];
    bool r;
    if (c.field == PDR_FIELD_PDG || c.field == PDR_FIELD_CHARGE) {
      int32_t v = c.field == PDR_FIELD_PDG ? o.pdg : o.q;
      if (c.abs) v = v < 0 ? -v : v;
      r = cmp_i(c.op, v, c);
    } else {
      float v = c.field == PDR_FIELD_PT ? o.pt : c.field == PDR_FIELD_ETA ? o.eta : c.field == PDR_FIELD_PHI ? o.phi
              : c.field == PDR_FIELD_E ? o.e : o.et;
      if (c.abs) v = fabsf(v);
      r = cmp_f(c.op, v, c);
    }
    all &= r;
    any |= r;
  }
  return p.combine == PDR_COMBINE_ALL ? all : any;
}

// x 2^24 rounded to the nearest integer (|x| < 2^39), with 32-bit conversions
// only (a 64-bit float-to-integer conversion is a slow-pipe instruction): the
// scaled magnitude a = h 2^32 + l is split exactly in float32 (h integral; l
// exact because it holds a subset of a's significant bits), l is rounded, and
// the sign is applied to the integer.
__device__ __forceinline__ long long to_q(float x) {
  const float a = fabsf(x) * PDR_FEAT_Q;
  const float h = truncf(a * 2.3283064365386963e-10f);   // a / 2^32
  const float l = fmaf(-h, 4294967296.0f, a);
  const unsigned long long u = ((unsigned long long)__float2uint_rz(h) << 32) + __float2uint_rn(l);
  return x < 0.0f ? -(long long)u : (long long)u;
}

// A fixed-point sum v (|v| < 2^55) in GeV as float32, with 32-bit conversions
// only (64-bit integer and double conversions run on the FP64 pipe, of which
// B300 has little): v = h 2^32 + l with h the signed high word (exact in
// float32 below 2^24) and l the unsigned low word; relative error below one
// float32 ulp plus 2^7 / |v|.
__device__ __forceinline__ float from_q(long long v) {
  const float h = (float)(int32_t)(v >> 32);
  const float l = __uint2float_rn((uint32_t)(unsigned long long)v);
  return fmaf(h, 4294967296.0f, l) * (1.0f / PDR_FEAT_Q);
}

// Slot of a surviving lane's record among this chunk's survivors.
__device__ __forceinline__ uint32_t rank_in(uint32_t mask, uint32_t lane) {
  return __popc(mask & ((1u << lane) - 1u));
}

// One PFlow object's contribution to H_T and the missing E_T (fixed point).
__device__ __forceinline__ void add_term(float pt, float phi, long long& ht, long long& mx, long long& my) {
  float sn, cs;
  __sincosf(phi, &sn, &cs);   // |phi| <= pi: absolute error below 4e-7
  ht += to_q(pt);
  mx -= to_q(pt * cs);
  my -= to_q(pt * sn);
}

__global__ void __launch_bounds__(256, 5) postprocess_kernel(const __grid_constant__ PostParams p) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const bool f_trk = p.filtered && (p.collection == PDR_COLL_PFLOW || p.collection == PDR_COLL_TRACK);
  const bool f_neu = p.filtered && (p.collection == PDR_COLL_PFLOW || p.collection == PDR_COLL_NEUTRAL);
  const bool f_twr = p.filtered && p.collection == PDR_COLL_TOWER;
  const bool f_cand = p.filtered && p.collection == PDR_COLL_CAND;
  const bool compact = p.filtered && p.compact;
  const bool all_terms = !p.update_features;
  for (uint64_t e = w0; e < p.n_events; e += nw) {
    const uint64_t a = p.offsets[e], n = p.offsets[e + 1] - a;
    const uint32_t c0 = p.counts[4 * e], c1 = p.counts[4 * e + 1], c2 = p.counts[4 * e + 2],
                   c3 = p.counts[4 * e + 3];
    if (!csr_ok(a, p.offsets[e + 1], p.offsets[p.n_events]) || c0 > n || c1 > n || c2 > n || c3 > n) {
      if (lane == 0) atomicOr(p.err, ERR_CSR);
      continue;
    }
    long long ht = 0, mx = 0, my = 0;
    // PFlow objects: tracks [0, c0) then EFlow neutrals [c0, c0 + c2), 32 at a
    // time; the next chunk's records are loaded before this chunk is
    // processed (two chunks in flight per warp).  Lane record r: a track
    // (pt, eta, phi, idx) or a neutral (key, e, et).
    uint32_t wt = 0, wf = 0;
    const uint32_t np = c0 + c2;
    uint4 nxt = make_uint4(0u, 0u, 0u, 0u);
    if (lane < c0) nxt = *reinterpret_cast<const uint4*>(p.tracks + a + lane);
    else if (lane < np) {
      const pdr_eflow& g = p.eflow[a + lane - c0];
      nxt = make_uint4(g.key, __float_as_uint(g.e), __float_as_uint(g.et), 0u);
    }
    for (uint32_t b0 = 0; b0 < np; b0 += 32u) {
      const uint32_t i = b0 + lane;
      const uint4 r = nxt;
      const uint32_t i2 = i + 32u;
      if (i2 < c0) nxt = *reinterpret_cast<const uint4*>(p.tracks + a + i2);
      else if (i2 < np) {
        const pdr_eflow& g = p.eflow[a + i2 - c0];
        nxt = make_uint4(g.key, __float_as_uint(g.e), __float_as_uint(g.et), 0u);
      }
      const bool is_t = i < c0, is_f = !is_t && i < np;
      bool keep_t = false, keep_f = false;
      if (is_t) {
        const float pt = __uint_as_float(r.x), eta = __uint_as_float(r.y), phi = __uint_as_float(r.z);
        keep_t = true;
        if (f_trk) {
          Obj o;
          o.pt = pt; o.eta = eta; o.phi = phi; o.et = pt; o.e = 0.0f; o.pdg = 0; o.q = 0;
          if (p.need_gen) { o.pdg = __ldg(p.pdg + a + r.w); o.q = __ldg(p.charge + a + r.w); }
          if (p.need_mass) {
            const float pc = pt * coshf(eta), m = __ldg(p.mass + a + r.w);
            o.e = sqrtf(fmaf(pc, pc, m * m));
          }
          keep_t = passes(p, o);
        }
        if (keep_t || all_terms) add_term(pt, phi, ht, mx, my);
      } else if (is_f) {
        const float fe = __uint_as_float(r.y), fet = __uint_as_float(r.z);
        float eta_c, phi_c;
        centre_of(p, r.x, eta_c, phi_c);
        keep_f = true;
        if (f_neu) {
          Obj o;
          o.pt = fet; o.eta = eta_c; o.phi = phi_c; o.e = fe; o.et = fet;
          o.pdg = (r.x >> 24) == PDR_ECAL ? 22 : 130; o.q = 0;
          keep_f = passes(p, o);
        }
        if (keep_f || all_terms) add_term(fet, phi_c, ht, mx, my);
      }
      const uint32_t mt = __ballot_sync(PDR_FULL, keep_t), mf = __ballot_sync(PDR_FULL, keep_f);
      if (compact) {
        __syncwarp();  // every lane's reads of this chunk are ordered before the moves
        if (keep_t && f_trk) *reinterpret_cast<uint4*>(p.tracks + a + wt + rank_in(mt, lane)) = r;
        if (keep_f && f_neu)
          p.eflow[a + wf + rank_in(mf, lane)] = pdr_eflow{r.x, __uint_as_float(r.y), __uint_as_float(r.z)};
      }
      wt += __popc(mt);
      wf += __popc(mf);
    }
    // towers and candidates only when they are the target
    uint32_t ww = c1, wc = c3;
    if (f_twr) {
      ww = 0;
      for (uint32_t b0 = 0; b0 < c1; b0 += 32u) {
        const uint32_t i = b0 + lane;
        bool keep = false;
        pdr_tower w;
        if (i < c1) {
          w = p.towers[a + i];
          Obj o;
          centre_of(p, w.key, o.eta, o.phi);
          o.pt = w.et; o.e = w.e; o.et = w.et; o.pdg = 0; o.q = 0;
          keep = passes(p, o);
        }
        const uint32_t m = __ballot_sync(PDR_FULL, keep);
        if (compact) {
          __syncwarp();
          if (keep) p.towers[a + ww + rank_in(m, lane)] = w;
        }
        ww += __popc(m);
      }
    }
    if (f_cand) {
      wc = 0;
      for (uint32_t b0 = 0; b0 < c3; b0 += 32u) {
        const uint32_t i = b0 + lane;
        bool keep = false;
        pdr_cand k;
        pdr_iso s;
        if (i < c3) {
          k = p.cands[a + i];
          s = p.iso[a + i];
          const uint32_t idx = PDR_CAND_IDX(k.info);
          Obj o;
          o.pt = k.pt; o.eta = k.eta; o.phi = k.phi; o.e = k.pt * coshf(k.eta); o.et = k.pt;
          o.pdg = 0; o.q = 0;
          if (p.need_gen) { o.pdg = __ldg(p.pdg + a + idx); o.q = __ldg(p.charge + a + idx); }
          keep = passes(p, o);
        }
        const uint32_t m = __ballot_sync(PDR_FULL, keep);
        if (compact) {
          __syncwarp();
          if (keep) {
            const uint32_t d = wc + rank_in(m, lane);
            p.cands[a + d] = k;
            p.iso[a + d] = s;
          }
        }
        wc += __popc(m);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ht += __shfl_xor_sync(PDR_FULL, ht, o);
      mx += __shfl_xor_sync(PDR_FULL, mx, o);
      my += __shfl_xor_sync(PDR_FULL, my, o);
    }
    if (lane == 0) {
      if (compact) {
        p.counts[4 * e] = f_trk ? wt : c0;
        p.counts[4 * e + 1] = ww;
        p.counts[4 * e + 2] = f_neu ? wf : c2;
        p.counts[4 * e + 3] = wc;
      }
      if (p.features) {
        const float x = from_q(mx), y = from_q(my);
        p.features[e] = pdr_features{from_q(ht), x, y, sqrtf(fmaf(x, x, y * y))};
      }
    }
  }
}

}  // namespace

cudaError_t launch_postprocess(const PostParams& p, int n_sms, cudaStream_t s) {
  const uint64_t warps = p.n_events;
  const uint64_t blocks = (warps + 7) / 8;
  const uint64_t cap = (uint64_t)n_sms * 16;
  postprocess_kernel<<<(unsigned)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap), 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pdr
