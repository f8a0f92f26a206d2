// Device arithmetic shared by the detector-response kernel and the pile-up
// merge kernels (sm_103a): the counter-based Philox4x32-10 generator, uniform
// and normal deviates, and the single-precision function approximations the
// kernels use in place of the library calls (each with its error bound).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdr {

#define PDR_FULL 0xFFFFFFFFu

static constexpr float PI_F = 3.14159265358979323846f;
static constexpr float TWO_PI_F = 6.28318530717958647692f;
static constexpr float PIO2_HI = 1.57079637050628662109375f;  // float32(pi/2)
static constexpr float PIO2_LO = -4.37113900018624283e-8f;     // pi/2 - PIO2_HI

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten multiply/xor rounds on a 128-bit
// counter under a 64-bit key bumped by the Weyl constants each round.  The
// round keys of the batch's seed are precomputed (KSeg::rk), so a round is two
// 32 x 32 -> 64-bit products and two three-way xors.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = 0xD2511F53ull * c0;
    const unsigned long long p1 = 0xCD9E8D57ull * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk[2 * r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk[2 * r + 1];
    c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Reciprocal to 1 ulp (the hardware approximation, 1 ulp at most by the PTX
// ISA: relative error below 2^-23 over 1e-20 ... 1e20); used where the result
// only needs a few ulp:
// every such quotient feeds either an output compared at 2e-6 relative or a
// decision taken with the 1e-5 marginal band.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float fdiv(float a, float b) { return a * rcp_approx(b); }

// Square root to 1 ulp (the hardware approximation; relative error below
// 2^-22 over 1e-20 ... 1e20): energies, smearing widths and the Box-Muller
// radius need only a few ulp.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Polynomial approximations.  Coefficients: least-squares polynomial fits in
// double precision of the reduced function in its reduced variable, sampled
// at the 64 Chebyshev points of the first kind of the interval, rounded to
// float32 (fit_poly.py beside this file computes them; the relative error of
// each fit before float32 evaluation is given in brackets):
//   asin(x) = x + x^3 P(x^2), P on x^2 in [0, 1/4]      (2.5e-9)
//   sin(x)  = x + x^3 Q(x^2), Q on x^2 in [0, pi^2/4]   (1.9e-8)
//   ln(1 - v) = -v L(v),      L on v in [0, 1/4]        (4.6e-9)
//   ln(1 + x) = x M(x),       M on x in [0, 1/4]        (3.0e-9)
// Each function below states its float32 error bound over its whole argument
// range; a GPU test (through pdr_math_eval) holds it to that bound, at every
// one of the 2^23 uniforms for the Box-Muller pieces and on dense grids for
// the others.
__device__ __forceinline__ float asin_half(float x) {
  const float t = x * x;
  float p = fmaf(t, 0.033805776f, 0.01707784f);
  p = fmaf(t, p, 0.031116161f);
  p = fmaf(t, p, 0.04459803f);
  p = fmaf(t, p, 0.07500099f);
  p = fmaf(t, p, 0.16666666f);
  return fmaf(x * t, p, x);
}

__device__ __forceinline__ float sin_quarter(float x) {
  const float t = x * x;
  float q = fmaf(t, -2.4080485e-08f, 2.7536478e-06f);
  q = fmaf(t, q, -0.00019841087f);
  q = fmaf(t, q, 0.008333333f);
  q = fmaf(t, q, -0.16666667f);
  return fmaf(x * t, q, x);
}

// asin_half: relative error below 2.4e-7 on [0, 1/2].
// sin_half_turn: sin on [0, pi], reflected to [0, pi/2] with pi split in two
// floats; absolute error below 1.8e-7.
__device__ __forceinline__ float sin_half_turn(float y) {
  return sin_quarter(y > PIO2_HI ? (3.14159274101257324f - y) + -8.74227766e-8f : y);
}

// ln u for u in (0, 1): hardware log2 below 3/4 (|ln u| > 0.28 there),
// -v L(v) with v = 1 - u (exact) above; relative error below 6e-7 at every
// uniform the generator makes.
__device__ __forceinline__ float ln_unit(float u) {
  const float v = 1.0f - u;
  float p = fmaf(v, 0.33390906f, 0.08952039f);
  p = fmaf(v, p, 0.21425246f);
  p = fmaf(v, p, 0.24869019f);
  p = fmaf(v, p, 0.33338976f);
  p = fmaf(v, p, 0.4999991f);
  p = fmaf(v, p, 1.0f);
  return u > 0.75f ? -v * p : __logf(u);
}

// ln(1 + x) for x >= 0: x M(x) up to 1/4, hardware log2 of 1 + x above
// (ln(1 + x) > 0.22 there); relative error below 6e-7 up to 1e8.
__device__ __forceinline__ float log1p_pos(float x) {
  float m = fmaf(x, 0.070751615f, -0.14544724f);
  m = fmaf(x, m, 0.19665538f);
  m = fmaf(x, m, -0.24972063f);
  m = fmaf(x, m, 0.33332205f);
  m = fmaf(x, m, -0.49999982f);
  m = fmaf(x, m, 1.0f);
  return x > 0.25f ? __logf(1.0f + x) : x * m;
}

// cos(2 pi u) for u in (0, 1): folded exactly in turns to sin of at most a
// quarter turn (cos(2 pi u) = -cos(pi t), t = |2u - 1|); absolute error below
// 2.4e-7 at every uniform the generator makes.
__device__ __forceinline__ float cos_two_pi(float u) {
  const float t = fabsf(2.0f * u - 1.0f);
  const float r = t > 0.5f ? t - 0.5f : 0.5f - t;
  const float s = sin_quarter(PI_F * r);
  return t > 0.5f ? s : -s;
}

// cosh and sinh from one exponential: cosh = (e + 1/e) / 2; sinh likewise for
// |x| >= 1/2 (no cancellation there: e - 1/e >= 1.04) and from its odd Taylor
// series through x^9 below 1/2 (truncation < 3e-11 relative); relative error
// of both below 4e-7 on [-12, 12].
__device__ __forceinline__ void cosh_sinh(float x, float& ch, float& sh) {
  const float ax = fabsf(x);
  const float e = expf(ax);
  const float ie = rcp_approx(e);
  ch = 0.5f * (e + ie);
  const float x2 = ax * ax;
  const float series =
      ax * fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 362880.0f, 1.0f / 5040.0f), 1.0f / 120.0f), 1.0f / 6.0f),
                1.0f);
  const float s = ax < 0.5f ? series : 0.5f * (e - ie);
  sh = copysignf(s, x);
}

// asinh(u) = sign(u) log(|u| + sqrt(u^2 + 1)) with the hardware log2 (the
// argument of the log is >= 1, so no cancellation): error below
// 2.5e-7 max(|asinh u|, 1) up to |u| = 1e7.  Used for the surface
// pseudorapidity, whose tolerance is 2e-6 max(|eta|, 1).
__device__ __forceinline__ float asinh_fast(float u) {
  const float au = fabsf(u);
  return copysignf(__logf(au + sqrt_approx(fmaf(au, au, 1.0f))), u);
}

// (2k + 1) / 2^24 for the top 23 bits k of w: exact in float32.
__device__ __forceinline__ float u01(uint32_t w) {
  return (__uint2float_rn(w >> 9) + 0.5f) * 1.1920928955078125e-7f;
}

// Box-Muller, cosine branch: at every value of either word (the other fixed
// at several values) the deviate is within 1e-6 absolute of its FP64 value.
__device__ __forceinline__ float normal(uint32_t wa, uint32_t wb) {
  return sqrt_approx(-2.0f * ln_unit(u01(wa))) * cos_two_pi(u01(wb));
}

}  // namespace pdr
