// Float-float ("double-word") arithmetic for the one quantity of the response
// whose float32 rounding the method amplifies without bound: the endcap
// turning angle psi of a helix that has nearly closed (psi -> 2 pi), where
// the transverse distance rho = 2 r sin(psi / 2) at the endcap, and with it
// the surface pseudorapidity, depends on pi - psi / 2 (the helix
// propagation of Sec. 2.2 / App. D.1).  A value is the unevaluated sum
// hi + lo of two float32.  Error-free transformations: TwoSum (Knuth),
// FastTwoSum (Dekker; needs |a| >= |b| or a = 0) and TwoProduct through the
// fused multiply-add.
#pragma once

#include "pdr_math.cuh"

namespace pdr {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

// 2^(j/32), j = 0..31, each as float32 hi + float32 lo (ff_tables.py beside
// this file computes them in 60-digit decimal arithmetic; |hi + lo - 2^(j/32)|
// below 1.5e-15 relative).
static __constant__ float2 kExp2Tab[32] = {
    {1.0f, 0.0f},                    {1.0218972f, -4.81156e-08f},     {1.0442737f, 4.83347e-08f},
    {1.0671405f, -5.933752e-08f},    {1.0905077f, -1.307754e-08f},    {1.1143868f, -5.43554e-08f},
    {1.1387886f, 5.3862223e-08f},    {1.1637249f, -4.0514415e-08f},   {1.1892071f, 3.7976353e-08f},
    {1.2152474f, -3.267395e-08f},    {1.2418578f, 4.496838e-08f},     {1.269051f, 1.4193333e-09f},
    {1.2968396f, -4.0189995e-08f},   {1.3252367f, -3.4963733e-08f},   {1.3542556f, -1.0123349e-08f},
    {1.38391f, -5.8755774e-08f},     {1.4142135f, 2.4203235e-08f},    {1.4451808f, 3.3242e-08f},
    {1.4768262f, -4.500899e-08f},    {1.5091645f, -2.4959373e-08f},   {1.5422108f, 8.070905e-09f},
    {1.5759809f, -5.6610254e-08f},   {1.6104903f, 9.836217e-09f},     {1.6457555f, -5.124972e-08f},
    {1.6817929f, -2.4755327e-08f},   {1.7186193f, -4.8496176e-08f},   {1.7562522f, -9.23577e-09f},
    {1.7947091f, -1.1415045e-08f},   {1.8340081f, -1.1239278e-08f},   {1.8741677f, -4.6630056e-08f},
    {1.9152066f, 9.845328e-09f},     {1.9571441f, -1.7021804e-08f},
};

// e^a for 0 <= a <= 88 by Tang's table-driven method (ACM TOMS 15(2), 1989)
// with 32 entries: n = rint(32 a / ln2), r = a - n ln2/32 with ln2/32 split
// into C1 + C2 + C3 (C1 has 12 significant bits, so n C1 is exact for
// n < 4096 and a - n C1 is exact by Sterbenz's lemma), |r| <= 0.01084, and
// e^r = 1 + r + r^2/2 + r^3 (1/6 + r/24 + r^2/120) (truncation below 2.2e-15
// relative) with r^2 exact through TwoProduct and the cubic tail, below
// 2.2e-7, in float32; then e^a = 2^(n div 32) 2^((n mod 32)/32) e^r.
// Relative error of hi + lo below 2^-42.
__device__ __forceinline__ ff exp_ff(float a) {
  const float nf = rintf(a * 46.16624f);
  const int n = (int)nf;
  const float rh = fmaf(-nf, 0.021659851f, a);
  const ff p = two_prod(nf, 9.983182e-07f);
  const ff s = two_sum(rh, -p.hi);
  const float r = s.hi;
  const float rl = fmaf(-nf, 5.1456093e-14f, s.lo - p.lo);
  const ff q = two_prod(r, r);
  const float tail = r * q.hi * fmaf(r, fmaf(r, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f);
  const ff u = two_sum(r, 0.5f * q.hi);
  const ff h = fast_two_sum(1.0f, u.hi);
  // e^(r + rl) = e^r (1 + rl): the rl^2 term is below 2^-90
  const float lo = fmaf(h.hi, rl, ((h.lo + u.lo) + fmaf(0.5f, q.lo, tail)));
  const ff er = fast_two_sum(h.hi, lo);
  const float2 T = kExp2Tab[n & 31];
  const float m = T.x * er.hi;
  const float ml = fmaf(T.x, er.hi, -m) + fmaf(T.x, er.lo, T.y * er.hi);
  const ff e = fast_two_sum(m, ml);
  const float scale = __int_as_float((127 + (n >> 5)) << 23);
  return {e.hi * scale, e.lo * scale};
}

// sinh(a) for a >= 0 (arguments above 88 are taken as 88).  Below 1/64 the
// odd series a + a w, w = a^2 (1/6 + a^2/120 + a^4/5040) (truncation below
// 2e-21 relative; w < 4.1e-5 in float32, so its rounding is below 2^-37 of
// the result); above, (E - 1/E) / 2 with E = exp_ff(a) and 1/E from the
// hardware reciprocal and one correction (error below 2^-43), where the
// cancellation multiplies E's error by coth(a) <= 64.  Relative error of
// hi + lo below 2^-36 on [0, 88] and below 2^-41 from 1/4 up.
__device__ __forceinline__ ff sinh_ff(float a) {
  if (a < 0.015625f) {
    const float a2 = a * a;
    const float w = a2 * fmaf(a2, fmaf(a2, 1.0f / 5040.0f, 1.0f / 120.0f), 1.0f / 6.0f);
    const ff p = two_prod(a, w);
    const ff s = fast_two_sum(a, p.hi);
    return fast_two_sum(s.hi, s.lo + p.lo);
  }
  const ff e = exp_ff(fminf(a, 88.0f));
  const float i0 = rcp_approx(e.hi);
  const float il = i0 * (fmaf(-e.hi, i0, 1.0f) - e.lo * i0);
  const ff d = two_sum(e.hi, -i0);
  const ff s = fast_two_sum(d.hi, d.lo + (e.lo - il));
  return {0.5f * s.hi, 0.5f * s.lo};
}

// pi - psi/2 for the endcap helix, psi = s_z / r = (z_e - vz) kq / (pT sinh(eta))
// with z_e = sign(eta) L, taken as (L - sign(eta) vz) kq / (pT sinh|eta|), all
// in float-float from the float32 inputs, the card's L = L_hi + L_lo and
// kB = 0.299792458 |B| = kB_hi + kB_lo, and kq = kB |q|.  The quotient is a
// float32 estimate corrected once by its float-float remainder.  For
// psi / 2 >= pi / 2 (the caller's range) pi - psi_hi / 2 is exact by
// Sterbenz's lemma, so the result's absolute error is about pi times the
// relative error of psi (2^-36, 2^-41 for |eta| >= 1/4) plus its own float32
// rounding: relative error below 2^-24 + 2^-34 / (pi - psi/2) (2^-24 +
// 2^-39 / (pi - psi/2) for |eta| >= 1/4).
__device__ __forceinline__ float half_turn_gap(float pt, float eta, float vz, int aq, float L_hi, float L_lo,
                                               float kB_hi, float kB_lo) {
  const ff S = sinh_ff(fabsf(eta));
  const ff n0 = two_sum(L_hi, eta > 0.0f ? -vz : vz);
  const float nl = n0.lo + L_lo;
  const float qf = (float)aq;
  const ff k = two_prod(kB_hi, qf);
  const float kl = fmaf(kB_lo, qf, k.lo);
  const ff u = two_prod(n0.hi, k.hi);
  const float ul = fmaf(n0.hi, kl, fmaf(nl, k.hi, u.lo));
  const ff d = two_prod(pt, S.hi);
  const float dl = fmaf(pt, S.lo, d.lo);
  const float id = rcp_approx(d.hi);
  const float q1 = u.hi * id;
  const float rem = fmaf(-q1, dl, fmaf(-q1, d.hi, u.hi) + ul);
  const float q2 = rem * id;
  // pi = 3.14159274101257324 - 8.74227766e-8 (both float32; remainder ~1e-15)
  return (3.14159274101257324f - 0.5f * q1) + (-8.74227766e-8f - 0.5f * q2);
}

// The same, out of line (a call keeps the rarely taken code out of a hot loop).
static __device__ __noinline__ float half_turn_gap_call(float pt, float eta, float vz, int aq, float L_hi,
                                                        float L_lo, float kB_hi, float kB_lo) {
  return half_turn_gap(pt, eta, vz, aq, L_hi, L_lo, kB_hi, kB_lo);
}

}  // namespace pdr
