// Track impact parameters of one track (sm_103a; the output table of Sec. 2.5:
// d0, z0 and their errors for charged particles), shared by the standalone
// pass (pdr_track_ip) and the response kernel's fused form (pdr_run_ip), so
// both give the same bits.  The definitions are documented with pdr_track_ip
// in the C header.
//
// The point of closest approach is taken in closed form, arranged so that
// float32 loses nothing to cancellation when the helix radius r (metres to
// kilometres) dwarfs the vertex offset v0 (millimetres).  With phi the
// momentum azimuth at the vertex and h = sign(qB), let
// w = x0 sin(phi) - y0 cos(phi) and u = x0 cos(phi) + y0 sin(phi).  The helix
// centre c lies at v0 + h r (sin phi, -cos phi), so
// |c|^2 = r^2 + 2 h r w + |v0|^2 and
//   d0 = h (r - |c|) = -(2 r w + h |v0|^2) / (r + |c|);
// the turning angle from the vertex to the closest point is the angle between
// the two radii, atan2(h u, r + h w), and the transverse path is
// s = -h r times that angle.  For B = 0 these become d0 = -w and s = -u.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pdr.h"
#include "pdr_internal.h"
#include "pdr_math.cuh"

namespace pdr {

// Track of particle i (index inside its event) of event `event`: generated
// pT, eta, phi, charge q and vertex (x0, y0, zv); Philox counter
// (i, event, 9, 0) under the round keys rk.
__device__ __forceinline__ pdr_ip track_ip_of(float pt, float eta, float phi, int q, float x0, float y0, float zv,
                                              uint32_t i, uint32_t event, const uint32_t* rk, const IPConst& c) {
  float sp, cp;
  sincosf(phi, &sp, &cp);
  const float w = fmaf(x0, sp, -y0 * cp), u = fmaf(x0, cp, y0 * sp);
  float d0, s;
  if (!c.has_field || q == 0) {
    d0 = -w;
    s = -u;
  } else {
    const float h = ((q > 0) == (c.bsign > 0)) ? 1.0f : -1.0f;
    const float r = pt / (c.kB * fabsf((float)q));
    const float v2 = fmaf(x0, x0, y0 * y0);
    const float cc = sqrtf(fmaf(r, r, fmaf(2.0f * h * r, w, v2)));
    d0 = -fmaf(2.0f * r, w, h * v2) / (r + cc);
    s = -h * r * atan2f(h * u, fmaf(h, w, r));
  }
  const float z0 = fmaf(s, sinhf(eta), zv);
  const float ipt = 1.0f / pt;
  const float bd = c.b_d0 * ipt, bz = c.b_z0 * ipt;
  const float sd = sqrtf(fmaf(c.a_d0, c.a_d0, bd * bd)), sz = sqrtf(fmaf(c.a_z0, c.a_z0, bz * bz));
  const uint4 wd = philox(i, event, 9u, 0u, rk);
  return pdr_ip{fmaf(sd, normal(wd.x, wd.y), d0), fmaf(sz, normal(wd.z, wd.w), z0), sd, sz};
}

}  // namespace pdr
