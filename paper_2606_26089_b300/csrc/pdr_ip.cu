// Track impact parameters (sm_103a; the output table of Sec. 2.5: d0, z0 and
// their errors for charged particles).  The definitions are documented with
// pdr_track_ip in the C header.
//
// One warp per event, one lane per track record.  The point of closest
// approach is taken in closed form, arranged so that float32 loses nothing to
// cancellation when the helix radius r (metres to kilometres) dwarfs the
// vertex offset v0 (millimetres).  With phi the momentum azimuth at the
// vertex and h = sign(qB), let w = x0 sin(phi) - y0 cos(phi) and
// u = x0 cos(phi) + y0 sin(phi).  The helix centre c lies at
// v0 + h r (sin phi, -cos phi), so |c|^2 = r^2 + 2 h r w + |v0|^2 and
//   d0 = h (r - |c|) = -(2 r w + h |v0|^2) / (r + |c|);
// the turning angle from the vertex to the closest point is the angle between
// the two radii, atan2(h u, r + h w), and the transverse path is
// s = -h r times that angle.  For B = 0 these become d0 = -w and s = -u.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdr_internal.h"
#include "pdr_math.cuh"

namespace pdr {

namespace {

__global__ void __launch_bounds__(256) track_ip_kernel(const __grid_constant__ IPParams p) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t e = w0; e < p.n_events; e += nw) {
    const uint64_t a = p.offsets[e], b = p.offsets[e + 1];
    const uint32_t nt = p.counts[4 * e];
    if (!csr_ok(a, b, p.offsets[p.n_events]) || nt > b - a) {
      if (lane == 0) atomicOr(p.err, ERR_CSR);
      continue;
    }
    const uint32_t event = p.event_base + (uint32_t)e;
    for (uint32_t k = lane; k < nt; k += 32u) {
      const uint32_t i = p.tracks[a + k].idx;
      if (i >= b - a) {  // not a particle of this event
        atomicOr(p.err, ERR_CSR);
        continue;
      }
      const uint64_t g = a + i;
      const float pt = __ldg(p.pt + g), eta = __ldg(p.eta + g), phi = __ldg(p.phi + g);
      const int q = __ldg(p.charge + g);
      const float x0 = p.vx ? __ldg(p.vx + g) : 0.0f, y0 = p.vy ? __ldg(p.vy + g) : 0.0f;
      const float zv = p.vz ? __ldg(p.vz + g) : 0.0f;
      float sp, cp;
      sincosf(phi, &sp, &cp);
      const float w = fmaf(x0, sp, -y0 * cp), u = fmaf(x0, cp, y0 * sp);
      float d0, s;
      if (!p.has_field || q == 0) {
        d0 = -w;
        s = -u;
      } else {
        const float h = ((q > 0) == (p.bsign > 0)) ? 1.0f : -1.0f;
        const float r = pt / (p.kB * fabsf((float)q));
        const float v2 = fmaf(x0, x0, y0 * y0);
        const float c = sqrtf(fmaf(r, r, fmaf(2.0f * h * r, w, v2)));
        d0 = -fmaf(2.0f * r, w, h * v2) / (r + c);
        s = -h * r * atan2f(h * u, fmaf(h, w, r));
      }
      const float z0 = fmaf(s, sinhf(eta), zv);
      const float ipt = 1.0f / pt;
      const float bd = p.b_d0 * ipt, bz = p.b_z0 * ipt;
      const float sd = sqrtf(fmaf(p.a_d0, p.a_d0, bd * bd)), sz = sqrtf(fmaf(p.a_z0, p.a_z0, bz * bz));
      const uint4 wd = philox(i, event, 9u, 0u, p.rk);
      p.ip[a + k] = pdr_ip{fmaf(sd, normal(wd.x, wd.y), d0), fmaf(sz, normal(wd.z, wd.w), z0), sd, sz};
    }
  }
}

}  // namespace

cudaError_t launch_track_ip(const IPParams& p, int n_sms, cudaStream_t s) {
  const uint64_t blocks = (p.n_events + 7) / 8;
  // one warp an event and no persistent cap: the block scheduler balances
  // events of different sizes (a capped grid left warps with one event more
  // than others)
  const uint64_t cap = (uint64_t)n_sms * 4096;
  track_ip_kernel<<<(unsigned)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap), 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pdr
