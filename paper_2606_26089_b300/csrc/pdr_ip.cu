// Track impact parameters (sm_103a; the output table of Sec. 2.5): the
// standalone pass over pdr_run's track records.  One warp per event, one lane
// per track record; the arithmetic of one track is track_ip_of (pdr_ip.cuh).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdr_internal.h"
#include "pdr_ip.cuh"
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
      p.ip[a + k] = track_ip_of(pt, eta, phi, q, x0, y0, zv, i, event, p.rk, p.c);
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
