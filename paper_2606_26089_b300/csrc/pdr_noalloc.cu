// pdr_run_noalloc: the batched detector response without any memory
// allocation by the library.
//
// Who needs this: code that is not allowed to call cudaMalloc (or any other
// device/pinned allocator) at the point where it wants to run the detector
// response - for example a host application that hands all device memory out
// through its own fixed-budget allocator and forbids allocations after start-up,
// or a latency-critical path where an allocation's implicit device-wide
// synchronisation is not acceptable.  Such a caller passes its own input and
// output buffers; everything else the kernel needs (the expanded detector card,
// an error word, and the global-memory tower tables for events too large for
// shared memory) lives in one static device array compiled into the library.
//
// The static array is PDR_NOALLOC_SCRATCH_BYTES (32 MiB) per GPU and every GPU
// that loads the library holds it until the process exits.  All calls share it
// and it keeps whatever the previous call left there: each call rewrites the
// card, clears the error word and re-initialises every tower table it uses
// before use.  Calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race on the array and must not be
// issued.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pdr.h"
#include "pdr_hot.h"
#include "pdr_internal.h"

namespace pdr {
bool shape_supported(uint32_t team, uint32_t block);
cudaError_t launch_fused(uint32_t team, uint32_t block, const KParams& p, uint32_t grid, size_t smem,
                         cudaStream_t s);
cudaError_t occupancy_fused(uint32_t team, uint32_t block, size_t smem, int* blocks);
cudaError_t launch_max_event(const uint64_t* offsets, uint64_t n_events, uint32_t* out, uint32_t* err,
                             cudaStream_t s);
int set_last_error(int code, const char* msg);
}  // namespace pdr

using namespace pdr;

namespace {

// Layout of the static array: [error word, max-event word | card | card cache
// image | tower tables].
constexpr uint64_t kHeaderBytes = 256;
constexpr uint64_t kCardOffset = kHeaderBytes;
constexpr uint64_t kCardBytes = (sizeof(DevCard) + 255) & ~255ull;
constexpr uint64_t kHotOffset = kCardOffset + kCardBytes;
constexpr uint64_t kTableOffset = kHotOffset + PDR_HOT_MAX_BYTES;
static_assert(kTableOffset < PDR_NOALLOC_SCRATCH_BYTES, "scratch too small for the card");

static __device__ __align__(256) unsigned char g_noalloc_scratch[PDR_NOALLOC_SCRATCH_BYTES];

struct DeviceSlot {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int n_sms = 0;
  int smem_optin = 0;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mu;
DevCard g_host_card;  // host staging of the expanded card (static storage, no heap)
unsigned char g_host_hot[PDR_HOT_MAX_BYTES];  // host staging of the card cache image

int err(int code, const char* msg) { return set_last_error(code, msg); }

// One-time set-up per device, with that device current: the static array's
// device address (host code cannot use the symbol's name as an address).
int device_setup(int dev, DeviceSlot*& out) {
  if (dev < 0 || dev >= kMaxDevices) return err(PDR_EINVAL, "device index out of range");
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) return err(PDR_EDEVICE, "cudaGetSymbolAddress of the static scratch failed");
    if (cudaDeviceGetAttribute(&s.n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return err(PDR_EDEVICE, "cannot query the device");
    s.base = (unsigned char*)ptr;
    s.ready = true;
  }
  out = &s;
  return PDR_OK;
}

// ---- detector card expansion into fixed-size storage (same definitions as
// pdr_card_load: ring edges lo + ((hi - lo) k) / n in double, segment ends
// exact; phi edges -pi + (2 pi k) / n_phi; float32 tables).
int expand_calo_fixed(const pdr_card* c, int calo, DevCalo& D, float* pool, int& pool_used) {
  const int nseg = c->nseg[calo];
  if (nseg < 1 || nseg > PDR_MAXSEG) return err(PDR_ECARD, "calorimeter needs 1..4 eta segments");
  double p[PDR_MAXRING / 2 + 1];
  int pn[PDR_MAXRING / 2];
  int m = 0;
  double lo = 0.0;
  p[0] = 0.0;
  std::memset(&D, 0, sizeof D);
  D.nseg = nseg;
  for (int s = 0; s < nseg; ++s) {
    const double hi = c->seg_eta_hi[calo][s];
    const int n = c->seg_neta[calo][s];
    const int nphi = c->seg_nphi[calo][s];
    if (!(hi > lo) || n < 1 || nphi < 1 || nphi > PDR_MAXPHI || m + n > PDR_MAXRING / 2)
      return err(PDR_ECARD, "bad calorimeter segment");
    D.seg_lo[s] = (float)lo;
    D.seg_hi[s] = (float)hi;
    D.seg_scale[s] = (float)(n / (hi - lo));
    D.seg_n[s] = n;
    D.seg_first[s] = m;
    for (int k = 1; k <= n; ++k) {
      p[m + k] = (k == n) ? hi : lo + ((hi - lo) * (double)k) / (double)n;
      pn[m + k - 1] = nphi;
    }
    m += n;
    lo = hi;
  }
  D.nring = 2 * m;
  double edge[PDR_MAXRING + 1];
  int nphi[PDR_MAXRING];
  for (int j = 0; j <= m; ++j) {
    edge[m + j] = p[j];
    edge[m - j] = -p[j];
  }
  edge[m] = 0.0;
  for (int r = 0; r < m; ++r) {
    nphi[m + r] = pn[r];
    nphi[m - 1 - r] = pn[r];
  }
  for (int j = 0; j <= 2 * m; ++j) D.edge[j] = (float)edge[j];
  for (int j = 0; j < 2 * m; ++j)
    if (!(D.edge[j] < D.edge[j + 1])) return err(PDR_ECARD, "eta ring edges not increasing in float32");
  int tab_np[2 * PDR_MAXSEG], tab_off[2 * PDR_MAXSEG], ntab = 0;
  int base = 0;
  for (int r = 0; r < 2 * m; ++r) {
    D.base[r] = base;
    D.nphi[r] = nphi[r];
    base += nphi[r];
    int off = -1;
    for (int t = 0; t < ntab; ++t)
      if (tab_np[t] == nphi[r]) off = tab_off[t];
    if (off < 0) {
      const int np = nphi[r];
      if (pool_used + 2 * np + 1 > PDR_PHIPOOL || ntab >= 2 * PDR_MAXSEG) return err(PDR_ECARD, "phi tables exhausted");
      off = pool_used;
      for (int k = 0; k <= np; ++k)
        pool[off + k] = (float)(k == 0 ? -M_PI : (k == np ? M_PI : -M_PI + (2.0 * M_PI * (double)k) / (double)np));
      for (int k = 0; k < np; ++k) {
        const double e0 = k == 0 ? -M_PI : -M_PI + (2.0 * M_PI * (double)k) / (double)np;
        const double e1 = k + 1 == np ? M_PI : -M_PI + (2.0 * M_PI * (double)(k + 1)) / (double)np;
        pool[off + np + 1 + k] = (float)(0.5 * (e0 + e1));
      }
      pool_used += 2 * np + 1;
      tab_np[ntab] = np;
      tab_off[ntab] = off;
      ++ntab;
    }
    D.phioff[r] = off;
    D.phi_scale[r] = (float)(nphi[r] / (2.0 * M_PI));
    const double ec = 0.5 * (edge[r] + edge[r + 1]);
    D.eta_c[r] = (float)ec;
    D.inv_cosh_c[r] = (float)(1.0 / std::cosh(ec));
  }
  D.ntowers = base;
  // ring groups in ring order: negative-side segments outermost first, then
  // positive-side segments innermost first
  D.ngroup = 2 * nseg;
  for (int s = 0; s < nseg; ++s) {
    const int gn = nseg - 1 - s, gp = nseg + s;
    D.grp_first[gn] = m - D.seg_first[s] - D.seg_n[s];
    D.grp_first[gp] = m + D.seg_first[s];
    D.grp_nphi[gn] = D.grp_nphi[gp] = c->seg_nphi[calo][s];
    D.grp_base[gn] = D.base[D.grp_first[gn]];
    D.grp_base[gp] = D.base[D.grp_first[gp]];
  }
  if (base >= (1 << 24)) return err(PDR_ECARD, "too many towers");
  return PDR_OK;
}

unsigned long long threshold_of(double eff) {
  if (eff >= 1.0) return 4294967296ull;
  if (!(eff > 0.0)) return 0ull;
  return (unsigned long long)std::floor(eff * 4294967296.0);
}

bool rising(const double* v, int n) {
  for (int i = 0; i + 1 < n; ++i)
    if (!((float)v[i] < (float)v[i + 1])) return false;
  return true;
}

int expand_card_fixed(const pdr_card* c, DevCard& D) {
  std::memset(&D, 0, sizeof D);
  if (!(c->R > 0.0) || !(c->L > 0.0) || !std::isfinite(c->B)) return err(PDR_ECARD, "need R > 0, L > 0, finite B");
  int pool_used = 0;
  for (int calo = 0; calo < 2; ++calo) {
    int rc = expand_calo_fixed(c, calo, D.calo[calo], D.phi_pool, pool_used);
    if (rc) return rc;
  }
  D.R = (float)c->R;
  D.L = (float)c->L;
  D.kB = (float)(0.299792458 * std::fabs(c->B));
  D.Bsign = c->B > 0.0 ? 1 : -1;
  D.has_field = c->B != 0.0;
  for (int q = 1; q <= PDR_MAXQ; ++q) {
    const double cR = 0.299792458 * std::fabs((double)q) * std::fabs(c->B) * c->R;
    D.cR_hi[q] = (float)cR;
    D.cR_lo[q] = (float)(cR - (double)D.cR_hi[q]);
  }
  if (c->trk_npt < 1 || c->trk_npt > PDR_MAXEDGE || c->trk_neta < 1 || c->trk_neta > PDR_MAXEDGE ||
      c->id_n < 1 || c->id_n > PDR_MAXEDGE || !rising(c->trk_pt_edges, c->trk_npt) ||
      !rising(c->trk_eta_edges, c->trk_neta) || !rising(c->id_edges, c->id_n))
    return err(PDR_ECARD, "bad efficiency table edges");
  D.trk_npt = c->trk_npt;
  D.trk_neta = c->trk_neta;
  for (int k = 0; k < PDR_MAXEDGE; ++k) {
    D.trk_pt_edges[k] = D.trk_eta_edges[k] = D.id_edges[k] = INFINITY;
    for (int comp = 0; comp < 4; ++comp) D.res_edges[comp][k] = INFINITY;
  }
  for (int k = 0; k < c->trk_npt; ++k) D.trk_pt_edges[k] = (float)c->trk_pt_edges[k];
  for (int k = 0; k < c->trk_neta; ++k) D.trk_eta_edges[k] = (float)c->trk_eta_edges[k];
  for (int t = 0; t < 3; ++t)
    for (int i = 0; i < c->trk_npt; ++i)
      for (int j = 0; j < c->trk_neta; ++j) {
        const double e = c->trk_eff[t][i][j];
        if (!(e >= 0.0 && e <= 1.0)) return err(PDR_ECARD, "tracking efficiency outside [0, 1]");
        D.trk_T[t][i][j] = threshold_of(e);
      }
  D.id_n = c->id_n;
  for (int k = 0; k < c->id_n; ++k) D.id_edges[k] = (float)c->id_edges[k];
  for (int t = 0; t < 3; ++t)
    for (int k = 0; k < c->id_n; ++k) {
      const double e = c->id_eff[t][k];
      if (!(e >= 0.0 && e <= 1.0)) return err(PDR_ECARD, "identification efficiency outside [0, 1]");
      D.id_T[t][k] = threshold_of(e);
    }
  for (int comp = 0; comp < 4; ++comp) {
    const int n = c->res_n[comp];
    if (n < 1 || n > PDR_MAXEDGE || !rising(c->res_edges[comp], n)) return err(PDR_ECARD, "bad resolution table");
    D.res_n[comp] = n;
    for (int k = 0; k < n; ++k) {
      D.res_edges[comp][k] = (float)c->res_edges[comp][k];
      const double a = c->res_abcd[comp][k][0], b = c->res_abcd[comp][k][1];
      const double cc = c->res_abcd[comp][k][2], d = c->res_abcd[comp][k][3];
      if (!(a >= 0 && b >= 0 && cc >= 0 && d >= 0)) return err(PDR_ECARD, "negative resolution coefficient");
      D.res_a2[comp][k] = (float)(a * a);
      D.res_b2[comp][k] = (float)(b * b);
      D.res_c2[comp][k] = (float)(cc * cc);
      D.res_d2[comp][k] = (float)(d * d);
    }
  }
  for (int calo = 0; calo < 2; ++calo) {
    DevCalo& C = D.calo[calo];
    const int comp = calo == 0 ? RES_ECAL : RES_HCAL;
    for (int r = 0; r < C.nring; ++r) {
      int k = -1;
      for (int j = 0; j < c->res_n[comp]; ++j)
        if ((float)c->res_edges[comp][j] <= std::fabs(C.eta_c[r])) k = j;
      C.resbin[r] = k < 0 ? 0 : k;
    }
    D.e_min[calo] = (float)c->e_min[calo];
    D.s_min[calo] = (float)c->s_min[calo];
  }
  D.cand_ptmin = (float)c->cand_ptmin;
  D.dr2max = (float)(c->iso_dr * c->iso_dr);
  D.dr2min = (float)(c->iso_drmin * c->iso_drmin);
  D.iso_ptmin = (float)c->iso_ptmin;
  D.imax = (float)c->iso_imax;
  return PDR_OK;
}

// Tower-table slots for events up to max_n particles: at least 4/3 max_n,
// a multiple of 32 (at most 3/4 of the slots are ever in use).
uint32_t slots_at_least(uint32_t max_n) {
  return std::max<uint32_t>(64, (uint32_t)((((uint64_t)max_n * 4 + 2) / 3 + 31) & ~31ull));
}

}  // namespace

extern "C" int pdr_run_noalloc(const pdr_card* card, const pdr_batch* b, const pdr_outputs* o, void* stream) {
  if (!card || !b || !o) return err(PDR_EINVAL, "null argument");
  if (b->n_events >= (1ull << 31)) return err(PDR_EINVAL, "n_events must be < 2^31");
  if (b->n_events > 0 && (!b->offsets || !b->pt || !b->eta || !b->phi || !b->mass || !b->pdg || !b->charge))
    return err(PDR_EINVAL, "null input array");
  if (!o->tracks || !o->towers || !o->eflow || !o->cands || !o->iso || !o->counts)
    return err(PDR_EINVAL, "null output buffer");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return err(PDR_EDEVICE, "no current CUDA device");
  std::lock_guard<std::mutex> g(g_mu);
  DeviceSlot* slot = nullptr;
  int rc = device_setup(dev, slot);
  if (rc) return rc;
  unsigned char* base = slot->base;
  uint32_t* d_err = (uint32_t*)base;
  uint32_t* d_max = d_err + 1;
  if ((rc = expand_card_fixed(card, g_host_card))) return rc;
  const size_t hot_bytes = build_hot_card(g_host_card, g_host_hot, sizeof g_host_hot);
  if (hot_bytes == 0) return err(PDR_ECARD, "card tables exceed the 40 KiB shared-memory card cache");
  if (cudaMemsetAsync(base, 0, 16, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kCardOffset, &g_host_card, sizeof(DevCard), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kHotOffset, g_host_hot, hot_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return err(PDR_EDEVICE, "cannot stage the card in the static scratch");
  if (b->n_events == 0) return cudaStreamSynchronize(s) == cudaSuccess ? PDR_OK : err(PDR_EDEVICE, "sync");
  uint32_t max_n = b->max_event_size;
  if (max_n == 0) {
    if (launch_max_event(b->offsets, b->n_events, d_max, d_err, s) != cudaSuccess ||
        cudaMemcpyAsync(&max_n, d_max, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return err(PDR_EDEVICE, "cannot size the batch");
  }
  if (max_n > 49152) return err(PDR_EOVERFLOW, "pdr_run_noalloc: an event has more than 49152 particles");
  // launch shape by event size (as pdr_run's default)
  uint32_t team, block;
  if (max_n <= 128) { team = 32; block = 256; }
  else if (max_n <= 640) { team = 128; block = 256; }
  else if (max_n <= 1500) { team = 256; block = 256; }
  else if (max_n <= 3000) { team = 512; block = 512; }
  else { team = 1024; block = 1024; }
  const uint32_t nt = block / team;
  uint32_t slots = slots_at_least(max_n);
  while (slots > 64 && hot_bytes + nt * team_smem_bytes(team, slots, slots * 3 / 4) > (uint64_t)slot->smem_optin)
    slots = std::max<uint32_t>(64, (slots / 2) & ~31u);
  const size_t smem = (size_t)(hot_bytes + nt * team_smem_bytes(team, slots, slots * 3 / 4));
  int per_sm = 0;
  if (occupancy_fused(team, block, smem, &per_sm) != cudaSuccess || per_sm < 1)
    return err(PDR_EDEVICE, "launch shape cannot be resident");
  uint32_t grid = (uint32_t)(per_sm * slot->n_sms);
  static KParams p;  // 5 KB parameter block: static storage (calls are serialised by g_mu)
  std::memset(&p, 0, sizeof p);
  p.n_cards = 1;
  p.hot[0] = base + kHotOffset;
  p.hot_bytes[0] = (uint32_t)hot_bytes;
  p.hot_off[0] = 0;
  p.hot_total = (uint32_t)hot_bytes;
  p.n_segs = 1;
  p.n_events = b->n_events;
  KSeg& sg = p.seg[0];
  sg.event_start = 0;
  sg.n_events = b->n_events;
  sg.offsets = b->offsets;
  sg.pt = b->pt; sg.eta = b->eta; sg.phi = b->phi; sg.mass = b->mass; sg.vz = b->vz;
  sg.pdg = b->pdg; sg.charge = b->charge;
  set_round_keys(sg, b->seed);
  sg.event_base = b->event_index_base;
  sg.card = 0;
  sg.tracks = o->tracks; sg.towers = o->towers; sg.eflow = o->eflow; sg.cands = o->cands;
  sg.iso = o->iso; sg.counts = o->counts;
  sg.debug = (b->flags & PDR_BATCH_DEBUG) ? o->debug : nullptr;
  p.table_slots = slots;
  p.nmax_smem = slots * 3 / 4;
  p.err = d_err;
  if (max_n > p.nmax_smem) {
    // global tower tables in the static array; fewer teams if they do not fit
    const uint32_t gs = slots_at_least(max_n);
    p.g_slots = gs;
    p.g_nmax = gs * 3 / 4;
    p.g_team_bytes = global_team_bytes(gs, p.g_nmax);
    const uint64_t room = PDR_NOALLOC_SCRATCH_BYTES - kTableOffset;
    const uint64_t fit_ctas = room / (p.g_team_bytes * nt);
    if (fit_ctas < 1)
      return err(PDR_EOVERFLOW, "pdr_run_noalloc: the largest event needs more tower-table scratch than the "
                                "static 32 MiB array holds");
    if (grid > fit_ctas) grid = (uint32_t)fit_ctas;
    p.gscratch = base + kTableOffset;
  }
  if (launch_fused(team, block, p, grid, smem, s) != cudaSuccess) return err(PDR_EDEVICE, "kernel launch failed");
  uint32_t h_err = 0;
  if (cudaMemcpyAsync(&h_err, d_err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return err(PDR_EDEVICE, "kernel failed");
  if (h_err) return err(PDR_EDEVICE, (h_err & ERR_CSR) ? "device error: malformed CSR offsets"
                                                      : "device error: event too large or tower table full");
  return PDR_OK;
}
