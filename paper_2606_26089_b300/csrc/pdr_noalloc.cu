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
// issued.  Under CUDA's default lazy module loading the array's memory is
// committed when the first call resolves its address, so a caller that hands
// the rest of the device memory to its own allocator makes a warm-up call
// (an empty batch) first.  Each call reads the error word back and
// synchronises its stream, so none can be recorded into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pdr.h"
#include "pdr_card.h"
#include "pdr_hot.h"
#include "pdr_internal.h"

namespace pdr {
bool shape_supported(uint32_t team, uint32_t block);
cudaError_t launch_fused(uint32_t team, uint32_t block, const KParams& p, uint32_t grid, size_t smem,
                         cudaStream_t s, bool ip = false);
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
  if ((rc = expand_card(card, g_host_card))) return rc;
  const size_t hot_bytes = build_hot_card(g_host_card, g_host_hot, sizeof g_host_hot);
  if (hot_bytes == 0) return err(PDR_ECARD, "card tables exceed the 40 KiB shared-memory card cache");
  if (cudaMemsetAsync(base, 0, 16, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kCardOffset, &g_host_card, sizeof(DevCard), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kHotOffset, g_host_hot, hot_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return err(PDR_EDEVICE, "cannot stage the card in the static scratch");
  if (b->n_events == 0) return cudaStreamSynchronize(s) == cudaSuccess ? PDR_OK : err(PDR_EDEVICE, "sync");
  uint32_t max_n = b->max_event_size;
  if (max_n == 0) {
    uint32_t words[2] = {0u, 0u};  // error word, largest event (adjacent in the array)
    if (launch_max_event(b->offsets, b->n_events, d_max, d_err, s) != cudaSuccess ||
        cudaMemcpyAsync(words, d_err, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return err(PDR_EDEVICE, "cannot size the batch");
    if (words[0] & ERR_CSR) return err(PDR_EDEVICE, "device error: malformed CSR offsets");
    max_n = words[1];
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
