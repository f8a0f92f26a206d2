// Host runtime of the CUDA library behind include/pdr.h: contexts, detector
// cards, launch shapes and autotuning, scratch and the result pool, the
// batched / per-event / host-buffer entry points and tickets.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pdr.h"
#include "pdr_card.h"
#include "pdr_hot.h"
#include "pdr_internal.h"

namespace pdr {
bool shape_supported(uint32_t team, uint32_t block);
cudaError_t launch_fused(uint32_t team, uint32_t block, const KParams& p, uint32_t grid, size_t smem,
                         cudaStream_t s, bool ip = false);
cudaError_t occupancy_fused(uint32_t team, uint32_t block, size_t smem, int* blocks);
cudaError_t occupancy_fused_ovf(uint32_t team, uint32_t block, size_t smem, int* blocks);
bool shape_supports_overflow(uint32_t team, uint32_t block);
cudaError_t launch_max_event(const uint64_t* offsets, uint64_t n_events, uint32_t* out, uint32_t* err,
                             cudaStream_t s);
cudaError_t launch_pileup_count(const PuParams& p, int n_sms, cudaStream_t s);
cudaError_t launch_postprocess(const PostParams& p, int n_sms, cudaStream_t s);
cudaError_t launch_track_ip(const IPParams& p, int n_sms, cudaStream_t s);
cudaError_t launch_jet_max_objects(const JetParams& p, uint32_t* out, cudaStream_t s);
cudaError_t launch_cluster(const JetParams& p, uint32_t grid, size_t smem, cudaStream_t s);
cudaError_t occupancy_cluster(uint32_t threads, size_t smem, int* blocks);
cudaError_t launch_pileup_fill(const PuParams& p, int n_sms, cudaStream_t s);
cudaError_t launch_dense(const uint64_t* offsets, uint64_t n_events, const uint32_t* counts,
                         uint64_t* dense_off, uint64_t stride, unsigned long long* carry,
                         const pdr_outputs& src, const pdr_outputs& dst, int n_sms, cudaStream_t s);
}  // namespace pdr

using namespace pdr;

namespace {

thread_local std::string t_err;

// NVTX range for the duration of a scope: the host-side stages of each entry
// point show up in a timeline tool (Nsight Systems, ncu's NVTX filter).  The
// response's device stages S0-S9 run inside one fused kernel, so they have no
// ranges of their own.  NVTX3 is header-only: without an attached tool a range
// costs a check of a null pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int fail(int code, const std::string& msg) {
  t_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(PDR_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

#define PDR_CUDA(call, what)                       \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cuda_fail(_e, what); \
  } while (0)

uint32_t next_pow2(uint64_t v) {
  uint32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// ---------------------------------------------------------------- pool
// First-fit allocator over one device region (results of submit(), staging
// of the host-buffer path, scratch).  256-byte granularity.
struct Pool {
  unsigned char* base = nullptr;
  uint64_t size = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> length
  std::map<uint64_t, uint64_t> used_;

  int init(uint64_t bytes) {
    size = (bytes + 255) & ~255ull;
    if (cudaMalloc((void**)&base, size) != cudaSuccess) {
      base = nullptr;
      return PDR_ENOMEM;
    }
    free_[0] = size;
    return PDR_OK;
  }
  void destroy() {
    if (base) cudaFree(base);
    base = nullptr;
    free_.clear();
    used_.clear();
  }
  void* alloc(uint64_t bytes) {
    bytes = (bytes + 255) & ~255ull;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const uint64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_[off] = bytes;
        return base + off;
      }
    }
    return nullptr;
  }
  void release(void* p) {
    if (!p) return;
    const uint64_t off = (uint64_t)((unsigned char*)p - base);
    auto it = used_.find(off);
    if (it == used_.end()) return;
    uint64_t len = it->second;
    used_.erase(it);
    uint64_t o = off;
    auto nx = free_.lower_bound(o);
    if (nx != free_.end() && nx->first == o + len) {
      len += nx->second;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(o);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == o) {
        o = pv->first;
        len += pv->second;
        free_.erase(pv);
      }
    }
    free_[o] = len;
  }
};

struct CardEntry {
  DevCard* dev = nullptr;
  unsigned char* hot = nullptr;   // shared-memory card cache image (device)
  uint32_t hot_bytes = 0;
  uint32_t ntowers[2] = {0, 0};
  float2* centres = nullptr;      // (eta_c, phi_c) of every ECAL then HCAL tower id (device)
  float kB = 0.0f;                // field terms of the device card, kept on the host
  int32_t bsign = 1, has_field = 0;
};

struct Ticket {
  cudaEvent_t done = nullptr;
  void* mem = nullptr;
  pdr_result res{};
  int state = 2;   // 0 queued (serving), 1 inputs on the device, 2 launched (done is recorded), -1 failed
};

}  // namespace

namespace pdr {
// Record a failure message for pdr_last_error from other files of the library.
int set_last_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace pdr

struct Server;  // the serving loop (defined with its code below)

#define PDR_HOST_CHUNKS 16  // pipeline depth of the end-to-end host path

struct pdr_ctx {
  int device = 0;
  int n_sms = 0;
  size_t smem_optin = 0;
  uint32_t* d_err = nullptr;      // device error word
  uint32_t* d_word = nullptr;     // small device word for reductions
  uint32_t* d_next = nullptr;     // device work counters of the clustering launches (one a size tier)
  // fused-launch work counters, one pair a stream (launches on one stream run
  // in order; each launch leaves its counter at zero)
  uint32_t* d_work = nullptr;
  void* work_stream[PDR_WORK_STREAMS] = {};
  bool work_used[PDR_WORK_STREAMS] = {};
  uint32_t* h_word = nullptr;     // pinned host word
  std::map<uint32_t, CardEntry> cards;
  uint32_t next_card = 1;
  Pool pool;
  uint32_t max_tickets = 64;
  std::map<uint64_t, Ticket> tickets;
  uint64_t next_ticket = 1;
  std::map<uint64_t, pdr_launch> tuned;  // (card, size class) -> shape
  unsigned char* gscratch = nullptr;      // global tower tables for large events
  uint64_t gscratch_bytes = 0;
  Server* serve = nullptr;                // serving loop, if started
  std::mutex mu;
  // end-to-end host path: its copy streams, per-chunk events and a pinned
  // block for the chunks' record totals (created on first use)
  std::mutex host_mu;                     // one pdr_run_host at a time per context
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr, s_aux = nullptr;
  cudaEvent_t ev_in[PDR_HOST_CHUNKS] = {}, ev_comp[PDR_HOST_CHUNKS] = {}, ev_tot[PDR_HOST_CHUNKS] = {};
  unsigned long long* h_tot = nullptr;    // [PDR_HOST_CHUNKS][4]
  // pile-up merging: the Poisson thresholds of the last mean on the device
  unsigned long long* pu_T = nullptr;
  uint32_t pu_K = 0, pu_cap = 0;
  double pu_mean = -1.0;
  uint64_t* pu_hoff_total = nullptr;      // pinned: the merged total of a first pass
  // jet clustering: per-warp four-momentum scratch (device)
  double* jet_scratch = nullptr;
  uint64_t jet_scratch_bytes = 0;
  cudaStream_t s_jet = nullptr;   // side stream of the clustering's second size tier
  cudaEvent_t ev_jfork = nullptr, ev_jjoin = nullptr;
};

namespace {

// ------------------------------------------------------------ launch shapes
struct Shape {
  uint32_t team, block, slots, nmax, grid;
  size_t smem;
  bool may_overflow = false;   // shared table sized below the particle count (see optimistic_shape)
};

const uint32_t kTeams[] = {32, 64, 128, 256, 512, 1024};

uint32_t slots_for(uint32_t max_n) {
  // at most 3/4 of the slots can be in use (an event never has more distinct
  // towers than particles); probing stays short at that load
  // (a multiple of 32 slots: the kernel scales its hash to any table size)
  return std::max<uint32_t>(64, (uint32_t)((((uint64_t)max_n * 4 + 2) / 3 + 31) & ~31ull));
}

// Build a concrete shape for (team, block) handling events up to max_n in shared
// memory where possible.
int make_shape(pdr_ctx* ctx, uint32_t team, uint32_t block, uint32_t want_slots, uint32_t grid,
               uint32_t hot_bytes, Shape& S) {
  if (!shape_supported(team, block)) return fail(PDR_EINVAL, "unsupported launch shape (team, block)");
  const uint32_t nt = block / team;
  uint32_t slots = std::max<uint32_t>(64, (want_slots + 31u) & ~31u);
  // shrink until the CTA fits in shared memory
  while (slots > 64 && hot_bytes + nt * team_smem_bytes(team, slots, slots * 3 / 4) > ctx->smem_optin)
    slots = std::max<uint32_t>(64, (slots / 2) & ~31u);
  S.team = team;
  S.block = block;
  S.slots = slots;
  S.nmax = slots * 3 / 4;
  S.smem = (size_t)(hot_bytes + nt * team_smem_bytes(team, slots, S.nmax));
  if (S.smem > ctx->smem_optin) return fail(PDR_EINVAL, "launch shape does not fit in shared memory");
  int per_sm = 0;
  cudaError_t e = occupancy_fused(team, block, S.smem, &per_sm);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) return fail(PDR_EINVAL, "launch shape cannot be resident");
  S.grid = grid ? grid : (uint32_t)(per_sm * ctx->n_sms);
  return PDR_OK;
}

// For events larger than a table sized by particle count allows in shared
// memory: keep every particle's entries on chip and give the tower table the
// rest.  An event has far fewer distinct towers than particles (pile-up
// events of 5,500 particles hit a few thousand), so the table rarely fills;
// an event that fills it is redone by the kernel with the global table.  Not
// worth it when the table would get fewer slots than half the particles.
bool optimistic_shape(pdr_ctx* ctx, uint32_t max_n, uint32_t hot_bytes, uint32_t grid, Shape& S) {
  const uint32_t nt = S.block / S.team;
  if (!shape_supports_overflow(S.team, S.block) || max_n > 65535u || hot_bytes + 16u >= ctx->smem_optin)
    return false;
  // per team; 16 bytes stay free for the kernel's static shared flag
  const uint64_t budget = (uint64_t)(ctx->smem_optin - hot_bytes - 16u) / nt;
  const uint64_t fixed = tail_bytes(S.team) + (uint64_t)max_n * PDR_PART_BYTES;
  if (budget <= fixed) return false;
  const uint64_t slots = std::min<uint64_t>(((budget - fixed) / 24u) & ~31ull, 65536u);
  if (slots < 64 || slots < max_n / 2) return false;
  Shape T = S;
  T.slots = (uint32_t)slots;
  T.nmax = max_n;
  T.smem = (size_t)(hot_bytes + nt * team_smem_bytes(S.team, T.slots, T.nmax));
  if (T.smem + 16u > ctx->smem_optin) return false;
  int per_sm = 0;
  if (occupancy_fused_ovf(S.team, S.block, T.smem, &per_sm) != cudaSuccess || per_sm < 1) return false;
  T.grid = grid ? grid : (uint32_t)(per_sm * ctx->n_sms);
  T.may_overflow = true;
  S = T;
  return true;
}

pdr_launch default_launch(uint32_t max_n) {
  pdr_launch l{};
  if (max_n <= 128) { l.team = 32; l.block = 256; }
  else if (max_n <= 640) { l.team = 128; l.block = 256; }
  else if (max_n <= 1500) { l.team = 256; l.block = 256; }
  else if (max_n <= 3000) { l.team = 512; l.block = 512; }
  else { l.team = 1024; l.block = 1024; }
  l.table_slots = slots_for(max_n);
  l.grid = 0;
  return l;
}

uint64_t tune_key(uint32_t card_id, uint32_t max_n) {
  return ((uint64_t)card_id << 32) | (uint64_t)next_pow2(std::max<uint32_t>(max_n, 1));
}

int ensure_gscratch(pdr_ctx* ctx, uint64_t bytes) {
  if (ctx->gscratch_bytes >= bytes) return PDR_OK;
  if (ctx->gscratch) cudaFree(ctx->gscratch);
  ctx->gscratch = nullptr;
  ctx->gscratch_bytes = 0;
  if (cudaMalloc((void**)&ctx->gscratch, bytes) != cudaSuccess) {
    ctx->gscratch = nullptr;
    return fail(PDR_ENOMEM, "cannot allocate the global tower tables for large events");
  }
  ctx->gscratch_bytes = bytes;
  return PDR_OK;
}

// The work counter of fused launches on stream s (caller holds ctx->mu), or
// null when every slot belongs to another stream (the launch then hands out
// its events in a fixed round-robin).
uint32_t* work_counter(pdr_ctx* ctx, cudaStream_t s) {
  if (!ctx->d_work) return nullptr;
  const uintptr_t h = (uintptr_t)s;
  uint32_t k = (uint32_t)((h >> 4) ^ (h >> 17)) % PDR_WORK_STREAMS;
  for (uint32_t probe = 0; probe < PDR_WORK_STREAMS; ++probe, k = (k + 1) % PDR_WORK_STREAMS) {
    if (ctx->work_used[k] && ctx->work_stream[k] == (void*)s) return ctx->d_work + 2 * k;
    if (!ctx->work_used[k]) {
      ctx->work_used[k] = true;
      ctx->work_stream[k] = (void*)s;
      return ctx->d_work + 2 * k;
    }
  }
  return nullptr;
}

int check_batch(pdr_ctx* ctx, const pdr_batch* b) {
  if (!ctx || !b) return fail(PDR_EINVAL, "null context or batch");
  if (b->n_events >= (1ull << 31)) return fail(PDR_EINVAL, "n_events must be < 2^31");
  if (b->n_events > 0 && (!b->offsets || !b->pt || !b->eta || !b->phi || !b->mass || !b->pdg || !b->charge))
    return fail(PDR_EINVAL, "null input array");
  if (ctx->cards.find(b->card_id) == ctx->cards.end()) return fail(PDR_ENOTFOUND, "unknown card id");
  return PDR_OK;
}

int check_outputs(const pdr_outputs* o) {
  if (!o || !o->tracks || !o->towers || !o->eflow || !o->cands || !o->iso || !o->counts)
    return fail(PDR_EINVAL, "null output buffer");
  return PDR_OK;
}

int max_event_size_impl(pdr_ctx* ctx, const pdr_batch* b, cudaStream_t s, uint32_t* out) {
  if (b->n_events == 0) { *out = 0; return PDR_OK; }
  PDR_CUDA(cudaMemsetAsync(ctx->d_word, 0, 4, s), "memset");
  PDR_CUDA(launch_max_event(b->offsets, b->n_events, ctx->d_word, ctx->d_err, s), "max event kernel");
  PDR_CUDA(cudaMemcpyAsync(ctx->h_word, ctx->d_word, 4, cudaMemcpyDeviceToHost, s), "copy max");
  PDR_CUDA(cudaStreamSynchronize(s), "sync");
  *out = *ctx->h_word;
  return PDR_OK;
}

// Launch plan: the team shape before the card images of a launch are known.
struct Plan {
  uint32_t team, block, want_slots, grid;
};

Plan plan_launch(pdr_ctx* ctx, uint32_t card_id, uint32_t max_n, const pdr_launch* l) {
  pdr_launch use;
  if (l) use = *l;
  else {
    auto it = ctx->tuned.find(tune_key(card_id, max_n));
    use = it != ctx->tuned.end() ? it->second : default_launch(max_n);
  }
  Plan P;
  P.team = use.team;
  P.block = use.block;
  P.want_slots = use.table_slots ? use.table_slots : slots_for(max_n);
  P.grid = use.grid;
  return P;
}

void fill_seg(KSeg& g, const pdr_batch* b, const pdr_outputs* o, uint64_t start, uint32_t card) {
  g.event_start = start;
  g.n_events = b->n_events;
  g.offsets = b->offsets;
  g.pt = b->pt; g.eta = b->eta; g.phi = b->phi; g.mass = b->mass; g.vz = b->vz;
  g.pdg = b->pdg; g.charge = b->charge;
  set_round_keys(g, b->seed);
  g.event_base = b->event_index_base;
  g.card = card;
  g.tracks = o->tracks; g.towers = o->towers; g.eflow = o->eflow; g.cands = o->cands;
  g.iso = o->iso; g.counts = o->counts;
  g.debug = (b->flags & PDR_BATCH_DEBUG) ? o->debug : nullptr;
}

// Table and scratch parameters of a launch for events up to max_n.
int set_tables(pdr_ctx* ctx, KParams& p, const Shape& S, uint32_t max_n) {
  p.table_slots = S.slots;
  p.nmax_smem = S.nmax;
  p.smem_may_overflow = S.may_overflow ? 1u : 0u;
  p.err = ctx->d_err;
  if (max_n > S.nmax || S.may_overflow) {   // the global table: larger events, or the redo of an overflow
    const uint32_t gs = slots_for(max_n);
    if (gs > 65536) return fail(PDR_EOVERFLOW, "event larger than 49152 particles");
    p.g_slots = gs;
    p.g_nmax = gs * 3 / 4;
    p.g_team_bytes = global_team_bytes(gs, p.g_nmax);
    const uint64_t need = p.g_team_bytes * (uint64_t)S.grid * (S.block / S.team);
    int rc = ensure_gscratch(ctx, need);
    if (rc) return rc;
    p.gscratch = ctx->gscratch;
  }
  return PDR_OK;
}

// Parameter block and shape of one fused launch over up to PDR_LAUNCH_SEGS
// batches using up to PDR_LAUNCH_CARDS distinct cards (the caller groups them).
int prepare_group(pdr_ctx* ctx, const pdr_batch* const* bs, const pdr_outputs* const* os, uint32_t n,
                  const Plan& P, uint32_t max_n, KParams& p, Shape& S) {
  std::memset(&p, 0, sizeof p);
  uint64_t start = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const CardEntry& ce = ctx->cards[bs[k]->card_id];
    uint32_t slot = p.n_cards;
    for (uint32_t c = 0; c < p.n_cards; ++c)
      if (p.hot[c] == ce.hot) slot = c;
    if (slot == p.n_cards) {
      if (p.n_cards == PDR_LAUNCH_CARDS) return fail(PDR_EINVAL, "too many cards in one launch group");
      p.hot[slot] = ce.hot;
      p.hot_bytes[slot] = ce.hot_bytes;
      p.hot_off[slot] = p.hot_total;
      p.hot_total += ce.hot_bytes;
      ++p.n_cards;
    }
    fill_seg(p.seg[k], bs[k], os[k], start, slot);
    start += bs[k]->n_events;
  }
  p.n_segs = n;
  p.n_events = start;
  int rc = make_shape(ctx, P.team, P.block, P.want_slots, P.grid, p.hot_total, S);
  if (rc) return rc;
  if (max_n > S.nmax) optimistic_shape(ctx, max_n, p.hot_total, P.grid, S);
  return set_tables(ctx, p, S, max_n);
}

int launch_group(pdr_ctx* ctx, const pdr_batch* const* bs, const pdr_outputs* const* os, uint32_t n,
                 const Plan& P, uint32_t max_n, cudaStream_t s) {
  static thread_local KParams p;  // 5 KB: keep it off the stack
  Shape S;
  int rc = prepare_group(ctx, bs, os, n, P, max_n, p, S);
  if (rc) return rc;
  if (p.n_events == 0) return PDR_OK;
  p.work = work_counter(ctx, s);
  PDR_CUDA(launch_fused(S.team, S.block, p, S.grid, S.smem, s), "fused kernel launch");
  return PDR_OK;
}

// Any number of batches: consecutive groups of at most PDR_LAUNCH_SEGS batches
// and PDR_LAUNCH_CARDS cards, one fused launch each.
int launch_batches(pdr_ctx* ctx, const pdr_batch* bs, const pdr_outputs* os, uint32_t n, const Plan& P,
                   uint32_t max_n, cudaStream_t s) {
  std::vector<const pdr_batch*> gb;
  std::vector<const pdr_outputs*> go;
  std::vector<uint32_t> cards;
  auto flush = [&]() -> int {
    int rc = gb.empty() ? PDR_OK : launch_group(ctx, gb.data(), go.data(), (uint32_t)gb.size(), P, max_n, s);
    gb.clear(); go.clear(); cards.clear();
    return rc;
  };
  for (uint32_t k = 0; k < n; ++k) {
    const bool new_card = std::find(cards.begin(), cards.end(), bs[k].card_id) == cards.end();
    if (gb.size() == PDR_LAUNCH_SEGS || (new_card && cards.size() == PDR_LAUNCH_CARDS)) {
      int rc = flush();
      if (rc) return rc;
    }
    if (std::find(cards.begin(), cards.end(), bs[k].card_id) == cards.end()) cards.push_back(bs[k].card_id);
    gb.push_back(&bs[k]);
    go.push_back(&os[k]);
  }
  return flush();
}

int batch_max_n(pdr_ctx* ctx, const pdr_batch* b, cudaStream_t s, uint32_t* max_n) {
  *max_n = b->max_event_size;
  if (*max_n == 0 && b->n_events > 0) return max_event_size_impl(ctx, b, s, max_n);
  return PDR_OK;
}

}  // namespace

// =================================================================== ABI
extern "C" {

int pdr_abi_version(void) { return PDR_ABI_VERSION; }

const char* pdr_last_error(pdr_ctx*) { return t_err.c_str(); }

int pdr_create(pdr_ctx** out, int cuda_device, const pdr_options* opt) {
  if (!out) return fail(PDR_EINVAL, "null out");
  *out = nullptr;
  PDR_CUDA(cudaSetDevice(cuda_device), "cudaSetDevice");
  pdr_ctx* ctx = new pdr_ctx();
  ctx->device = cuda_device;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, cuda_device);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e, "cudaGetDeviceProperties");
  }
  ctx->n_sms = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  if (cudaMalloc((void**)&ctx->d_err, 32) != cudaSuccess || cudaMemset(ctx->d_err, 0, 32) != cudaSuccess) {
    delete ctx;
    return fail(PDR_ENOMEM, "cannot allocate the device error word");
  }
  ctx->d_word = ctx->d_err + 2;
  ctx->d_next = ctx->d_err + 4;
  // work counters (optional: without them launches use a fixed round-robin)
  if (cudaMalloc((void**)&ctx->d_work, 8ull * PDR_WORK_STREAMS) != cudaSuccess ||
      cudaMemset(ctx->d_work, 0, 8ull * PDR_WORK_STREAMS) != cudaSuccess) {
    if (ctx->d_work) cudaFree(ctx->d_work);
    ctx->d_work = nullptr;
    cudaGetLastError();
  }
  if (cudaMallocHost((void**)&ctx->h_word, 16) != cudaSuccess) {
    cudaFree(ctx->d_err);
    if (ctx->d_work) cudaFree(ctx->d_work);
    delete ctx;
    return fail(PDR_ENOMEM, "cannot allocate pinned host word");
  }
  const uint64_t pool = opt && opt->pool_bytes ? opt->pool_bytes : (1ull << 30);
  if (ctx->pool.init(pool) != PDR_OK) {
    cudaFree(ctx->d_err);
    if (ctx->d_work) cudaFree(ctx->d_work);
    cudaFreeHost(ctx->h_word);
    delete ctx;
    return fail(PDR_ENOMEM, "cannot allocate the device pool");
  }
  if (opt && opt->max_tickets) ctx->max_tickets = opt->max_tickets;
  *out = ctx;
  return PDR_OK;
}

int pdr_destroy(pdr_ctx* ctx) {
  if (!ctx) return PDR_OK;
  if (ctx->serve) pdr_serve_stop(ctx);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->tickets)
    if (kv.second.done) cudaEventDestroy(kv.second.done);
  for (auto& kv : ctx->cards) cudaFree(kv.second.dev);
  ctx->pool.destroy();
  if (ctx->gscratch) cudaFree(ctx->gscratch);
  if (ctx->s_h2d) cudaStreamDestroy(ctx->s_h2d);
  if (ctx->s_d2h) cudaStreamDestroy(ctx->s_d2h);
  if (ctx->s_aux) cudaStreamDestroy(ctx->s_aux);
  for (int k = 0; k < PDR_HOST_CHUNKS; ++k) {
    if (ctx->ev_in[k]) cudaEventDestroy(ctx->ev_in[k]);
    if (ctx->ev_comp[k]) cudaEventDestroy(ctx->ev_comp[k]);
    if (ctx->ev_tot[k]) cudaEventDestroy(ctx->ev_tot[k]);
  }
  if (ctx->h_tot) cudaFreeHost(ctx->h_tot);
  if (ctx->pu_T) cudaFree(ctx->pu_T);
  if (ctx->pu_hoff_total) cudaFreeHost(ctx->pu_hoff_total);
  if (ctx->jet_scratch) cudaFree(ctx->jet_scratch);
  if (ctx->s_jet) cudaStreamDestroy(ctx->s_jet);
  if (ctx->ev_jfork) cudaEventDestroy(ctx->ev_jfork);
  if (ctx->ev_jjoin) cudaEventDestroy(ctx->ev_jjoin);
  if (ctx->d_work) cudaFree(ctx->d_work);
  cudaFree(ctx->d_err);
  cudaFreeHost(ctx->h_word);
  delete ctx;
  return PDR_OK;
}

int pdr_card_load(pdr_ctx* ctx, const pdr_card* card, uint32_t* card_id) {
  NvtxRange nvtx_range("pdr_card_load");
  if (!ctx || !card || !card_id) return fail(PDR_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(ctx->mu);
  DevCard* host = new DevCard();
  int rc = expand_card(card, *host);
  if (rc) {
    delete host;
    return rc;
  }
  CardEntry ce;
  ce.ntowers[0] = (uint32_t)host->calo[0].ntowers;
  ce.kB = host->kB;
  ce.bsign = host->Bsign;
  ce.has_field = host->has_field;
  ce.ntowers[1] = (uint32_t)host->calo[1].ntowers;
  std::vector<unsigned char> hot(PDR_HOT_MAX_BYTES);
  const size_t hot_bytes = build_hot_card(*host, hot.data(), hot.size());
  if (hot_bytes == 0) {
    delete host;
    return fail(PDR_ECARD, "card tables exceed the 40 KiB shared-memory card cache");
  }
  // tower centres by id, for the post-processing (float32 of the double centres)
  std::vector<float2> centres;
  centres.reserve((size_t)ce.ntowers[0] + ce.ntowers[1]);
  for (int calo = 0; calo < 2; ++calo) {
    const DevCalo& D = host->calo[calo];
    for (int r = 0; r < D.nring; ++r)
      for (int k = 0; k < D.nphi[r]; ++k)
        centres.push_back(make_float2(D.eta_c[r], host->phi_pool[D.phioff[r] + D.nphi[r] + 1 + k]));
  }
  cudaSetDevice(ctx->device);
  const size_t hot_off = (sizeof(DevCard) + 255) & ~(size_t)255;
  const size_t ctr_off = (hot_off + hot_bytes + 255) & ~(size_t)255;
  if (cudaMalloc((void**)&ce.dev, ctr_off + centres.size() * sizeof(float2)) != cudaSuccess) {
    delete host;
    return fail(PDR_ENOMEM, "cannot allocate card tables");
  }
  ce.hot = (unsigned char*)ce.dev + hot_off;
  ce.hot_bytes = (uint32_t)hot_bytes;
  ce.centres = (float2*)((unsigned char*)ce.dev + ctr_off);
  cudaError_t e = cudaMemcpy(ce.dev, host, sizeof(DevCard), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ce.hot, hot.data(), hot_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ce.centres, centres.data(), centres.size() * sizeof(float2), cudaMemcpyHostToDevice);
  delete host;
  if (e != cudaSuccess) {
    cudaFree(ce.dev);
    return cuda_fail(e, "card upload");
  }
  *card_id = ctx->next_card++;
  ctx->cards[*card_id] = ce;
  return PDR_OK;
}

int pdr_card_unload(pdr_ctx* ctx, uint32_t card_id) {
  if (!ctx) return fail(PDR_EINVAL, "null context");
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->cards.find(card_id);
  if (it == ctx->cards.end()) return fail(PDR_ENOTFOUND, "unknown card id");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(it->second.dev);
  ctx->cards.erase(it);
  return PDR_OK;
}

int pdr_card_towers(pdr_ctx* ctx, uint32_t card_id, int calo, uint32_t* n) {
  if (!ctx || !n || calo < 0 || calo > 1) return fail(PDR_EINVAL, "bad argument");
  auto it = ctx->cards.find(card_id);
  if (it == ctx->cards.end()) return fail(PDR_ENOTFOUND, "unknown card id");
  *n = it->second.ntowers[calo];
  return PDR_OK;
}

int pdr_max_event_size(pdr_ctx* ctx, const pdr_batch* b, void* stream, uint32_t* out) {
  if (!ctx || !b || !out) return fail(PDR_EINVAL, "null argument");
  if (b->n_events > 0 && !b->offsets) return fail(PDR_EINVAL, "null offsets");
  cudaSetDevice(ctx->device);
  return max_event_size_impl(ctx, b, (cudaStream_t)stream, out);
}

int pdr_run(pdr_ctx* ctx, const pdr_batch* b, const pdr_outputs* o, const pdr_launch* l, void* stream) {
  NvtxRange nvtx_range("pdr_run");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if ((rc = check_outputs(o))) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  uint32_t max_n = 0;
  if ((rc = batch_max_n(ctx, b, (cudaStream_t)stream, &max_n))) return rc;
  return launch_batches(ctx, b, o, 1, plan_launch(ctx, b->card_id, max_n, l), max_n, (cudaStream_t)stream);
}

int pdr_run_multi(pdr_ctx* ctx, const pdr_batch* bs, uint32_t n, const pdr_outputs* os, const pdr_launch* l,
                  void* stream) {
  NvtxRange nvtx_range("pdr_run_multi");
  if (!ctx || (n > 0 && (!bs || !os))) return fail(PDR_EINVAL, "null argument");
  for (uint32_t k = 0; k < n; ++k) {
    int rc = check_batch(ctx, &bs[k]);
    if (rc) return rc;
    if ((rc = check_outputs(&os[k]))) return rc;
  }
  if (n == 0) return PDR_OK;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t max_n = 0;
  for (uint32_t k = 0; k < n; ++k) {
    uint32_t m = 0;
    int rc = batch_max_n(ctx, &bs[k], s, &m);
    if (rc) return rc;
    max_n = std::max(max_n, m);
  }
  return launch_batches(ctx, bs, os, n, plan_launch(ctx, bs[0].card_id, max_n, l), max_n, s);
}

int pdr_run_per_event(pdr_ctx* ctx, const pdr_batch* b, const pdr_outputs* o, void* stream) {
  NvtxRange nvtx_range("pdr_run_per_event");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if ((rc = check_outputs(o))) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t max_n = 0;
  if ((rc = batch_max_n(ctx, b, s, &max_n))) return rc;
  const CardEntry& ce = ctx->cards[b->card_id];
  Shape S;
  if ((rc = make_shape(ctx, 256, 256, slots_for(max_n), 1, ce.hot_bytes, S))) return rc;
  S.grid = 1;
  static thread_local KParams p;
  std::memset(&p, 0, sizeof p);
  p.n_cards = 1;
  p.hot[0] = ce.hot;
  p.hot_bytes[0] = ce.hot_bytes;
  p.hot_total = ce.hot_bytes;
  p.n_segs = 1;
  p.n_events = 1;
  if ((rc = set_tables(ctx, p, S, max_n))) return rc;
  for (uint64_t e = 0; e < b->n_events; ++e) {
    pdr_batch one = *b;
    one.n_events = 1;
    one.offsets = b->offsets + e;
    one.event_index_base = b->event_index_base + (uint32_t)e;
    pdr_outputs oe = *o;
    oe.counts = o->counts + 4 * e;
    fill_seg(p.seg[0], &one, &oe, 0, 0);
    PDR_CUDA(launch_fused(S.team, S.block, p, S.grid, S.smem, s), "fused kernel launch");
  }
  return PDR_OK;
}

int pdr_check(pdr_ctx* ctx, void* stream) {
  if (!ctx) return fail(PDR_EINVAL, "null context");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  PDR_CUDA(cudaMemcpyAsync(ctx->h_word, ctx->d_err, 4, cudaMemcpyDeviceToHost, s), "read error word");
  PDR_CUDA(cudaStreamSynchronize(s), "sync");
  const uint32_t w = *ctx->h_word;
  PDR_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, s), "clear error word");
  PDR_CUDA(cudaStreamSynchronize(s), "sync");
  if (w) {
    std::string m = "device error:";
    if (w & ERR_CSR) m += " malformed CSR offsets;";
    if (w & ERR_OVERSIZE) m += " event larger than the launch allows;";
    if (w & ERR_TABLE) m += " tower table full;";
    if (w & ERR_PILEUP) m += " pile-up merge arguments differ from the first pass;";
    if (w & ERR_VERTEX) m += " no pile-up vertex inside the truncation in 1024 draws;";
    if (w & ERR_JETS) m += " jet clustering: more jets than the event's slots (the rest dropped) or a bookkeeping error;";
    if (w & ERR_BOUNDS) m += " index out of bounds (bounds-checking build);";
    return fail(PDR_EDEVICE, m);
  }
  return PDR_OK;
}

int pdr_autotune(pdr_ctx* ctx, const pdr_batch* b, const pdr_outputs* o, void* stream, pdr_launch* best) {
  NvtxRange nvtx_range("pdr_autotune");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if ((rc = check_outputs(o))) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t max_n = b->max_event_size;
  if (max_n == 0 && b->n_events > 0 && (rc = max_event_size_impl(ctx, b, s, &max_n))) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  pdr_launch best_l = default_launch(max_n);
  const uint32_t blocks_for[] = {256, 256, 256, 256, 512, 1024};
  for (int ti = 0; ti < 6; ++ti) {
    const uint32_t team = kTeams[ti];
    for (uint32_t block : {blocks_for[ti], team < 256 ? 128u : 0u}) {
      if (block == 0 || block < team || !shape_supported(team, block)) continue;
      // table sized for the largest event, or for the typical event with the
      // largest ones spilling to the global table
      for (uint32_t want : {slots_for(max_n), 2 * slots_for(max_n), slots_for(std::max<uint32_t>(max_n / 2, 1))}) {
        Shape S;
        if (make_shape(ctx, team, block, want, 0, ctx->cards[b->card_id].hot_bytes, S) != PDR_OK) continue;
        // a team must not walk a huge event alone in tiny chunks
        if (team == 32 && max_n > 1024) continue;
        const Plan P{team, block, want, 0};
        if (launch_batches(ctx, b, o, 1, P, max_n, s) != PDR_OK) continue;  // warm-up
        cudaEventRecord(e0, s);
        if (launch_batches(ctx, b, o, 1, P, max_n, s) != PDR_OK) continue;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best_l.team = team;
          best_l.block = block;
          best_l.table_slots = S.slots;
          best_l.grid = 0;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  ctx->tuned[tune_key(b->card_id, max_n)] = best_l;
  if (best) *best = best_l;
  return PDR_OK;
}

int pdr_run_host(pdr_ctx* ctx, const pdr_batch* hb, const pdr_outputs* ho, const pdr_launch* l, void* stream) {
  NvtxRange nvtx_range("pdr_run_host");
  int rc = check_batch(ctx, hb);
  if (rc) return rc;
  if (!ho || !ho->tracks || !ho->towers || !ho->eflow || !ho->cands || !ho->iso || !ho->counts)
    return fail(PDR_EINVAL, "null host output buffer");
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> hg(ctx->host_mu);
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->s_h2d) {
    if (cudaStreamCreateWithFlags(&ctx->s_h2d, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_d2h, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc((void**)&ctx->h_tot, sizeof(unsigned long long) * 4 * PDR_HOST_CHUNKS, 0) != cudaSuccess)
      return fail(PDR_EDEVICE, "cannot create the host-path streams");
    for (int k = 0; k < PDR_HOST_CHUNKS; ++k)
      if (cudaEventCreateWithFlags(&ctx->ev_in[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->ev_comp[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->ev_tot[k], cudaEventDisableTiming) != cudaSuccess)
        return fail(PDR_EDEVICE, "cannot create the host-path events");
  }
  const uint64_t ne = hb->n_events;
  const uint64_t np = ne ? hb->offsets[ne] : 0;
  const uint64_t cap = np ? np : 1;
  for (uint64_t e = 0; e < ne; ++e)
    if (hb->offsets[e + 1] < hb->offsets[e]) return fail(PDR_EINVAL, "offsets not monotone");
  uint32_t max_n = hb->max_event_size;
  if (max_n == 0)
    for (uint64_t e = 0; e < ne; ++e) max_n = std::max<uint32_t>(max_n, (uint32_t)(hb->offsets[e + 1] - hb->offsets[e]));
  // device staging from the pool: inputs, slot-layout outputs, dense outputs
  const uint64_t in_bytes = (ne + 1) * 8 + np * (4 * 4 + 4 + 1) + (hb->vz ? np * 4 : 0) + 8 * 256;
  const uint64_t out_bytes = cap * (sizeof(pdr_track) + sizeof(pdr_tower) + sizeof(pdr_eflow) +
                                    sizeof(pdr_cand) + sizeof(pdr_iso)) + (ne + 1) * 16 + 8 * 256;
  const uint64_t dense_bytes = out_bytes + 4 * (ne + 1) * 8 + 4 * 8 + 2 * 256;
  std::unique_lock<std::mutex> g(ctx->mu);
  unsigned char* m = (unsigned char*)ctx->pool.alloc(in_bytes + out_bytes + dense_bytes);
  g.unlock();
  if (!m) return fail(PDR_ENOMEM, "device pool too small for this batch");
  auto carve = [&](uint64_t bytes) {
    unsigned char* r = m;
    m += (bytes + 255) & ~255ull;
    return (void*)r;
  };
  unsigned char* mem0 = m;
  pdr_batch db = *hb;
  db.offsets = (const uint64_t*)carve((ne + 1) * 8);
  db.pt = (const float*)carve(np * 4);
  db.eta = (const float*)carve(np * 4);
  db.phi = (const float*)carve(np * 4);
  db.mass = (const float*)carve(np * 4);
  db.pdg = (const int32_t*)carve(np * 4);
  db.charge = (const int8_t*)carve(np);
  db.vz = hb->vz ? (const float*)carve(np * 4) : nullptr;
  db.max_event_size = max_n;
  db.flags &= ~PDR_BATCH_DEBUG;
  pdr_outputs so{};
  so.tracks = (pdr_track*)carve(cap * sizeof(pdr_track));
  so.towers = (pdr_tower*)carve(cap * sizeof(pdr_tower));
  so.eflow = (pdr_eflow*)carve(cap * sizeof(pdr_eflow));
  so.cands = (pdr_cand*)carve(cap * sizeof(pdr_cand));
  so.iso = (pdr_iso*)carve(cap * sizeof(pdr_iso));
  so.counts = (uint32_t*)carve((ne + 1) * 16);
  pdr_outputs dd{};
  dd.tracks = (pdr_track*)carve(cap * sizeof(pdr_track));
  dd.towers = (pdr_tower*)carve(cap * sizeof(pdr_tower));
  dd.eflow = (pdr_eflow*)carve(cap * sizeof(pdr_eflow));
  dd.cands = (pdr_cand*)carve(cap * sizeof(pdr_cand));
  dd.iso = (pdr_iso*)carve(cap * sizeof(pdr_iso));
  uint64_t* dense_off = (uint64_t*)carve(4 * (ne + 1) * 8);
  unsigned long long* carry = (unsigned long long*)carve(4 * 8);
  cudaStream_t s_in = ctx->s_h2d, s_out = ctx->s_d2h, s_aux = ctx->s_aux;
  auto done = [&](int code) {
    cudaStreamSynchronize(s_in);
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(s_aux);
    cudaStreamSynchronize(s_out);
    std::lock_guard<std::mutex> g2(ctx->mu);
    ctx->pool.release(mem0);
    return code;
  };
  // Chunks of whole events, about 2 M particles each (at most PDR_HOST_CHUNKS):
  // all input copies are queued at once (copy stream), each chunk's kernels
  // wait for its inputs (the caller's stream), a third stream brings back each
  // chunk's record totals and counts, and each chunk's records follow on the
  // second copy stream as soon as its totals are known on the host.
  const uint32_t K = ne == 0 ? 0 : (uint32_t)std::min<uint64_t>(
      std::min<uint64_t>(PDR_HOST_CHUNKS, ne), std::max<uint64_t>(1, np >> 21));
  std::vector<uint64_t> eb(K + 1, ne);
  for (uint32_t k = 0; k < K; ++k)  // first event of each chunk, by particle count
    eb[k] = (uint64_t)(std::lower_bound(hb->offsets, hb->offsets + ne, np * k / K) - hb->offsets);
  eb[0] = 0;
  for (uint32_t k = 1; k < K; ++k) eb[k] = std::max(eb[k], eb[k - 1]);
  const Plan P = plan_launch(ctx, db.card_id, max_n, l);
  if (K > 0 && cudaMemsetAsync(carry, 0, 4 * 8, s) != cudaSuccess) return done(fail(PDR_EDEVICE, "memset"));
#define PDR_CP(dst, src, bytes, kind, st)                                                      \
  if ((bytes) && cudaMemcpyAsync((void*)(dst), (const void*)(src), (bytes), kind, st) != cudaSuccess) \
    return done(fail(PDR_EDEVICE, "host-device copy"));
  for (uint32_t k = 0; k < K; ++k) {
    const uint64_t e0 = eb[k], e1 = eb[k + 1], nk = e1 - e0;
    const uint64_t a0 = hb->offsets[e0], a1 = hb->offsets[e1], pk = a1 - a0;
    PDR_CP(db.offsets + e0, hb->offsets + e0, (nk + 1) * 8, cudaMemcpyHostToDevice, s_in);
    PDR_CP(db.pt + a0, hb->pt + a0, pk * 4, cudaMemcpyHostToDevice, s_in);
    PDR_CP(db.eta + a0, hb->eta + a0, pk * 4, cudaMemcpyHostToDevice, s_in);
    PDR_CP(db.phi + a0, hb->phi + a0, pk * 4, cudaMemcpyHostToDevice, s_in);
    PDR_CP(db.mass + a0, hb->mass + a0, pk * 4, cudaMemcpyHostToDevice, s_in);
    PDR_CP(db.pdg + a0, hb->pdg + a0, pk * 4, cudaMemcpyHostToDevice, s_in);
    PDR_CP(db.charge + a0, hb->charge + a0, pk, cudaMemcpyHostToDevice, s_in);
    if (hb->vz) PDR_CP(db.vz + a0, hb->vz + a0, pk * 4, cudaMemcpyHostToDevice, s_in);
    cudaEventRecord(ctx->ev_in[k], s_in);
    cudaStreamWaitEvent(s, ctx->ev_in[k], 0);
    if (nk > 0) {
      // the chunk as a batch of its own: same arrays (absolute offsets), its
      // events' indices, its counts
      pdr_batch bk = db;
      bk.n_events = nk;
      bk.offsets = db.offsets + e0;
      bk.event_index_base = hb->event_index_base + (uint32_t)e0;
      pdr_outputs ok = so;
      ok.counts = so.counts + 4 * e0;
      {
        std::lock_guard<std::mutex> g2(ctx->mu);
        if ((rc = launch_batches(ctx, &bk, &ok, 1, P, max_n, s))) return done(rc);
      }
      cudaError_t e = launch_dense(bk.offsets, nk, ok.counts, dense_off + e0, ne + 1, carry, so, dd, ctx->n_sms, s);
      if (e != cudaSuccess) return done(cuda_fail(e, "dense compaction"));
    }
    cudaEventRecord(ctx->ev_comp[k], s);
    // the chunk's record totals (running, after the chunk) and its counts
    cudaStreamWaitEvent(s_aux, ctx->ev_comp[k], 0);
    PDR_CP(ctx->h_tot + 4 * k, carry, 4 * 8, cudaMemcpyDeviceToHost, s_aux);
    cudaEventRecord(ctx->ev_tot[k], s_aux);
    PDR_CP(ho->counts + 4 * e0, so.counts + 4 * e0, nk * 16, cudaMemcpyDeviceToHost, s_aux);
  }
  // dense records of each chunk, as soon as its totals are known on the host
  // (their kernels are then complete: the totals' copy waited for them)
  uint64_t prev[4] = {0, 0, 0, 0};
  for (uint32_t k = 0; k < K; ++k) {
    if (cudaEventSynchronize(ctx->ev_tot[k]) != cudaSuccess) return done(fail(PDR_EDEVICE, "event synchronise"));
    const unsigned long long* t = ctx->h_tot + 4 * k;
    PDR_CP(ho->tracks + prev[0], dd.tracks + prev[0], (t[0] - prev[0]) * sizeof(pdr_track), cudaMemcpyDeviceToHost, s_out);
    PDR_CP(ho->towers + prev[1], dd.towers + prev[1], (t[1] - prev[1]) * sizeof(pdr_tower), cudaMemcpyDeviceToHost, s_out);
    PDR_CP(ho->eflow + prev[2], dd.eflow + prev[2], (t[2] - prev[2]) * sizeof(pdr_eflow), cudaMemcpyDeviceToHost, s_out);
    PDR_CP(ho->cands + prev[3], dd.cands + prev[3], (t[3] - prev[3]) * sizeof(pdr_cand), cudaMemcpyDeviceToHost, s_out);
    PDR_CP(ho->iso + prev[3], dd.iso + prev[3], (t[3] - prev[3]) * sizeof(pdr_iso), cudaMemcpyDeviceToHost, s_out);
    for (int c = 0; c < 4; ++c) prev[c] = t[c];
  }
#undef PDR_CP
  if (cudaStreamSynchronize(s_out) != cudaSuccess || cudaStreamSynchronize(s_aux) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return done(fail(PDR_EDEVICE, "stream synchronise"));
  return done(PDR_OK);
}

// ---------------------------------------------------------------- tickets
int pdr_submit(pdr_ctx* ctx, const pdr_batch* b, void* stream, uint64_t* ticket) {
  NvtxRange nvtx_range("pdr_submit");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if (!ticket) return fail(PDR_EINVAL, "null ticket");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> g(ctx->mu);
  if (ctx->tickets.size() >= ctx->max_tickets) return fail(PDR_EBUSY, "too many tickets in flight");
  uint64_t np = 0;
  if (b->n_events > 0) {
    PDR_CUDA(cudaMemcpyAsync(ctx->h_word, b->offsets + b->n_events, 8, cudaMemcpyDeviceToHost, s), "read size");
    PDR_CUDA(cudaStreamSynchronize(s), "sync");
    std::memcpy(&np, ctx->h_word, 8);
  }
  const uint64_t cap = np ? np : 1;
  const bool dbg = (b->flags & PDR_BATCH_DEBUG) != 0;
  const uint64_t rec = sizeof(pdr_track) + sizeof(pdr_tower) + sizeof(pdr_eflow) + sizeof(pdr_cand) +
                       sizeof(pdr_iso) + (dbg ? sizeof(pdr_debug) : 0);
  const uint64_t bytes = cap * rec + (b->n_events + 1) * (16 + 8) + 16 * 256;
  unsigned char* m = (unsigned char*)ctx->pool.alloc(bytes);
  if (!m) return fail(PDR_ENOMEM, "device pool has no room for this batch (admission refused)");
  Ticket t;
  t.mem = m;
  auto carve = [&](uint64_t n) {
    unsigned char* r = m;
    m += (n + 255) & ~255ull;
    return (void*)r;
  };
  pdr_outputs o{};
  o.tracks = (pdr_track*)carve(cap * sizeof(pdr_track));
  o.towers = (pdr_tower*)carve(cap * sizeof(pdr_tower));
  o.eflow = (pdr_eflow*)carve(cap * sizeof(pdr_eflow));
  o.cands = (pdr_cand*)carve(cap * sizeof(pdr_cand));
  o.iso = (pdr_iso*)carve(cap * sizeof(pdr_iso));
  o.counts = (uint32_t*)carve((b->n_events + 1) * 16);
  o.debug = dbg ? (pdr_debug*)carve(cap * sizeof(pdr_debug)) : nullptr;
  uint64_t* offs = (uint64_t*)carve((b->n_events + 1) * 8);
  if (b->n_events > 0)
    PDR_CUDA(cudaMemcpyAsync(offs, b->offsets, (b->n_events + 1) * 8, cudaMemcpyDeviceToDevice, s), "copy offsets");
  uint32_t max_n = 0;
  if ((rc = batch_max_n(ctx, b, s, &max_n)) ||
      (rc = launch_batches(ctx, b, &o, 1, plan_launch(ctx, b->card_id, max_n, nullptr), max_n, s))) {
    ctx->pool.release(t.mem);
    return rc;
  }
  if (cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(t.done, s) != cudaSuccess) {
    ctx->pool.release(t.mem);
    return fail(PDR_EDEVICE, "cannot record completion event");
  }
  t.res.n_events = b->n_events;
  t.res.n_particles = np;
  t.res.offsets = offs;
  t.res.counts = o.counts;
  t.res.tracks = o.tracks;
  t.res.towers = o.towers;
  t.res.eflow = o.eflow;
  t.res.cands = o.cands;
  t.res.iso = o.iso;
  t.res.debug = o.debug;
  *ticket = ctx->next_ticket++;
  ctx->tickets[*ticket] = t;
  return PDR_OK;
}

int pdr_wait(pdr_ctx* ctx, uint64_t ticket, int timeout_ms) {
  if (!ctx) return fail(PDR_EINVAL, "null context");
  cudaSetDevice(ctx->device);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaEvent_t ev = nullptr;
    int state;
    {
      std::lock_guard<std::mutex> g(ctx->mu);
      auto it = ctx->tickets.find(ticket);
      if (it == ctx->tickets.end()) return fail(PDR_ENOTFOUND, "unknown ticket");
      state = it->second.state;
      ev = it->second.done;
    }
    if (state < 0) return fail(PDR_EDEVICE, "the request failed");
    if (state == 2) {
      cudaError_t e = cudaEventQuery(ev);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return cuda_fail(e, "ticket");
    }
    if (timeout_ms >= 0 &&
        std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return fail(PDR_ETIMEDOUT, "ticket still running");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  return PDR_OK;
}

int pdr_fetch(pdr_ctx* ctx, uint64_t ticket, pdr_result* r) {
  if (!ctx || !r) return fail(PDR_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return fail(PDR_ENOTFOUND, "unknown ticket");
  if (it->second.state != 2 || cudaEventQuery(it->second.done) != cudaSuccess)
    return fail(PDR_EBUSY, "ticket not finished");
  *r = it->second.res;
  return PDR_OK;
}

int pdr_release(pdr_ctx* ctx, uint64_t ticket) {
  if (!ctx) return fail(PDR_EINVAL, "null context");
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return fail(PDR_ENOTFOUND, "unknown ticket");
  if (it->second.state == 0 || it->second.state == 1) return fail(PDR_EBUSY, "request not launched yet");
  cudaSetDevice(ctx->device);
  if (it->second.state == 2) cudaEventSynchronize(it->second.done);
  cudaEventDestroy(it->second.done);
  ctx->pool.release(it->second.mem);
  ctx->tickets.erase(it);
  return PDR_OK;
}

}  // extern "C"

// =================================================================== serving
namespace {

using Clock = std::chrono::steady_clock;

struct ServeReq {
  uint64_t ticket = 0;
  pdr_batch hb{};         // caller's host batch
  pdr_batch db{};         // device copy of the inputs
  pdr_outputs o{};        // device results
  unsigned char* mem = nullptr;
  uint64_t np = 0, bytes = 0;
  uint32_t max_n = 0;
  bool waited = false;
  cudaEvent_t in_ready = nullptr;
  Clock::time_point t_submit;
};

struct Wave {
  cudaEvent_t done = nullptr;
  std::vector<ServeReq*> reqs;
};

struct GraphSlot {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t node = nullptr;
};

}  // namespace

struct Server {
  pdr_serve_options opt{};
  std::thread th;
  std::mutex m;  // arrivals, stop, statistics
  std::condition_variable cv;
  std::deque<ServeReq*> arrivals;
  std::deque<ServeReq*> admitted;
  std::deque<Wave> inflight;
  bool stop = false;
  cudaStream_t s_copy = nullptr, s_comp = nullptr, s_cap = nullptr;
  // keyed by the launch shape and the kernel variant (shared table sized
  // below the particle count or not)
  std::map<std::tuple<uint32_t, uint32_t, uint32_t, size_t, bool>, GraphSlot> graphs;
  std::vector<double> lat_ms;
  uint64_t requests_done = 0, events_done = 0, particles_done = 0, waves = 0, admission_waits = 0,
           graph_launches = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
};

namespace {

// Carve a request's device memory and queue its input copies (ctx->mu held).
void serve_admit(pdr_ctx* ctx, Server& sv, ServeReq* r) {
  NvtxRange nvtx_range("serve: admit");
  unsigned char* m = r->mem;
  auto carve = [&](uint64_t bytes) {
    unsigned char* q = m;
    m += (bytes + 255) & ~255ull;
    return (void*)q;
  };
  const uint64_t ne = r->hb.n_events, np = r->np, cap = np ? np : 1;
  r->db = r->hb;
  r->db.offsets = (const uint64_t*)carve((ne + 1) * 8);
  r->db.pt = (const float*)carve(np * 4);
  r->db.eta = (const float*)carve(np * 4);
  r->db.phi = (const float*)carve(np * 4);
  r->db.mass = (const float*)carve(np * 4);
  r->db.pdg = (const int32_t*)carve(np * 4);
  r->db.charge = (const int8_t*)carve(np);
  r->db.vz = r->hb.vz ? (const float*)carve(np * 4) : nullptr;
  r->db.max_event_size = r->max_n;
  r->db.flags &= ~PDR_BATCH_DEBUG;
  r->o.tracks = (pdr_track*)carve(cap * sizeof(pdr_track));
  r->o.towers = (pdr_tower*)carve(cap * sizeof(pdr_tower));
  r->o.eflow = (pdr_eflow*)carve(cap * sizeof(pdr_eflow));
  r->o.cands = (pdr_cand*)carve(cap * sizeof(pdr_cand));
  r->o.iso = (pdr_iso*)carve(cap * sizeof(pdr_iso));
  r->o.counts = (uint32_t*)carve((ne + 1) * 16);
  r->o.debug = nullptr;
  cudaStream_t s = sv.s_copy;
  cudaMemcpyAsync((void*)r->db.offsets, r->hb.offsets, (ne + 1) * 8, cudaMemcpyHostToDevice, s);
  if (np) {
    cudaMemcpyAsync((void*)r->db.pt, r->hb.pt, np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)r->db.eta, r->hb.eta, np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)r->db.phi, r->hb.phi, np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)r->db.mass, r->hb.mass, np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)r->db.pdg, r->hb.pdg, np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)r->db.charge, r->hb.charge, np, cudaMemcpyHostToDevice, s);
    if (r->hb.vz) cudaMemcpyAsync((void*)r->db.vz, r->hb.vz, np * 4, cudaMemcpyHostToDevice, s);
  }
  cudaEventRecord(r->in_ready, s);
  Ticket& t = ctx->tickets[r->ticket];
  t.mem = r->mem;
  t.state = 1;
  t.res.n_events = ne;
  t.res.n_particles = np;
  t.res.offsets = r->db.offsets;
  t.res.counts = r->o.counts;
  t.res.tracks = r->o.tracks;
  t.res.towers = r->o.towers;
  t.res.eflow = r->o.eflow;
  t.res.cands = r->o.cands;
  t.res.iso = r->o.iso;
  t.res.debug = nullptr;
}

// Launch a prepared parameter block through a captured graph of its shape.
cudaError_t graph_launch(Server& sv, const KParams& p, const Shape& S) {
  const auto key = std::make_tuple(S.team, S.block, S.grid, S.smem, S.may_overflow);
  auto it = sv.graphs.find(key);
  if (it == sv.graphs.end()) {
    GraphSlot g;
    cudaError_t e = cudaStreamBeginCapture(sv.s_cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = launch_fused(S.team, S.block, p, S.grid, S.smem, sv.s_cap);
    e = cudaStreamEndCapture(sv.s_cap, &g.graph);
    if (le != cudaSuccess) return le;
    if (e != cudaSuccess) return e;
    size_t nn = 1;
    if ((e = cudaGraphGetNodes(g.graph, &g.node, &nn)) != cudaSuccess) return e;
    if (nn != 1) return cudaErrorUnknown;
    if ((e = cudaGraphInstantiate(&g.exec, g.graph, 0)) != cudaSuccess) return e;
    it = sv.graphs.emplace(key, g).first;
  } else {
    cudaKernelNodeParams kp;
    cudaError_t e = cudaGraphKernelNodeGetParams(it->second.node, &kp);
    if (e != cudaSuccess) return e;
    void* args[1] = {(void*)&p};
    kp.kernelParams = args;
    kp.extra = nullptr;
    if ((e = cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.node, &kp)) != cudaSuccess) return e;
  }
  ++sv.graph_launches;
  return cudaGraphLaunch(it->second.exec, sv.s_comp);
}

void fail_wave(pdr_ctx* ctx, std::vector<ServeReq*>& reqs) {
  for (ServeReq* r : reqs) {
    auto it = ctx->tickets.find(r->ticket);
    if (it != ctx->tickets.end()) it->second.state = -1;
    cudaEventDestroy(r->in_ready);
    delete r;
  }
  reqs.clear();
}

// One wave: the first admitted requests (up to the limits), one fused launch.
bool serve_launch_wave(pdr_ctx* ctx, Server& sv) {
  NvtxRange nvtx_range("serve: wave");
  std::vector<ServeReq*> reqs;
  std::vector<uint32_t> cards;
  uint64_t particles = 0;
  uint32_t max_n = 0;
  const uint32_t max_req = std::min<uint32_t>(sv.opt.max_wave_requests, PDR_LAUNCH_SEGS);
  while (!sv.admitted.empty() && reqs.size() < max_req) {
    ServeReq* r = sv.admitted.front();
    const bool new_card = std::find(cards.begin(), cards.end(), r->hb.card_id) == cards.end();
    if (new_card && cards.size() == PDR_LAUNCH_CARDS) break;
    if (!reqs.empty() && particles + r->np > sv.opt.max_wave_particles) break;
    if (new_card) cards.push_back(r->hb.card_id);
    sv.admitted.pop_front();
    reqs.push_back(r);
    particles += r->np;
    max_n = std::max(max_n, r->max_n);
  }
  if (reqs.empty()) return false;
  std::lock_guard<std::mutex> g(ctx->mu);
  std::vector<const pdr_batch*> bs;
  std::vector<const pdr_outputs*> os;
  for (ServeReq* r : reqs) {
    cudaStreamWaitEvent(sv.s_comp, r->in_ready, 0);
    bs.push_back(&r->db);
    os.push_back(&r->o);
  }
  static thread_local KParams p;
  Shape S;
  const Plan P = plan_launch(ctx, reqs[0]->hb.card_id, max_n, nullptr);
  int rc = prepare_group(ctx, bs.data(), os.data(), (uint32_t)bs.size(), P, max_n, p, S);
  p.work = work_counter(ctx, sv.s_comp);   // (the graphs run on the compute stream)
  cudaError_t e = cudaSuccess;
  if (rc == PDR_OK && p.n_events > 0)
    e = sv.opt.use_graphs ? graph_launch(sv, p, S) : launch_fused(S.team, S.block, p, S.grid, S.smem, sv.s_comp);
  if (rc != PDR_OK || e != cudaSuccess) {
    fail_wave(ctx, reqs);
    return true;
  }
  Wave w;
  cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
  for (ServeReq* r : reqs) {
    Ticket& t = ctx->tickets[r->ticket];
    cudaEventRecord(t.done, sv.s_comp);
    t.state = 2;
  }
  cudaEventRecord(w.done, sv.s_comp);
  w.reqs = std::move(reqs);
  sv.inflight.push_back(std::move(w));
  return true;
}

void serve_loop(pdr_ctx* ctx) {
  Server& sv = *ctx->serve;
  cudaSetDevice(ctx->device);
  for (;;) {
    bool progress = false;
    // admission in arrival order, while the pool has room
    for (;;) {
      ServeReq* r = nullptr;
      {
        std::lock_guard<std::mutex> lk(sv.m);
        if (!sv.arrivals.empty()) r = sv.arrivals.front();
      }
      if (!r) break;
      bool ok = false;
      {
        std::lock_guard<std::mutex> g(ctx->mu);
        r->mem = (unsigned char*)ctx->pool.alloc(r->bytes);
        if (r->mem) {
          serve_admit(ctx, sv, r);
          ok = true;
        }
      }
      std::lock_guard<std::mutex> lk(sv.m);
      if (!ok) {
        if (!r->waited) { r->waited = true; ++sv.admission_waits; }
        break;
      }
      sv.arrivals.pop_front();
      sv.admitted.push_back(r);
      progress = true;
    }
    // waves
    while (sv.inflight.size() < sv.opt.max_inflight_waves && !sv.admitted.empty())
      progress |= serve_launch_wave(ctx, sv);
    // completions (waves finish in launch order on the compute stream)
    while (!sv.inflight.empty() && cudaEventQuery(sv.inflight.front().done) == cudaSuccess) {
      Wave& w = sv.inflight.front();
      const Clock::time_point now = Clock::now();
      {
        std::lock_guard<std::mutex> lk(sv.m);
        for (ServeReq* r : w.reqs) {
          sv.lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
          ++sv.requests_done;
          sv.events_done += r->hb.n_events;
          sv.particles_done += r->np;
        }
        ++sv.waves;
        sv.t_last = now;
      }
      for (ServeReq* r : w.reqs) {
        cudaEventDestroy(r->in_ready);
        delete r;
      }
      cudaEventDestroy(w.done);
      sv.inflight.pop_front();
      progress = true;
    }
    std::unique_lock<std::mutex> lk(sv.m);
    if (sv.stop && sv.arrivals.empty() && sv.admitted.empty() && sv.inflight.empty()) break;
    if (!progress) sv.cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" {

int pdr_serve_start(pdr_ctx* ctx, const pdr_serve_options* opt) {
  if (!ctx) return fail(PDR_EINVAL, "null context");
  std::lock_guard<std::mutex> g(ctx->mu);
  if (ctx->serve) return fail(PDR_EBUSY, "serving loop already running");
  cudaSetDevice(ctx->device);
  Server* sv = new Server();
  if (opt) sv->opt = *opt;
  else sv->opt.use_graphs = 1;
  if (sv->opt.max_inflight_waves == 0) sv->opt.max_inflight_waves = 2;
  if (sv->opt.max_wave_requests == 0 || sv->opt.max_wave_requests > PDR_LAUNCH_SEGS)
    sv->opt.max_wave_requests = PDR_LAUNCH_SEGS;
  if (sv->opt.max_wave_particles == 0) sv->opt.max_wave_particles = 64ull << 20;
  if (cudaStreamCreateWithFlags(&sv->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->s_comp, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->s_cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete sv;
    return fail(PDR_EDEVICE, "cannot create serving streams");
  }
  ctx->serve = sv;
  sv->th = std::thread(serve_loop, ctx);
  return PDR_OK;
}

int pdr_serve_submit(pdr_ctx* ctx, const pdr_batch* hb, uint64_t* ticket) {
  NvtxRange nvtx_range("pdr_serve_submit");
  int rc = check_batch(ctx, hb);
  if (rc) return rc;
  if (!ticket) return fail(PDR_EINVAL, "null ticket");
  if (!ctx->serve) return fail(PDR_EINVAL, "serving loop not started");
  ServeReq* r = new ServeReq();
  r->hb = *hb;
  const uint64_t ne = hb->n_events;
  r->np = ne ? hb->offsets[ne] : 0;
  uint32_t mx = 0;
  for (uint64_t e = 0; e < ne; ++e) {
    if (hb->offsets[e + 1] < hb->offsets[e]) {
      delete r;
      return fail(PDR_EINVAL, "offsets not monotone");
    }
    mx = std::max<uint32_t>(mx, (uint32_t)(hb->offsets[e + 1] - hb->offsets[e]));
  }
  r->max_n = mx;
  const uint64_t cap = r->np ? r->np : 1;
  r->bytes = (ne + 1) * (8 + 16) + r->np * (4 * 4 + 4 + 1) + (hb->vz ? r->np * 4 : 0) +
             cap * (sizeof(pdr_track) + sizeof(pdr_tower) + sizeof(pdr_eflow) + sizeof(pdr_cand) +
                    sizeof(pdr_iso)) + 16 * 256;
  cudaSetDevice(ctx->device);
  Ticket t;
  t.state = 0;
  if (cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->in_ready, cudaEventDisableTiming) != cudaSuccess) {
    delete r;
    return fail(PDR_EDEVICE, "cannot create events");
  }
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (r->bytes > ctx->pool.size) {
      cudaEventDestroy(t.done);
      cudaEventDestroy(r->in_ready);
      delete r;
      return fail(PDR_ENOMEM, "request larger than the device pool");
    }
    r->ticket = ctx->next_ticket++;
    ctx->tickets[r->ticket] = t;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(ctx->serve->m);
    if (!ctx->serve->any) {
      ctx->serve->any = true;
      ctx->serve->t_first = r->t_submit;
    }
    ctx->serve->arrivals.push_back(r);
  }
  ctx->serve->cv.notify_one();
  *ticket = r->ticket;
  return PDR_OK;
}

int pdr_serve_stats_get(pdr_ctx* ctx, pdr_serve_stats* out) {
  if (!ctx || !out) return fail(PDR_EINVAL, "null argument");
  if (!ctx->serve) return fail(PDR_EINVAL, "serving loop not started");
  Server& sv = *ctx->serve;
  std::lock_guard<std::mutex> lk(sv.m);
  std::memset(out, 0, sizeof *out);
  out->requests_done = sv.requests_done;
  out->events_done = sv.events_done;
  out->particles_done = sv.particles_done;
  out->waves = sv.waves;
  out->admission_waits = sv.admission_waits;
  out->graph_launches = sv.graph_launches;
  if (!sv.lat_ms.empty()) {
    std::vector<double> v = sv.lat_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min<size_t>(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    out->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
    out->span_s = std::chrono::duration<double>(sv.t_last - sv.t_first).count();
  }
  return PDR_OK;
}

int pdr_serve_stop(pdr_ctx* ctx) {
  if (!ctx) return fail(PDR_EINVAL, "null context");
  Server* sv = ctx->serve;
  if (!sv) return PDR_OK;
  {
    std::lock_guard<std::mutex> lk(sv->m);
    sv->stop = true;
  }
  sv->cv.notify_one();
  if (sv->th.joinable()) sv->th.join();
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(sv->s_comp);
  for (auto& kv : sv->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  cudaStreamDestroy(sv->s_copy);
  cudaStreamDestroy(sv->s_comp);
  cudaStreamDestroy(sv->s_cap);
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->serve = nullptr;
  }
  delete sv;
  return PDR_OK;
}

}  // extern "C"

// ============================================================ pile-up merging
namespace {

// Poisson(mean) CDF thresholds (the definition in the C header): the CDF
// summed in double from exp(-mean), T[k] = floor(cdf 2^32), the first entry
// at or above 2^32 - 1 becoming 2^32.
int poisson_table(double mean, std::vector<unsigned long long>& T) {
  T.clear();
  double p = std::exp(-mean), cdf = p;
  for (int k = 0; k < 16384; ++k) {
    if (k > 0) {
      p = p * mean / (double)k;
      cdf = cdf + p;
    }
    const double t = std::floor(cdf * 4294967296.0);
    if (t >= 4294967295.0) {
      T.push_back(4294967296ull);
      return PDR_OK;
    }
    T.push_back((unsigned long long)t);
  }
  return fail(PDR_EOVERFLOW, "Poisson table does not end (mean too large)");
}

int pileup_args(pdr_ctx* ctx, const pdr_batch* h, const pdr_pileup* pu) {
  if (!ctx || !h || !pu) return fail(PDR_EINVAL, "null argument");
  if (h->n_events >= (1ull << 31)) return fail(PDR_EINVAL, "n_events must be < 2^31");
  if (h->n_events > 0 && (!h->offsets || !h->pt || !h->eta || !h->phi || !h->mass || !h->pdg || !h->charge))
    return fail(PDR_EINVAL, "null hard-scatter array");
  if (pu->n_pool < 1 || pu->n_pool >= (1ull << 32) || !pu->offsets || !pu->pt || !pu->eta || !pu->phi ||
      !pu->mass || !pu->pdg || !pu->charge)
    return fail(PDR_EINVAL, "empty pool or null pool array");
  if (!(pu->mean >= 0.0) || !(pu->mean <= 4000.0)) return fail(PDR_EOVERFLOW, "mean pile-up outside [0, 4000]");
  if (!(pu->sigma_z >= 0.0) || !std::isfinite(pu->sigma_z) || !(pu->max_z > 0.0) || !std::isfinite(pu->max_z))
    return fail(PDR_EINVAL, "vertex width must be >= 0 and the truncation > 0");
  if (pu->max_z < 0.05 * pu->sigma_z) return fail(PDR_EINVAL, "vertex truncation below 0.05 sigma_z");
  if (!(pu->sigma_t >= 0.0) || !std::isfinite(pu->sigma_t) || !(pu->max_t > 0.0) || !std::isfinite(pu->max_t))
    return fail(PDR_EINVAL, "vertex-time width must be >= 0 and the truncation > 0");
  if (pu->max_t < 0.05 * pu->sigma_t) return fail(PDR_EINVAL, "vertex-time truncation below 0.05 sigma_t");
  return PDR_OK;
}

// Parameter block of a merge; uploads the thresholds when the mean changed.
int pileup_params(pdr_ctx* ctx, const pdr_batch* h, const pdr_pileup* pu, cudaStream_t s, PuParams& p) {
  if (pu->mean != ctx->pu_mean) {
    std::vector<unsigned long long> T;
    int rc = poisson_table(pu->mean, T);
    if (rc) return rc;
    if (T.size() > ctx->pu_cap) {
      if (ctx->pu_T) cudaFree(ctx->pu_T);
      ctx->pu_T = nullptr;
      ctx->pu_cap = 0;
      PDR_CUDA(cudaMalloc(&ctx->pu_T, T.size() * sizeof(unsigned long long)), "pile-up table");
      ctx->pu_cap = (uint32_t)T.size();
    }
    PDR_CUDA(cudaMemcpyAsync(ctx->pu_T, T.data(), T.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, s),
             "pile-up table copy");
    PDR_CUDA(cudaStreamSynchronize(s), "sync");  // T is a host temporary
    ctx->pu_K = (uint32_t)T.size();
    ctx->pu_mean = pu->mean;
  }
  std::memset(&p, 0, sizeof p);
  p.n_events = h->n_events;
  p.n_pool = pu->n_pool;
  p.hoff = h->offsets; p.hpt = h->pt; p.heta = h->eta; p.hphi = h->phi; p.hmass = h->mass; p.hvz = h->vz;
  p.hpdg = h->pdg; p.hcharge = h->charge;
  p.poff = pu->offsets; p.ppt = pu->pt; p.peta = pu->eta; p.pphi = pu->phi; p.pmass = pu->mass;
  p.ppdg = pu->pdg; p.pcharge = pu->charge;
  p.T = ctx->pu_T;
  p.K = ctx->pu_K;
  p.event_base = h->event_index_base;
  p.smear_hs = pu->smear_hs ? 1u : 0u;
  p.sigma_z = (float)pu->sigma_z;
  p.max_z = (float)pu->max_z;
  p.sigma_t = (float)pu->sigma_t;
  p.max_t = (float)pu->max_t;
  fill_round_keys(p.rk, h->seed);
  p.err = ctx->d_err;
  return PDR_OK;
}

}  // namespace

extern "C" {

int pdr_pileup_offsets(pdr_ctx* ctx, const pdr_batch* h, const pdr_pileup* pu, uint64_t* merged_offsets,
                       uint64_t* total, void* stream) {
  NvtxRange nvtx_range("pdr_pileup_offsets");
  int rc = pileup_args(ctx, h, pu);
  if (rc) return rc;
  if (!merged_offsets || !total) return fail(PDR_EINVAL, "null offsets or total");
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->pu_hoff_total) PDR_CUDA(cudaHostAlloc((void**)&ctx->pu_hoff_total, 8, 0), "pinned word");
  PuParams p;
  if ((rc = pileup_params(ctx, h, pu, s, p))) return rc;
  uint64_t* counts = (uint64_t*)ctx->pool.alloc(std::max<uint64_t>(h->n_events, 1) * 8);
  if (!counts) return fail(PDR_ENOMEM, "device pool too small for the pile-up counts");
  p.counts = counts;
  p.moff = merged_offsets;
  cudaError_t e = launch_pileup_count(p, ctx->n_sms, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->pu_hoff_total, merged_offsets + h->n_events, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  ctx->pool.release(counts);
  if (e != cudaSuccess) return cuda_fail(e, "pile-up counting");
  *total = *ctx->pu_hoff_total;
  return PDR_OK;
}

int pdr_pileup_merge(pdr_ctx* ctx, const pdr_batch* h, const pdr_pileup* pu, const uint64_t* merged_offsets,
                     const pdr_particles* out, void* stream) {
  NvtxRange nvtx_range("pdr_pileup_merge");
  int rc = pileup_args(ctx, h, pu);
  if (rc) return rc;
  if (!merged_offsets || !out || !out->pt || !out->eta || !out->phi || !out->mass || !out->vz || !out->pdg ||
      !out->charge)
    return fail(PDR_EINVAL, "null offsets or output array");
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaStream_t s = (cudaStream_t)stream;
  PuParams p;
  if ((rc = pileup_params(ctx, h, pu, s, p))) return rc;
  p.moff = merged_offsets;
  p.opt = out->pt; p.oeta = out->eta; p.ophi = out->phi; p.omass = out->mass; p.ovz = out->vz; p.ovt = out->vt;
  p.opdg = out->pdg; p.ocharge = out->charge;
  PDR_CUDA(launch_pileup_fill(p, ctx->n_sms, s), "pile-up fill");
  return PDR_OK;
}

}  // extern "C"

// ============================================================ post-processing
namespace {

// Filter spec -> kernel conditions (thresholds in the type they are compared in).
int post_conditions(const pdr_filter* f, PostParams& p) {
  if (f->collection > PDR_COLL_CAND) return fail(PDR_EINVAL, "unknown filter collection");
  if (f->combine > PDR_COMBINE_ANY) return fail(PDR_EINVAL, "combine must be all or any");
  if (f->n_conditions > PDR_MAX_CONDITIONS) return fail(PDR_EINVAL, "more than 8 filter conditions");
  p.filtered = 1;
  p.collection = f->collection;
  p.combine = f->combine;
  p.n_cond = f->n_conditions;
  p.compact = f->compact ? 1u : 0u;
  p.update_features = f->update_features ? 1u : 0u;
  for (uint32_t k = 0; k < f->n_conditions; ++k) {
    const pdr_condition& c = f->cond[k];
    PostCond& d = p.cond[k];
    if (c.field > PDR_FIELD_CHARGE) return fail(PDR_EINVAL, "unknown filter field");
    if (c.op > PDR_OP_NOT_IN) return fail(PDR_EINVAL, "unknown filter operator");
    const bool set = c.op == PDR_OP_IN || c.op == PDR_OP_NOT_IN;
    if (c.n_values < 1 || c.n_values > PDR_MAX_VALUES || (!set && c.n_values != 1))
      return fail(PDR_EINVAL, "a comparison takes one value, in / not in 1 to 8");
    d.field = c.field;
    d.op = c.op;
    d.abs = c.abs ? 1u : 0u;
    d.n = c.n_values;
    const bool integer = c.field == PDR_FIELD_PDG || c.field == PDR_FIELD_CHARGE;
    for (uint32_t j = 0; j < c.n_values; ++j) {
      const double v = c.values[j];
      if (integer) {
        if (!(v == std::floor(v)) || v < -2147483648.0 || v > 2147483647.0)
          return fail(PDR_EINVAL, "pdg and charge thresholds must be 32-bit integers");
        d.iv[j] = (int32_t)v;
      } else {
        if (std::isnan(v)) return fail(PDR_EINVAL, "NaN filter threshold");
        d.fv[j] = (float)v;
      }
    }
    if (integer) p.need_gen = 1;
    if (c.field == PDR_FIELD_E) p.need_mass = 1;
  }
  return PDR_OK;
}

}  // namespace

extern "C" int pdr_postprocess(pdr_ctx* ctx, const pdr_batch* b, const pdr_outputs* o, const pdr_filter* f,
                               pdr_features* features, void* stream) {
  NvtxRange nvtx_range("pdr_postprocess");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if ((rc = check_outputs(o))) return rc;
  if (((uintptr_t)o->tracks & 15u) != 0) return fail(PDR_EINVAL, "track records must be 16-byte aligned");
  PostParams p;
  std::memset(&p, 0, sizeof p);
  p.update_features = 1;
  if (f && (rc = post_conditions(f, p))) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  if (b->n_events == 0) return PDR_OK;
  p.n_events = b->n_events;
  p.offsets = b->offsets;
  p.pdg = b->pdg;
  p.charge = b->charge;
  p.mass = b->mass;
  const CardEntry& ce = ctx->cards[b->card_id];
  p.centres = ce.centres;
  p.ntowers[0] = ce.ntowers[0];
  p.ntowers[1] = ce.ntowers[1];
  p.tracks = o->tracks;
  p.towers = o->towers;
  p.eflow = o->eflow;
  p.cands = o->cands;
  p.iso = o->iso;
  p.counts = o->counts;
  p.features = features;
  p.err = ctx->d_err;
  PDR_CUDA(launch_postprocess(p, ctx->n_sms, (cudaStream_t)stream), "post-processing launch");
  return PDR_OK;
}

// ============================================================ impact parameters
namespace {
IPConst ip_const(const CardEntry& ce, const pdr_ip_params* ipp) {
  IPConst c;
  c.kB = ce.kB;
  c.bsign = ce.bsign;
  c.has_field = ce.has_field;
  c.a_d0 = (float)ipp->a_d0; c.b_d0 = (float)ipp->b_d0;
  c.a_z0 = (float)ipp->a_z0; c.b_z0 = (float)ipp->b_z0;
  return c;
}

int check_ip_params(const pdr_ip_params* ipp) {
  if (!ipp) return fail(PDR_EINVAL, "null impact-parameter parameters");
  const double r[4] = {ipp->a_d0, ipp->b_d0, ipp->a_z0, ipp->b_z0};
  for (double v : r)
    if (!(v >= 0.0) || !std::isfinite(v)) return fail(PDR_EINVAL, "impact-parameter resolutions must be >= 0");
  return PDR_OK;
}
}  // namespace

extern "C" int pdr_run_ip(pdr_ctx* ctx, const pdr_batch* b, const pdr_outputs* o, const pdr_ip_params* ipp,
                          pdr_ip* ip, const pdr_launch* l, void* stream) {
  NvtxRange nvtx_range("pdr_run_ip");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if ((rc = check_outputs(o))) return rc;
  if (!ip) return fail(PDR_EINVAL, "null ip array");
  if ((rc = check_ip_params(ipp))) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t max_n = 0;
  if ((rc = batch_max_n(ctx, b, s, &max_n))) return rc;
  static thread_local KParams p;
  Shape S;
  const pdr_batch* bs[1] = {b};
  const pdr_outputs* os[1] = {o};
  if ((rc = prepare_group(ctx, bs, os, 1, plan_launch(ctx, b->card_id, max_n, l), max_n, p, S))) return rc;
  if (p.n_events == 0) return PDR_OK;
  p.seg[0].ip = ip;
  p.seg[0].vx = ipp->vx;
  p.seg[0].vy = ipp->vy;
  p.seg[0].ipc = ip_const(ctx->cards[b->card_id], ipp);
  p.work = work_counter(ctx, s);
  PDR_CUDA(launch_fused(S.team, S.block, p, S.grid, S.smem, s, true), "fused kernel launch (impact parameters)");
  return PDR_OK;
}

extern "C" int pdr_track_ip(pdr_ctx* ctx, const pdr_batch* b, const pdr_outputs* o, const pdr_ip_params* ipp,
                            pdr_ip* ip, void* stream) {
  NvtxRange nvtx_range("pdr_track_ip");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if (!o || !o->tracks || !o->counts || !ipp || !ip) return fail(PDR_EINVAL, "null track, count or ip array");
  if ((rc = check_ip_params(ipp))) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  if (b->n_events == 0) return PDR_OK;
  const CardEntry& ce = ctx->cards[b->card_id];
  IPParams p;
  std::memset(&p, 0, sizeof p);
  p.n_events = b->n_events;
  p.offsets = b->offsets;
  p.pt = b->pt; p.eta = b->eta; p.phi = b->phi; p.vz = b->vz;
  p.vx = ipp->vx; p.vy = ipp->vy;
  p.charge = b->charge;
  p.tracks = o->tracks;
  p.counts = o->counts;
  p.ip = ip;
  p.err = ctx->d_err;
  p.c = ip_const(ce, ipp);
  p.event_base = b->event_index_base;
  fill_round_keys(p.rk, b->seed);
  PDR_CUDA(launch_track_ip(p, ctx->n_sms, (cudaStream_t)stream), "impact-parameter launch");
  return PDR_OK;
}

// ============================================================ jet clustering
extern "C" int pdr_cluster_jets(pdr_ctx* ctx, const pdr_batch* b, const pdr_outputs* o, const pdr_jet_params* jp,
                                pdr_jet* jets, uint32_t* jet_counts, void* stream) {
  NvtxRange nvtx_range("pdr_cluster_jets");
  int rc = check_batch(ctx, b);
  if (rc) return rc;
  if (!jp || !jets || !jet_counts) return fail(PDR_EINVAL, "null parameters or jet arrays");
  if (jp->collection > PDR_JETS_TRUTH) return fail(PDR_EINVAL, "unknown jet collection");
  if (jp->collection == PDR_JETS_PFLOW && (!o || !o->tracks || !o->eflow || !o->counts))
    return fail(PDR_EINVAL, "PFlow jets need the response's tracks, EFlow neutrals and counts");
  if (!(jp->R > 0.0) || !(jp->R <= 10.0)) return fail(PDR_EINVAL, "jet radius must be in (0, 10]");
  if (jp->ee && !(jp->R <= M_PI)) return fail(PDR_EINVAL, "e+e- jet radius must be in (0, pi]");
  if (!std::isfinite(jp->p) || !(jp->pt_min >= 0.0) || !std::isfinite(jp->pt_min))
    return fail(PDR_EINVAL, "bad clustering exponent or pT cut");
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  if (b->n_events == 0) return PDR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const CardEntry& ce = ctx->cards[b->card_id];
  JetParams p;
  std::memset(&p, 0, sizeof p);
  p.n_events = b->n_events;
  p.offsets = b->offsets;
  p.pt = b->pt; p.eta = b->eta; p.phi = b->phi; p.mass = b->mass; p.pdg = b->pdg;
  if (o) { p.tracks = o->tracks; p.eflow = o->eflow; p.counts = o->counts; }
  p.centres = ce.centres;
  p.ntowers[0] = ce.ntowers[0];
  p.ntowers[1] = ce.ntowers[1];
  p.collection = jp->collection;
  p.nconst_min = jp->nconst_min;
  p.p = (float)jp->p;
  p.ee = jp->ee ? 1u : 0u;
  // the pair metric's normalisation: R^2, or |n_i - n_j|^2 at theta = R for e+e-
  const double R2 = jp->ee ? 2.0 * (1.0 - std::cos(jp->R)) : jp->R * jp->R;
  p.R2 = (float)R2;
  p.inv_R2 = (float)(1.0 / R2);
  p.pt_min = (float)jp->pt_min;
  // tiles at least R (plus a rounding margin) wide: rapidity [-6, 6]
  // (clamped beyond), azimuth periodic; at most 32 x 32
  // (e+e-: one tile; the neighbour searches then walk every object)
  const double rw = jp->R * 1.0001;
  p.nty = jp->ee ? 1 : (int32_t)std::min(32.0, std::max(1.0, std::floor(12.0 / rw)));
  int32_t ntp = jp->ee ? 1 : (int32_t)std::min(32.0, std::floor(2.0 * M_PI / rw));
  p.ntp = ntp < 3 ? 1 : ntp;
  p.ntiles = (uint32_t)(p.nty * p.ntp);
  p.y0 = -6.0f;
  p.inv_wy = (float)(p.nty / 12.0);
  p.inv_wp = (float)(p.ntp / (2.0 * M_PI));
  p.jets = jets;
  p.jet_counts = jet_counts;
  p.err = ctx->d_err;
  // size the per-warp workspace from the largest event
  PDR_CUDA(cudaMemsetAsync(ctx->d_word, 0, 4, s), "memset");
  PDR_CUDA(launch_jet_max_objects(p, ctx->d_word, s), "jet sizing kernel");
  PDR_CUDA(cudaMemcpyAsync(ctx->h_word, ctx->d_word, 4, cudaMemcpyDeviceToHost, s), "copy size");
  PDR_CUDA(cudaStreamSynchronize(s), "sync");
  const uint32_t max_n = *ctx->h_word;
  const uint32_t cap = std::max<uint32_t>(32u, (max_n + 31u) & ~31u);
  int smem_max = 0, smem_sm = 0, smem_rsv = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
  cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device);
  // dynamic shared memory of each of two blocks on one SM
  const uint64_t half_sm = std::min<uint64_t>((uint64_t)smem_max,
                                              (uint64_t)std::max(0, smem_sm / 2 - smem_rsv));
  if (cap > 32767u || jet_ws_bytes(cap, jp->ee != 0, p.ntiles) > (uint64_t)smem_max)
    return fail(PDR_EOVERFLOW, "event has more clustering objects than fit in shared memory");
  // The workspace of the largest event sets how many warps share an SM; so
  // events up to 288 objects (most of a batch of a few hundred particles a
  // event) run in a launch sized for them, and only the larger ones in a
  // launch sized for the largest.
  const uint32_t tier = 288;
  const uint32_t caps[2] = {std::min(cap, tier), cap};
  const int n_tiers = cap > tier ? 2 : 1;
  JetParams tp[2];
  uint64_t blocks[2] = {0, 0}, need[2] = {0, 0};
  size_t smem[2] = {0, 0};
  for (int k = 0; k < n_tiers; ++k) {
    tp[k] = p;
    tp[k].cap = caps[k];
    tp[k].min_obj = k == 0 ? 0u : tier + 1u;
    const uint64_t ws = jet_ws_bytes(tp[k].cap, p.ee != 0, p.ntiles);
    // two blocks an SM where the shared memory allows (shorter tails)
    tp[k].warps = (uint32_t)std::min<uint64_t>(16, std::max<uint64_t>(1, half_sm / ws));
    smem[k] = (size_t)(tp[k].warps * ws);
    int per_sm = 0;
    PDR_CUDA(occupancy_cluster(tp[k].warps * 32u, smem[k], &per_sm), "clustering occupancy");
    blocks[k] = std::min<uint64_t>((b->n_events + tp[k].warps - 1) / tp[k].warps,
                                   (uint64_t)ctx->n_sms * (uint64_t)std::max(per_sm, 1));
    // four-momentum scratch: PDR_JET_SCRATCH_DOUBLES per object for every warp of the grid
    need[k] = blocks[k] * tp[k].warps * (uint64_t)tp[k].cap * 8u * PDR_JET_SCRATCH_DOUBLES;
  }
  if (need[0] + need[1] > ctx->jet_scratch_bytes) {
    PDR_CUDA(cudaDeviceSynchronize(), "sync");   // earlier clusterings may still use the scratch
    if (ctx->jet_scratch) cudaFree(ctx->jet_scratch);
    ctx->jet_scratch = nullptr;
    ctx->jet_scratch_bytes = 0;
    PDR_CUDA(cudaMalloc((void**)&ctx->jet_scratch, need[0] + need[1]), "jet scratch");
    ctx->jet_scratch_bytes = need[0] + need[1];
  }
  // The two tiers run on two streams (the caller's and the context's side
  // stream, forked before and joined after), so the larger events' blocks
  // start as the smaller events' blocks drain instead of after the last one.
  if (n_tiers == 2 && !ctx->s_jet) {
    if (cudaStreamCreateWithFlags(&ctx->s_jet, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_jfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_jjoin, cudaEventDisableTiming) != cudaSuccess)
      return fail(PDR_EDEVICE, "cannot create the clustering side stream");
  }
  if (n_tiers == 2) {
    PDR_CUDA(cudaEventRecord(ctx->ev_jfork, s), "fork");
    PDR_CUDA(cudaStreamWaitEvent(ctx->s_jet, ctx->ev_jfork, 0), "fork");
  }
  for (int k = 0; k < n_tiers; ++k) {
    cudaStream_t sk = k == 0 ? s : ctx->s_jet;
    tp[k].scratch = ctx->jet_scratch + (k == 0 ? 0 : need[0] / 8);
    tp[k].next_event = ctx->d_next + k;
    PDR_CUDA(cudaMemsetAsync(tp[k].next_event, 0, 4, sk), "memset");
    PDR_CUDA(launch_cluster(tp[k], (uint32_t)blocks[k], smem[k], sk), "clustering launch");
  }
  if (n_tiers == 2) {
    PDR_CUDA(cudaEventRecord(ctx->ev_jjoin, ctx->s_jet), "join");
    PDR_CUDA(cudaStreamWaitEvent(s, ctx->ev_jjoin, 0), "join");
  }
  return PDR_OK;
}
