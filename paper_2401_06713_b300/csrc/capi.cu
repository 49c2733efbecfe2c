// capi.cu -- the C ABI of libpicasso: context, round driver (Alg. 1) and
// device-memory bookkeeping.  A context holds one string set or a batch of
// independent sets that advance through their rounds together (one launch
// per step for the whole batch).  All device work is launched on the
// context's stream; the host only computes the round parameters of every
// set and reads back sizes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

using namespace picasso;

namespace {
std::atomic<long long> g_launches{0};
// memory requests of the library: pool creations, device allocations from
// the pool, pinned and mapped host allocations
std::atomic<long long> g_mem_requests{0};
void count_request() { g_mem_requests.fetch_add(1, std::memory_order_relaxed); }
}

namespace picasso {
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace picasso

namespace {
// One memory pool per device, owned by the library.  Freed blocks stay
// reserved (release threshold = max) so the next round or context reuses
// them without mapping new pages; picasso_trim_memory hands them back.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[128] = {};

cudaError_t pool_for(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    count_request();
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = ~0ull;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

// Pinned read-back buffers of 16 words, kept for reuse across contexts:
// pinning host memory costs far more than a round, and a context needs
// only one.  picasso_trim_memory returns them.
std::mutex g_pin_mu;
std::vector<int64_t*> g_pin_free;
constexpr size_t kPinWords = 16;

cudaError_t pinned_get(int64_t** out) {
  {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (!g_pin_free.empty()) {
      *out = g_pin_free.back();
      g_pin_free.pop_back();
      return cudaSuccess;
    }
  }
  count_request();
  return cudaMallocHost((void**)out, sizeof(int64_t) * kPinWords);
}

void pinned_put(int64_t* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_pin_free.push_back(p);
}

// Host CSR buffers (budget mode HOST): mapped pinned memory, kept across
// contexts for the same reason; a request takes the largest cached buffer
// if it is big enough.
std::vector<std::pair<int32_t*, int64_t>> g_hcol_free;

cudaError_t hostcol_get(int64_t need, int32_t** out, int64_t* cap) {
  {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    auto best = g_hcol_free.end();
    for (auto it = g_hcol_free.begin(); it != g_hcol_free.end(); ++it)
      if (it->second >= need && (best == g_hcol_free.end() || it->second < best->second)) best = it;
    if (best != g_hcol_free.end()) {
      *out = best->first;
      *cap = best->second;
      g_hcol_free.erase(best);
      return cudaSuccess;
    }
  }
  *out = nullptr;
  *cap = 0;
  count_request();
  cudaError_t e = cudaHostAlloc((void**)out, sizeof(int32_t) * (size_t)std::max<int64_t>(need, 1),
                                cudaHostAllocMapped | cudaHostAllocPortable);
  if (e != cudaSuccess) {
    *out = nullptr;
    return e;
  }
  *cap = need;
  return cudaSuccess;
}

void hostcol_put(int32_t* p, int64_t cap) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_hcol_free.emplace_back(p, cap);
}

void pinned_trim() {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  for (int64_t* p : g_pin_free) cudaFreeHost(p);
  g_pin_free.clear();
  for (auto& b : g_hcol_free) cudaFreeHost(b.first);
  g_hcol_free.clear();
}
}  // namespace

namespace {

struct Ctx {
  picasso_config cfg{};
  // polls of one bounded device wait (cfg.wait_polls, 0 = the default)
  int32_t max_polls() const { return cfg.wait_polls > 0 ? cfg.wait_polls : kMaxPolls; }
  cudaStream_t s = nullptr;
  int dev = 0;
  cudaMemPool_t pool = nullptr;
  int64_t N = 0;
  int32_t q = 0;
  int32_t qw = 1;  // 64-bit words per part of a string: ceil(q / 64); a string is 2 qw words
  const uint64_t* xz_user = nullptr;

  // the sets of the batch (one for a plain context)
  int32_t nsets = 1;
  std::vector<int64_t> soff;        // [nsets+1] global id offsets
  std::vector<uint64_t> seed;       // [nsets]
  std::vector<int64_t> remaining;   // [nsets] |V_l| of every set
  std::vector<int64_t> set_base;    // [nsets] palette base of the next round
  std::vector<SetRound> sets;       // [nsets] this round's parameters
  int64_t* d_soff = nullptr;        // device copy of soff
  SetRound* d_sets = nullptr;       // device copy of sets
  uint32_t* d_hist = nullptr;       // [nsets] per-set counts
  int64_t* d_set_bytes = nullptr;   // [nsets] conflict-structure bytes of every set this round
  std::vector<int64_t> set_peak_bytes;  // [nsets] max over built rounds of those bytes

  int32_t round = 1;
  int64_t n = 0;          // vertices of the round (all sets)
  int32_t* gid = nullptr; // [n] batch-global ids (nullptr in round 1: identity)
  uint64_t* xz = nullptr; // [n][2] (nullptr in round 1: xz_user)
  int32_t* color = nullptr;

  // assign
  bool assigned = false;
  int64_t Ptot = 0, E = 0;
  int32_t Lmax = 0, Lu = 0;
  int64_t* loff = nullptr;
  int32_t* ent_v = nullptr;
  int32_t* lists = nullptr;
  uint32_t* prio = nullptr;
  // the round in coloring order: round-local id t is the t-th vertex in
  // ascending (priority, global id); perm[t] is its place in V_l (ascending
  // global id), gid_r / xz_r its global id and words
  int32_t* perm = nullptr;
  int32_t* gid_r = nullptr;
  uint64_t* xz_r = nullptr;
  uint32_t* bcount = nullptr;  // [P] bucket sizes, when assign counted them
  // build
  bool built = false;
  int64_t nnz = 0, max_bucket = 0;
  int32_t algo_used = 0;
  int64_t* off = nullptr;
  int32_t* col = nullptr;
  int64_t* runoff = nullptr;
  // a round over the byte budget in chunk mode: the count pass's buckets and
  // masks kept for the chunked emit (the runs of one chunk at a time)
  bool chunk_pending = false;
  int64_t *ck_boff = nullptr, *ck_moff = nullptr, *ck_jboff = nullptr;
  int32_t *ck_bmem = nullptr, *ck_ibkt = nullptr;
  uint32_t* ck_rmask = nullptr;
  int32_t round_chunks = 0;  // chunks of all chunked rounds
  // host CSR (budget mode HOST): the columns of a round over the budget live
  // in mapped pinned host memory, kept for the next such round
  int32_t* hcol = nullptr;
  int64_t hcol_cap = 0;
  bool col_host = false;  // c->col points into hcol
  int32_t host_rounds = 0;
  bool nvtx_open = false;  // an NVTX phase range is pushed
  // bit layout (the bit pass): G_c as every bucket's lower blocks of pair
  // bits (rmask at moff), each entry's row address, slot and run length
  // (rinfo) and the members in slot order (bt_bmem entries, bt_bpid vertex
  // ids); the canonical CSR is made from them on request
  bool bits = false;
  int64_t* rinfo = nullptr;
  uint32_t* bt_rmask = nullptr;
  uint32_t* bt_bcount = nullptr;
  int64_t *bt_boff = nullptr, *bt_moff = nullptr;
  int32_t *bt_bmem = nullptr, *bt_bpid = nullptr;
  // color
  bool colored_done = false;
  int64_t n_colored = 0, n_remaining = 0;
  int32_t sweeps = 0;
  uint64_t* state = nullptr;
  uint32_t* flag = nullptr;
  int64_t* pos = nullptr;

  int32_t* d_err = nullptr;
  int64_t* h_buf = nullptr;  // pinned readback buffer [16]
  int32_t sweep_log[kCtlWords] = {};
  int32_t ordered_fallbacks = 0;
  int sticky = PICASSO_OK;

  std::unordered_map<void*, size_t> sizes;
  int64_t cur_bytes = 0, peak_bytes = 0;

  // timing (CUDA events on s): ev[2..5] pair kernels; phase p (assign,
  // build, color, carry, small) ev[6 + 2p] .. ev[7 + 2p], read when the
  // phase comes again or the stats are asked for (no synchronisation of its
  // own: the elapsed time of events long complete)
  static constexpr int kEvents = 16;
  cudaEvent_t ev[kEvents] = {};
  double* phase_acc[5] = {};
  bool phase_pending[5] = {};
  int phase_cur = -1;
  int32_t rounds_done = 0;
  double t_assign = 0, t_build = 0, t_color = 0, t_carry = 0, t_pairs = 0, t_emit = 0;
  int64_t pairs_launches = 0, logical_pairs = 0, tested_pairs = 0, emit_launches = 0, emit_bytes = 0;
  int64_t nnz_total = 0;
  // small-round engine: rounds run, launches that handed a round back, the
  // round it handed back last (the per-round path takes that one); after a
  // CSR overflow the engine stays off for the context
  int32_t small_rounds = 0, small_stops = 0, small_skip_round = 0;
  // a bounded grid barrier that timed out: kernel (1 engine, 2 sweep
  // coloring, 3 dynamic order), its site, round or step, arrivals seen
  int32_t barrier_timeout[4] = {0, 0, 0, 0};
  bool small_off = false;
  double t_small = 0;

  const uint64_t* round_xz() const { return xz ? xz : xz_user; }
};

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return PICASSO_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return PICASSO_ERR_OOM;
  }
  return PICASSO_ERR_CUDA;
}

#define CK(expr)                                    \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) {                        \
      int _st = map_err(_e);                        \
      if (_st == PICASSO_ERR_CUDA) c->sticky = _st; \
      return _st;                                   \
    }                                               \
  } while (0)

#define ST(expr)                       \
  do {                                 \
    int _st = (expr);                  \
    if (_st != PICASSO_OK) return _st; \
  } while (0)

template <class T>
int alloc(Ctx* c, T** p, int64_t count) {
  *p = nullptr;
  const size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
  count_request();
  cudaError_t e = cudaMallocFromPoolAsync((void**)p, bytes, c->pool, c->s);
  if (e != cudaSuccess) {
    *p = nullptr;
    return map_err(e);
  }
  c->sizes[(void*)*p] = bytes;
  c->cur_bytes += (int64_t)bytes;
  if (c->cur_bytes > c->peak_bytes) c->peak_bytes = c->cur_bytes;
  return PICASSO_OK;
}

template <class T>
void release(Ctx* c, T** p) {
  if (*p) {
    auto it = c->sizes.find((void*)*p);
    if (it != c->sizes.end()) {
      c->cur_bytes -= (int64_t)it->second;
      c->sizes.erase(it);
    }
    cudaFreeAsync((void*)*p, c->s);
    *p = nullptr;
  }
}

void free_color(Ctx* c) {
  release(c, &c->state);
  release(c, &c->flag);
  release(c, &c->pos);
  c->colored_done = false;
}

void free_build(Ctx* c) {
  release(c, &c->off);
  if (c->col_host) {
    c->col = nullptr;  // hcol stays with the context
    c->col_host = false;
  } else {
    release(c, &c->col);
  }
  release(c, &c->runoff);
  release(c, &c->rinfo);
  release(c, &c->bt_rmask);
  release(c, &c->bt_bcount);
  release(c, &c->bt_boff);
  release(c, &c->bt_moff);
  release(c, &c->bt_bmem);
  release(c, &c->bt_bpid);
  c->bits = false;
  release(c, &c->ck_boff);
  release(c, &c->ck_moff);
  release(c, &c->ck_jboff);
  release(c, &c->ck_bmem);
  release(c, &c->ck_ibkt);
  release(c, &c->ck_rmask);
  c->chunk_pending = false;
  c->built = false;
  c->nnz = 0;
}

void free_assign(Ctx* c) {
  release(c, &c->bcount);
  release(c, &c->lists);
  release(c, &c->prio);
  release(c, &c->perm);
  release(c, &c->gid_r);
  release(c, &c->xz_r);
  release(c, &c->loff);
  release(c, &c->ent_v);
  c->assigned = false;
}

int check(Ctx* c) {
  if (!c) return PICASSO_ERR_INVALID_ARG;
  if (c->sticky != PICASSO_OK) return c->sticky;
  cudaError_t e = cudaSetDevice(c->dev);
  if (e != cudaSuccess) return map_err(e);
  return PICASSO_OK;
}

// Phase timers: CUDA events on the context's stream, and an NVTX range of
// the phase's name for profilers (a range left open by an error return is
// closed by the next phase).
int phase_index(const char* name) {
  static const char* names[5] = {"assign", "build", "color", "carry", "small"};
  for (int i = 0; i < 5; ++i)
    if (std::strcmp(name, names[i]) == 0) return i;
  return 0;
}

// Fold phase p's pending time into its accumulator (waits for its end
// event, which in the normal flow completed long before).
cudaError_t phase_resolve(Ctx* c, int p) {
  if (!c->phase_pending[p]) return cudaSuccess;
  c->phase_pending[p] = false;
  cudaError_t e = cudaEventSynchronize(c->ev[7 + 2 * p]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev[6 + 2 * p], c->ev[7 + 2 * p]);
  if (e == cudaSuccess) *c->phase_acc[p] += ms;
  return e;
}

cudaError_t phase_resolve_all(Ctx* c) {
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < 5; ++p) {
    const cudaError_t e2 = phase_resolve(c, p);
    if (e == cudaSuccess) e = e2;
  }
  return e;
}

void phase_begin(Ctx* c, const char* name) {
  if (c->nvtx_open) nvtxRangePop();
  nvtxRangePushA(name);
  c->nvtx_open = true;
  const int p = phase_index(name);
  phase_resolve(c, p);  // its events are about to be reused
  c->phase_cur = p;
  cudaEventRecord(c->ev[6 + 2 * p], c->s);
}
cudaError_t phase_end(Ctx* c, double* acc) {
  if (c->nvtx_open) nvtxRangePop();
  c->nvtx_open = false;
  const int p = c->phase_cur < 0 ? 0 : c->phase_cur;
  cudaError_t e = cudaEventRecord(c->ev[7 + 2 * p], c->s);
  c->phase_acc[p] = acc;
  c->phase_pending[p] = e == cudaSuccess;
  c->phase_cur = -1;
  return e;
}
double elapsed(Ctx* c, int a, int b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) return 0.0;
  return ms;
}

// Table I rule: P = max(1, ceil(n num / den)), L = min(P, max(1, ceil(alpha ln n))).
void params_for(const picasso_config& cfg, int64_t n, int64_t* P, int32_t* L) {
  int64_t p = (n * cfg.palette_num + cfg.palette_den - 1) / cfg.palette_den;
  if (p < 1) p = 1;
  double l = std::ceil(cfg.alpha * std::log((double)n));
  int64_t li = (int64_t)l;
  if (li < 1) li = 1;
  if (li > p) li = p;
  *P = p;
  *L = (int32_t)li;
}

// Every set's parameters for the current round from the configuration.
void plan_round(Ctx* c) {
  for (int k = 0; k < c->nsets; ++k) {
    SetRound& sr = c->sets[k];
    sr.seed = c->seed[k];
    sr.base = c->set_base[k];
    sr.P = 0;
    sr.L = 0;
    if (c->remaining[k] > 0) {
      int64_t P;
      int32_t L;
      params_for(c->cfg, c->remaining[k], &P, &L);
      sr.P = P;
      sr.L = L;
    }
  }
}

// Lists of the round from c->sets (P, L, base already set): bucket-color
// offsets, list offsets, entry owners, lists and priorities.
int assign_round(Ctx* c) {
  int64_t cofs = 0;
  int32_t Lmax = 0;
  for (int k = 0; k < c->nsets; ++k) {
    SetRound& sr = c->sets[k];
    if (sr.P > 0 && (sr.L < 1 || sr.L > sr.P)) return PICASSO_ERR_INVALID_ARG;
    if (sr.L > kMaxL) return PICASSO_ERR_UNSUPPORTED;
    sr.cofs = cofs;
    cofs += sr.P;
    Lmax = std::max(Lmax, sr.L);
  }
  if (cofs >= (int64_t(1) << 30)) return PICASSO_ERR_UNSUPPORTED;
  for (int k = 0; k < c->nsets; ++k)
    if (c->sets[k].base + c->sets[k].P > (int64_t)0x7fffffff) return PICASSO_ERR_UNSUPPORTED;
  free_color(c);
  free_build(c);
  free_assign(c);
  c->Ptot = cofs;
  c->Lmax = Lmax;
  const int64_t n = c->n;
  cudaStream_t s = c->s;
  CK(cudaMemcpyAsync(c->d_sets, c->sets.data(), sizeof(SetRound) * c->nsets, cudaMemcpyHostToDevice, s));

  uint32_t* prio_g = nullptr;
  uint32_t* hist = nullptr;
  uint32_t* len = nullptr;
  int64_t* hoff = nullptr;
  void* tmp = nullptr;
  const int nbins = prio_bins_for(n);
  auto done = [&]() {
    release(c, &prio_g);
    release(c, &hist);
    release(c, &len);
    release(c, &hoff);
    release(c, (uint8_t**)&tmp);
  };
  int st = alloc(c, &prio_g, n);
  if (st == PICASSO_OK) st = alloc(c, &hist, nbins);
  if (st == PICASSO_OK) st = alloc(c, &hoff, nbins + 1);
  if (st == PICASSO_OK) st = alloc(c, &len, n);
  if (st == PICASSO_OK) st = alloc(c, (uint8_t**)&tmp, (int64_t)scan_tmp_bytes(n > nbins ? n : nbins));
  if (st == PICASSO_OK) st = alloc(c, &c->perm, n);
  if (st == PICASSO_OK) st = alloc(c, &c->gid_r, n);
  if (st == PICASSO_OK) st = alloc(c, &c->xz_r, 2 * (int64_t)c->qw * n);
  if (st == PICASSO_OK) st = alloc(c, &c->prio, n);
  if (st == PICASSO_OK) st = alloc(c, &c->loff, n + 1);
  if (st != PICASSO_OK) {
    done();
    return st;
  }
  // Coloring order: priorities in V_l order, sorted by (priority, global id);
  // the round's global ids, words and priorities are gathered in that order,
  // so round-local id t is the t-th vertex to be colored.
  cudaError_t e = launch_round_prio(c->round, c->gid, n, c->d_soff, c->nsets, c->d_sets, prio_g, s);
  if (e == cudaSuccess) e = launch_prio_order(prio_g, n, nbins, hist, hoff, tmp, c->perm, s);
  if (e == cudaSuccess)
    e = launch_rank_gather(c->perm, n, c->gid, c->round_xz(), prio_g, c->gid_r, c->xz_r, c->prio, 2 * c->qw, s);
  // list offsets in that order
  if (e == cudaSuccess) {
    if (c->nsets == 1) {
      // one list length: loff[t] = t L, no scan and no readback
      e = launch_strided_offsets(c->loff, n, Lmax, s);
      c->E = n * (int64_t)Lmax;
    } else {
      e = launch_list_offsets(c->gid_r, n, c->d_soff, c->nsets, c->d_sets, len, c->loff, tmp, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_buf, c->loff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) c->E = c->h_buf[0];
    }
  }
  done();
  CK(e);
  // with one list length (a single set) owners follow from e / L
  c->Lu = c->nsets == 1 ? Lmax : 0;
  ST(alloc(c, &c->lists, c->E));
  if (!c->Lu) {
    ST(alloc(c, &c->ent_v, c->E));
    CK(launch_entry_owner(c->loff, n, c->ent_v, s));
  }
  // bucket sizes counted as the lists are drawn when the build will join
  // through buckets (lists of at most 32 colors)
  const int algo = c->cfg.conflict_algo;
  // (more bucket colors than one block's shared memory counts: the build
  // counts them without global atomics otherwise)
  const bool buckets = Lmax <= 32 && c->Ptot < kBucketMaxP && c->Ptot > kHistMaxP &&
                       algo != PICASSO_CONFLICT_ALLPAIRS && !(algo == PICASSO_CONFLICT_AUTO && n <= kSmallRoundAllPairs);
  if (buckets) {
    ST(alloc(c, &c->bcount, c->Ptot));
    CK(cudaMemsetAsync(c->bcount, 0, sizeof(uint32_t) * c->Ptot, s));
  }
  CK(launch_assign_lists(c->round, c->gid_r, n, c->d_soff, c->nsets, c->d_sets, Lmax, c->loff, c->lists, c->prio,
                         c->bcount, s));
  c->assigned = true;
  return PICASSO_OK;
}

int build_conflicts(Ctx* c, bool chunk_ok) {
  const int64_t n = c->n, P = c->Ptot, E = c->E;
  cudaStream_t s = c->s;

  uint32_t *cnt = nullptr, *bcount = nullptr, *bcursor = nullptr, *dmax = nullptr;
  uint32_t *words = nullptr, *rmask = nullptr;
  uint16_t* hist = nullptr;  // per entry range and color: counts, then the ranges before
  int64_t hist_g = 0;
  unsigned long long* dsq = nullptr;
  int64_t *boff = nullptr, *moff = nullptr, *jboff = nullptr;
  int32_t *bmem = nullptr, *ibkt = nullptr, *bpid = nullptr;
  uint4* bxz = nullptr;
  void* tmp = nullptr;
  int st = PICASSO_OK;
  auto cleanup = [&]() {
    release(c, &cnt);
    release(c, &bcount);
    release(c, &bcursor);
    release(c, &hist);
    release(c, &dmax);
    release(c, &dsq);
    release(c, &boff);
    release(c, &bmem);
    release(c, &words);
    release(c, &moff);
    release(c, &jboff);
    release(c, &ibkt);
    release(c, &bxz);
    release(c, &bpid);
    release(c, &rmask);
    release(c, (uint8_t**)&tmp);
  };
#define TRY(expr)           \
  do {                      \
    st = (expr);            \
    if (st != PICASSO_OK) { \
      cleanup();            \
      return st;            \
    }                       \
  } while (0)
#define TRYC(expr)                                \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) {                      \
      st = map_err(_e);                           \
      if (st == PICASSO_ERR_CUDA) c->sticky = st; \
      cleanup();                                  \
      return st;                                  \
    }                                             \
  } while (0)

  const size_t tmp_bytes = scan_tmp_bytes(E > P ? E : P);
  TRY(alloc(c, (uint8_t**)&tmp, (int64_t)tmp_bytes));
  TRY(alloc(c, &cnt, E));
  TRYC(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s));

  int algo = c->cfg.conflict_algo;
  // small rounds: testing all n (n-1) pairs costs less than building buckets
  // (chunk mode keeps small rounds on the bucket join, which can emit by chunk)
  const bool chunking = chunk_ok && c->cfg.byte_budget > 0 && c->cfg.budget_mode == PICASSO_BUDGET_CHUNK &&
                        c->nsets == 1 && c->cfg.color_algo != PICASSO_COLOR_DYNAMIC;
  if (algo == PICASSO_CONFLICT_AUTO && n <= kSmallRoundAllPairs && !chunking) algo = PICASSO_CONFLICT_ALLPAIRS;
  int64_t smax = 0, bucket_pairs = 0;
  if (algo != PICASSO_CONFLICT_ALLPAIRS) {
    // color buckets: sizes, offsets, largest bucket
    TRY(alloc(c, &boff, P + 1));
    TRY(alloc(c, &dmax, 2));
    TRY(alloc(c, &dsq, 1));
    if (c->bcount) {
      bcount = c->bcount;  // counted while the lists were drawn
      c->bcount = nullptr;
    } else if (P <= kHistMaxP) {
      hist_g = bucket_hist_blocks(E);
      TRY(alloc(c, &bcount, P));
      TRY(alloc(c, &hist, hist_g * 2 * ((P + 1) / 2)));
      TRYC(launch_bucket_count(c->lists, E, P, hist, hist_g, bcount, s));
    } else {
      TRY(alloc(c, &bcount, P));
      TRYC(cudaMemsetAsync(bcount, 0, sizeof(uint32_t) * P, s));
      TRYC(launch_bucket_hist(c->lists, E, bcount, s));
    }
    TRYC(launch_bucket_stats(bcount, P, dmax, dsq, s));
    TRYC(cudaMemcpyAsync(c->h_buf, dmax, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TRYC(cudaMemcpyAsync(c->h_buf + 1, dsq, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    TRYC(cudaStreamSynchronize(s));
    smax = (int64_t)(*(uint32_t*)c->h_buf);
    bucket_pairs = c->h_buf[1];
    const bool bucket_ok = smax <= kBucketCap && P < kBucketMaxP && E < (int64_t(1) << 31) &&
                           (c->qw == 1 || wide_mask_fits(smax, c->qw));
    if (algo == PICASSO_CONFLICT_AUTO) algo = bucket_ok ? PICASSO_CONFLICT_BUCKET : PICASSO_CONFLICT_ALLPAIRS;
    if (algo == PICASSO_CONFLICT_BUCKET && !bucket_ok) {
      cleanup();
      return PICASSO_ERR_UNSUPPORTED;
    }
  }
  c->max_bucket = smax;
  c->algo_used = algo;

  ConflictArgs a{};
  a.n = n;
  a.E = E;
  a.Lmax = c->Lmax;
  a.Lu = c->Lu;
  a.P = P;
  a.xz = c->xz_r;
  a.qw = c->qw;
  a.lists = c->lists;
  a.loff = c->loff;
  a.ent_v = c->ent_v;
  a.cnt = cnt;
  a.err = c->d_err;
  // Alg. 2's dynamic order strikes colors from later neighbours' lists too:
  // it needs both directions of every pair
  a.lower = c->cfg.csr_form == PICASSO_CSR_EARLIER && c->cfg.color_algo != PICASSO_COLOR_DYNAMIC ? 1 : 0;

  if (algo == PICASSO_CONFLICT_BUCKET) {
    TRYC(launch_scan_u32(bcount, P, boff, tmp, s));
    TRY(alloc(c, &bmem, E));
    const bool placed = hist != nullptr;  // members in entry order across the ranges
    if (hist) {
      TRYC(launch_bucket_place(c->lists, E, P, hist, hist_g, boff, bmem, s));
      release(c, &hist);
    } else {
      TRY(alloc(c, &bcursor, P));
      TRYC(cudaMemsetAsync(bcursor, 0, sizeof(uint32_t) * P, s));
      TRYC(launch_bucket_fill(c->lists, E, boff, bcursor, bmem, s));
      release(c, &bcursor);
    }
    // the bit layout: EARLIER form, no byte budget, buckets of at most
    // kFusedMax members, strings of one word per part
    // (the bit rows' words, bounded below, must fit rinfo's address field)
    const int64_t wcap = (bucket_pairs + E + 94 * E + 1953 * P) / 64 + 64;
    const bool bitl = a.lower && c->cfg.byte_budget == 0 && smax <= kFusedMax && c->qw == 1 &&
                      wcap < (int64_t(1) << kRinfoAddrBits);
    if (bitl) {
      // sorted buckets, and the members' words and vertex ids in slot order
      TRY(alloc(c, &bxz, E));
      TRY(alloc(c, &bpid, E));
      TRYC(launch_bucket_sort_gather(boff, P, bmem, (int32_t)smax, placed, a, bxz, bpid, s));
    } else {
      TRYC(launch_bucket_sort(boff, P, bmem, c->d_err, (int32_t)smax, placed, s));
    }
    if (bitl) {
      // the bit pass: every bucket's lower blocks of pair bits, no run
      // written.  The blocks' words are allocated from a bound, so nothing
      // is read back before the pass: a bucket of s members has
      // 16 nwb (nwb + 1) <= (s + 31)(s + 63) / 64 words, nwb = ceil(s / 32),
      // and sum s = E, sum s^2 = bucket_pairs + E.
      TRY(alloc(c, &words, P));
      TRY(alloc(c, &moff, P + 1));
      TRYC(launch_bucket_words(bcount, P, 1, words, s));
      TRYC(launch_scan_u32(words, P, moff, tmp, s));
      release(c, &words);
      TRY(alloc(c, &rmask, wcap));
      TRY(alloc(c, &c->rinfo, E));
      // the run total: the context's error block, words 2..3
      unsigned long long* dn = reinterpret_cast<unsigned long long*>(c->d_err + 2);
      TRYC(cudaMemsetAsync(dn, 0, sizeof(unsigned long long), s));
      a.bxz = bxz;
      a.bpid = bpid;
      a.rmask = rmask;
      a.rinfo = c->rinfo;
      a.nnz = dn;
      TRYC(cudaEventRecord(c->ev[2], s));
      TRYC(launch_bucket_bits(a, boff, bmem, moff, (int32_t)smax, c->q, s, c->cfg.sched.bits_blocks_per_sm));
      TRYC(cudaEventRecord(c->ev[3], s));
      TRYC(cudaMemcpyAsync(c->h_buf, dn, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      TRYC(cudaMemcpyAsync(c->h_buf + 1, moff + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      TRYC(cudaStreamSynchronize(s));
      const int64_t nnz = c->h_buf[0], mwords = c->h_buf[1];
      const float ms = (float)elapsed(c, 2, 3);
      c->bt_rmask = rmask;
      c->bt_bcount = bcount;
      c->bt_boff = boff;
      c->bt_moff = moff;
      c->bt_bmem = bmem;
      c->bt_bpid = bpid;
      rmask = nullptr;
      bcount = nullptr;
      boff = moff = nullptr;
      bmem = bpid = nullptr;
      c->bits = true;
      const int64_t csr_bytes = 8 * (n + 1) + 4 * nnz;
      if (c->nsets > 1) {
        std::vector<int64_t> h(c->nsets);
        TRYC(launch_rinfo_lengths(c->rinfo, E, cnt, s));
        TRYC(launch_set_csr_bytes(c->loff, nullptr, cnt, c->gid_r, n, c->d_soff, c->nsets, c->d_set_bytes, s));
        TRYC(cudaMemcpyAsync(h.data(), c->d_set_bytes, sizeof(int64_t) * c->nsets, cudaMemcpyDeviceToHost, s));
        TRYC(cudaStreamSynchronize(s));
        for (int k = 0; k < c->nsets; ++k)
          if (c->remaining[k] > 0) c->set_peak_bytes[k] = std::max(c->set_peak_bytes[k], h[k] + 8);
      } else {
        c->set_peak_bytes[0] = std::max(c->set_peak_bytes[0], csr_bytes);
      }
      // the pass tests the pairs and writes G_c: member words and entry ids
      // read (20 bytes per list entry), the bit rows (4 bytes per word), one
      // row address, slot and run length word per entry (8 bytes)
      c->t_pairs += ms;
      c->pairs_launches += 1;
      c->tested_pairs += bucket_pairs / 2;
      c->t_emit += ms;
      c->emit_launches += 1;
      c->emit_bytes += 28 * E + 4 * mwords;
      for (int k = 0; k < c->nsets; ++k) c->logical_pairs += c->remaining[k] * (c->remaining[k] - 1) / 2;
      cleanup();
      c->nnz = nnz;
      c->nnz_total += nnz;
      c->built = true;
      return PICASSO_OK;
    }
    // mask words: bucket c holds nwb x nwb blocks of 32 words, nwb = ceil(s_c / 32)
    TRY(alloc(c, &words, P));
    TRY(alloc(c, &moff, P + 1));
    TRYC(launch_bucket_words(bcount, P, a.lower, words, s));
    TRYC(launch_scan_u32(words, P, moff, tmp, s));
    TRYC(cudaMemcpyAsync(c->h_buf, moff + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    // emit work items: the 32-row blocks of every bucket
    TRY(alloc(c, &jboff, P + 1));
    TRYC(launch_bucket_jblocks(bcount, P, words, s));
    TRYC(launch_scan_u32(words, P, jboff, tmp, s));
    TRYC(cudaMemcpyAsync(c->h_buf + 3, jboff + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRYC(cudaStreamSynchronize(s));
    const int64_t nwords = c->h_buf[0];
    TRY(alloc(c, &ibkt, c->h_buf[3]));
    TRYC(launch_item_bucket(jboff, P, ibkt, s));
    release(c, &words);
    TRY(alloc(c, &rmask, nwords));
    a.rmask = rmask;
    TRYC(cudaEventRecord(c->ev[2], s));
    TRYC(launch_bucket_mask(a, boff, bmem, moff, (int32_t)smax, c->q, s));
    TRYC(cudaEventRecord(c->ev[3], s));
    c->emit_bytes += 4 * nwords;  // the emit pass reads every run word
  } else {
    TRYC(cudaEventRecord(c->ev[2], s));
    TRYC(launch_allpairs(a, false, s));
    TRYC(cudaEventRecord(c->ev[3], s));
  }
  const int64_t tested = algo == PICASSO_CONFLICT_BUCKET ? bucket_pairs : n * (n - 1);
  release(c, &bcount);

  TRY(alloc(c, &c->runoff, E + 1));
  TRYC(launch_scan_u32(cnt, E, c->runoff, tmp, s));
  release(c, &cnt);
  TRYC(cudaMemcpyAsync(c->h_buf, c->runoff + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRYC(cudaMemcpyAsync(c->h_buf + 2, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  const int64_t nnz = c->h_buf[0];
  if ((int32_t)c->h_buf[2] != 0) {
    cleanup();
    return PICASSO_ERR_INTERNAL;
  }
  const int64_t csr_bytes = 8 * (n + 1) + 4 * nnz;
  if (c->cfg.byte_budget > 0 && csr_bytes > c->cfg.byte_budget) {
    if (chunking && algo == PICASSO_CONFLICT_BUCKET) {
      // the round goes by chunks of coloring order (color_chunked)
      c->ck_boff = boff;
      c->ck_moff = moff;
      c->ck_jboff = jboff;
      c->ck_bmem = bmem;
      c->ck_ibkt = ibkt;
      c->ck_rmask = rmask;
      boff = moff = jboff = nullptr;
      bmem = ibkt = nullptr;
      rmask = nullptr;
      c->t_pairs += elapsed(c, 2, 3);
      c->pairs_launches += 1;
      c->tested_pairs += tested / 2;
      c->logical_pairs += c->remaining[0] * (c->remaining[0] - 1) / 2;
      cleanup();
      c->nnz = nnz;
      c->nnz_total += nnz;
      c->chunk_pending = true;
      return PICASSO_OK;
    }
    if (c->cfg.budget_mode != PICASSO_BUDGET_HOST) {
      cleanup();
      release(c, &c->runoff);
      return PICASSO_ERR_BUDGET;
    }
    // Alg. 3: a conflict graph the device cannot hold goes to host memory.
    // The columns are written to mapped pinned host memory by the emit
    // pass and read from there by the coloring (the row and run offsets
    // stay on the device).
    if (c->hcol_cap < nnz) {
      TRYC(cudaStreamSynchronize(s));
      hostcol_put(c->hcol, c->hcol_cap);
      c->hcol = nullptr;
      c->hcol_cap = 0;
      TRYC(hostcol_get(nnz, &c->hcol, &c->hcol_cap));
    }
    int32_t* dcol = nullptr;
    TRYC(cudaHostGetDevicePointer((void**)&dcol, c->hcol, 0));
    c->col = dcol;
    c->col_host = true;
    c->host_rounds += 1;
  }
  TRY(alloc(c, &c->off, n + 1));
  if (!c->col_host) TRY(alloc(c, &c->col, nnz));
  a.runoff = c->runoff;
  a.col = c->col;
  TRYC(cudaEventRecord(c->ev[4], s));
  if (algo == PICASSO_CONFLICT_BUCKET) {
    TRYC(launch_bucket_emit(a, boff, bmem, moff, jboff, ibkt, c->d_err + 2, 0, n, 0, s));
  } else {
    TRYC(launch_allpairs(a, true, s));
  }
  TRYC(cudaEventRecord(c->ev[5], s));
  TRYC(launch_row_offsets(c->runoff, c->loff, n, c->off, s));
  if (c->nsets > 1) {
    std::vector<int64_t> h(c->nsets);
    TRYC(launch_set_csr_bytes(c->loff, c->runoff, nullptr, c->gid_r, n, c->d_soff, c->nsets, c->d_set_bytes, s));
    TRYC(cudaMemcpyAsync(h.data(), c->d_set_bytes, sizeof(int64_t) * c->nsets, cudaMemcpyDeviceToHost, s));
    TRYC(cudaStreamSynchronize(s));
    for (int k = 0; k < c->nsets; ++k)
      if (c->remaining[k] > 0) c->set_peak_bytes[k] = std::max(c->set_peak_bytes[k], h[k] + 8);
  } else {
    c->set_peak_bytes[0] = std::max(c->set_peak_bytes[0], csr_bytes);
  }
  TRYC(cudaEventSynchronize(c->ev[5]));
  if (algo == PICASSO_CONFLICT_BUCKET) {
    // the mask pass tests every unordered pair of a bucket once; the emit
    // pass streams the words and writes the CSR
    c->t_pairs += elapsed(c, 2, 3);
    c->pairs_launches += 1;
    c->tested_pairs += tested / 2;
    c->t_emit += elapsed(c, 4, 5);
    c->emit_launches += 1;
    c->emit_bytes += 4 * nnz + 4 * E + 8 * E;  // CSR writes, member ids, run offsets
  } else {
    // the all-pairs kernel tests every ordered pair in both passes
    c->t_pairs += elapsed(c, 2, 3) + elapsed(c, 4, 5);
    c->pairs_launches += 2;
    c->tested_pairs += 2 * tested;
  }
  for (int k = 0; k < c->nsets; ++k) c->logical_pairs += c->remaining[k] * (c->remaining[k] - 1) / 2;
  cleanup();
  c->nnz = nnz;
  c->nnz_total += nnz;
  c->built = true;
#undef TRY
#undef TRYC
  return PICASSO_OK;
}

int canonical_bits(Ctx* c);

// The canonical CSR of the current build (the bit layout is converted; the
// other builds already are canonical).
int canonical_csr(Ctx* c) {
  if (c->built && c->bits) return canonical_bits(c);
  return PICASSO_OK;
}

// The canonical CSR of a bit-layout build: run offsets (a scan of the run
// lengths), row offsets, and the emit pass over the bit blocks, which writes
// every row's runs in ascending partner order.  The bit layout is released.
int canonical_bits(Ctx* c) {
  const int64_t n = c->n, E = c->E, P = c->Ptot;
  cudaStream_t s = c->s;
  void* tmp = nullptr;
  uint32_t* words = nullptr;
  uint32_t* lens = nullptr;
  int64_t* jboff = nullptr;
  int32_t* ibkt = nullptr;
  auto fail = [&](int st) {
    release(c, (uint8_t**)&tmp);
    release(c, &words);
    release(c, &lens);
    release(c, &jboff);
    release(c, &ibkt);
    release(c, &c->runoff);
    release(c, &c->off);
    release(c, &c->col);
    return st;
  };
  int st = alloc(c, (uint8_t**)&tmp, (int64_t)scan_tmp_bytes(E > P ? E : P));
  if (st == PICASSO_OK) st = alloc(c, &c->runoff, E + 1);
  if (st == PICASSO_OK) st = alloc(c, &c->off, n + 1);
  if (st == PICASSO_OK) st = alloc(c, &c->col, c->nnz);
  if (st == PICASSO_OK) st = alloc(c, &words, P);
  if (st == PICASSO_OK) st = alloc(c, &jboff, P + 1);
  if (st == PICASSO_OK) st = alloc(c, &lens, E);
  if (st != PICASSO_OK) return fail(st);
  cudaError_t e = launch_rinfo_lengths(c->rinfo, E, lens, s);
  if (e == cudaSuccess) e = launch_scan_u32(lens, E, c->runoff, tmp, s);
  if (e == cudaSuccess) e = launch_row_offsets(c->runoff, c->loff, n, c->off, s);
  if (e == cudaSuccess) e = launch_bucket_jblocks(c->bt_bcount, P, words, s);
  if (e == cudaSuccess) e = launch_scan_u32(words, P, jboff, tmp, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_buf, jboff + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    st = alloc(c, &ibkt, c->h_buf[0] > 0 ? c->h_buf[0] : 1);
    if (st != PICASSO_OK) return fail(st);
    e = launch_item_bucket(jboff, P, ibkt, s);
  }
  if (e == cudaSuccess) {
    ConflictArgs a{};
    a.n = n;
    a.E = E;
    a.Lu = c->Lu;
    a.P = P;
    a.loff = c->loff;
    a.ent_v = c->ent_v;
    a.runoff = c->runoff;
    a.col = c->col;
    a.rmask = c->bt_rmask;
    a.lower = 1;
    a.rowmajor = 1;
    e = launch_bucket_emit(a, c->bt_boff, c->bt_bmem, c->bt_moff, jboff, ibkt, c->d_err + 2, 0, n, 0, s);
  }
  if (e != cudaSuccess) {
    st = map_err(e);
    if (st == PICASSO_ERR_CUDA) c->sticky = st;
    return fail(st);
  }
  release(c, (uint8_t**)&tmp);
  release(c, &words);
  release(c, &jboff);
  release(c, &ibkt);
  release(c, &lens);
  release(c, &c->rinfo);
  release(c, &c->bt_rmask);
  release(c, &c->bt_bcount);
  release(c, &c->bt_boff);
  release(c, &c->bt_moff);
  release(c, &c->bt_bmem);
  release(c, &c->bt_bpid);
  c->bits = false;
  return PICASSO_OK;
}

// Alg. 2's dynamic order (parallel rule, kernels_dynamic.cu): steps until no
// uncolored vertex with a nonempty list is left; one read-back per step.
int color_dynamic(Ctx* c) {
  const int64_t n = c->n;
  cudaStream_t s = c->s;
  if (c->Lmax > 64) return PICASSO_ERR_UNSUPPORTED;
  ST(canonical_csr(c));
  uint64_t* mask = nullptr;
  int32_t *state = nullptr, *colorl = nullptr, *ctl = nullptr, *wa = nullptr, *wb = nullptr, *sel = nullptr,
          *fin = nullptr, *blk = nullptr, *stamp = nullptr, *bstep = nullptr, *parts = nullptr,
          *lng = nullptr;
  void* tmp = nullptr;
  int st = PICASSO_OK;
  auto cleanup = [&]() {
    release(c, &mask);
    release(c, &state);
    release(c, &colorl);
    release(c, &ctl);
    release(c, &wa);
    release(c, &wb);
    release(c, &sel);
    release(c, &fin);
    release(c, &blk);
    release(c, &stamp);
    release(c, &bstep);
    release(c, &parts);
    release(c, &lng);
    release(c, (uint8_t**)&tmp);
  };
#define TRY(expr)           \
  do {                      \
    st = (expr);            \
    if (st != PICASSO_OK) { \
      cleanup();            \
      return st;            \
    }                       \
  } while (0)
#define TRYC(expr)                                \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) {                      \
      st = map_err(_e);                           \
      if (st == PICASSO_ERR_CUDA) c->sticky = st; \
      cleanup();                                  \
      return st;                                  \
    }                                             \
  } while (0)
  free_color(c);
  TRY(alloc(c, &mask, n));
  TRY(alloc(c, &state, n));
  TRY(alloc(c, &colorl, n));
  TRY(alloc(c, &ctl, kDynCtlWords));
  TRY(alloc(c, &wa, n));
  TRY(alloc(c, &wb, n));
  TRY(alloc(c, &sel, n));
  TRY(alloc(c, &fin, n));
  TRY(alloc(c, &blk, n));
  TRY(alloc(c, &stamp, n));
  TRY(alloc(c, &bstep, n));
  TRY(alloc(c, &parts, n));
  TRY(alloc(c, &lng, n));
  TRY(alloc(c, &c->state, n));
  TRY(alloc(c, &c->flag, n));
  TRY(alloc(c, &c->pos, n + 1));
  TRY(alloc(c, (uint8_t**)&tmp, (int64_t)scan_tmp_bytes(n)));
  DynArgs d{};
  d.n = n;
  d.round = c->round;
  d.nsets = c->nsets;
  d.soff = c->d_soff;
  d.sets = c->d_sets;
  d.gid = c->gid_r;
  d.loff = c->loff;
  d.lists = c->lists;
  d.runoff = c->runoff;
  d.col = c->col;
  d.mask = mask;
  d.state = state;
  d.color = colorl;
  d.wa = wa;
  d.wb = wb;
  d.sel = sel;
  d.fin = fin;
  d.blk = blk;
  d.stamp = stamp;
  d.bstep = bstep;
  d.parts = parts;
  d.lng = lng;
  d.ctl = ctl;
  TRYC(launch_dyn_init(d, s));
  TRYC(launch_dyn_all(d, s));
  TRYC(launch_dyn_finish(d, c->state, s));
  TRYC(launch_carry_flags(c->state, n, c->gid_r, c->perm, c->d_soff, c->nsets, c->d_sets, c->color, c->flag, s));
  TRYC(launch_scan_u32(c->flag, n, c->pos, tmp, s));
  TRYC(cudaMemcpyAsync(c->h_buf, c->pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRYC(cudaMemcpyAsync(c->h_buf + 1, ctl + 6, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TRYC(cudaMemcpyAsync(c->h_buf + 2, ctl + 10, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  const int32_t steps = *(const int32_t*)(c->h_buf + 1);
  if (reinterpret_cast<const int32_t*>(c->h_buf + 2)[0] != 0) {
    // a grid barrier of the dynamic order gave up: the launch ended mid-step
    c->barrier_timeout[0] = 3;
    c->barrier_timeout[1] = 0;
    c->barrier_timeout[2] = steps;
    c->barrier_timeout[3] = reinterpret_cast<const int32_t*>(c->h_buf + 2)[1];
    c->sticky = PICASSO_ERR_TIMEOUT;
    cleanup();
    return PICASSO_ERR_TIMEOUT;
  }
  c->sweeps = steps;
  c->n_remaining = c->h_buf[0];
  c->n_colored = n - c->n_remaining;
  c->colored_done = true;
  cleanup();
#undef TRY
#undef TRYC
  return PICASSO_OK;
}

int color_round(Ctx* c) {
  if (c->cfg.color_algo == PICASSO_COLOR_DYNAMIC) return color_dynamic(c);
  const int64_t n = c->n;
  cudaStream_t s = c->s;
  int32_t *wa = nullptr, *wb = nullptr, *wact = nullptr, *nw = nullptr;
  uint16_t* kcur = nullptr;
  uint32_t *rcur = nullptr, *blkw = nullptr, *clist = nullptr;
  int32_t* blk = nullptr;
  void* tmp = nullptr;
  int st = PICASSO_OK;
  auto cleanup = [&]() {
    release(c, &wa);
    release(c, &wb);
    release(c, &wact);
    release(c, &nw);
    release(c, &kcur);
    release(c, &rcur);
    release(c, &blk);
    release(c, &blkw);
    release(c, &clist);
    release(c, (uint8_t**)&tmp);
  };
#define TRY(expr)           \
  do {                      \
    st = (expr);            \
    if (st != PICASSO_OK) { \
      cleanup();            \
      return st;            \
    }                       \
  } while (0)
#define TRYC(expr)                                \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) {                      \
      st = map_err(_e);                           \
      if (st == PICASSO_ERR_CUDA) c->sticky = st; \
      cleanup();                                  \
      return st;                                  \
    }                                             \
  } while (0)
  free_color(c);
  TRY(alloc(c, &c->state, n));
  TRY(alloc(c, &kcur, n));
  TRY(alloc(c, &rcur, n));
  TRY(alloc(c, &blk, n));
  TRY(alloc(c, &blkw, n));
  TRY(alloc(c, &wa, n));
  TRY(alloc(c, &wb, n));
  TRY(alloc(c, &wact, n));
  TRY(alloc(c, (uint8_t**)&tmp, (int64_t)scan_tmp_bytes(n)));
  TRY(alloc(c, &nw, kCtlWords));
  int32_t* ctl = nw;
  ColorArgs a{};
  a.n = n;
  a.lists = c->lists;
  a.loff = c->loff;
  a.runoff = c->runoff;
  if (c->bits) {
    a.rinfo = c->rinfo;
    a.bboff = c->bt_boff;
    a.Lu = c->Lu;
    a.rmask = c->bt_rmask;
    a.bpid = c->bt_bpid;
  }
  a.col = c->col;
  a.state = c->state;
  a.kcur = kcur;
  a.rcur = rcur;
  a.blk = blk;
  a.blkw = blkw;
  a.ranked = 1;  // round-local ids are ranks in coloring order
  if (c->bits) {
    // the ordered pass of the bit layout reads the buckets' masks
    TRY(alloc(c, &clist, 32 * c->Ptot));
    TRYC(cudaMemsetAsync(clist, 0, sizeof(uint32_t) * 32 * c->Ptot, s));
    a.cmask = clist;
  } else {
    TRY(alloc(c, &clist, kClistWords * c->Ptot));
    TRYC(cudaMemsetAsync(clist, 0, sizeof(uint32_t) * kClistWords * c->Ptot, s));
    a.clist = clist;
  }
  a.xz = c->xz_r;
  a.qw = c->qw;
  a.max_polls = c->max_polls();
  // Ordered persistent pass; if one of its bounded waits runs out (ctl[5]),
  // recolor the round with the sweep kernel from a fresh state.  The colors,
  // the carry flags and their prefix sum are enqueued behind the pass, so one
  // synchronisation reads both the pass's status and the uncolored count.
  TRY(alloc(c, &c->flag, n));
  TRY(alloc(c, &c->pos, n + 1));
  auto enqueue_carry = [&]() -> cudaError_t {
    cudaError_t e = launch_carry_flags(c->state, n, c->gid_r, c->perm, c->d_soff, c->nsets, c->d_sets, c->color,
                                       c->flag, s);
    if (e == cudaSuccess) e = launch_scan_u32(c->flag, n, c->pos, tmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_buf, c->pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    return e;
  };
  TRYC(cudaMemsetAsync(ctl, 0, sizeof(int32_t) * kCtlWords, s));
  int32_t sweeps = 0;
  bool need_sweeps = c->cfg.color_algo == PICASSO_COLOR_SWEEP;
  // the ordered pass over runs reads every vertex's starting state (priority,
  // first candidate); the mask pass writes each vertex's final state and
  // reads none
  if (!c->bits && !need_sweeps) TRYC(launch_color_init(a, c->prio, ctl, s));
  if (!need_sweeps) {
    TRYC(launch_color_ordered(a, nullptr, ctl + 5, s, c->bits ? c->cfg.sched.color_blocks_per_sm : 0));
    TRYC(cudaMemcpyAsync(c->sweep_log, ctl, sizeof(int32_t) * 8, cudaMemcpyDeviceToHost, s));
    TRYC(enqueue_carry());
    TRYC(cudaStreamSynchronize(s));
    need_sweeps = c->sweep_log[5] != 0;
    c->ordered_fallbacks += need_sweeps ? 1 : 0;
  }
  if (need_sweeps) {
    TRYC(cudaMemsetAsync(ctl, 0, sizeof(int32_t) * kCtlWords, s));
    TRYC(launch_iota(wa, n, s));  // the first work list: every vertex, in coloring order
    TRYC(launch_color_init(a, c->prio, ctl, s));
    TRYC(launch_color_all(a, wa, wb, wact, ctl, s));
    TRYC(cudaMemcpyAsync(c->sweep_log, ctl, sizeof(int32_t) * kCtlWords, cudaMemcpyDeviceToHost, s));
    TRYC(enqueue_carry());
    TRYC(cudaStreamSynchronize(s));
    sweeps = c->sweep_log[3];
    if (c->sweep_log[kCtlAbort] != 0) {
      // a grid barrier of the sweep kernel gave up: the launch ended mid-sweep
      c->barrier_timeout[0] = 2;
      c->barrier_timeout[1] = 0;
      c->barrier_timeout[2] = sweeps;
      c->barrier_timeout[3] = c->sweep_log[kCtlSeen];
      c->sticky = PICASSO_ERR_TIMEOUT;
      cleanup();
      return PICASSO_ERR_TIMEOUT;
    }
    if (c->sweep_log[4] != 0 || c->sweep_log[0] != 0) {
      cleanup();
      return PICASSO_ERR_INTERNAL;
    }
  }
  c->sweeps = sweeps;
  c->n_remaining = c->h_buf[0];
  c->n_colored = n - c->n_remaining;
  c->colored_done = true;
  cleanup();
#undef TRY
#undef TRYC
  return PICASSO_OK;
}

int carry_round(Ctx* c) {
  const int64_t m = c->n_remaining;
  int32_t* gid2 = nullptr;
  uint64_t* xz2 = nullptr;
  if (m > 0) {
    ST(alloc(c, &gid2, m));
    ST(alloc(c, &xz2, 2 * (int64_t)c->qw * m));
    CK(launch_carry_gather(c->flag, c->pos, c->n, c->gid, c->round_xz(), gid2, xz2, 2 * c->qw, c->s));
  }
  release(c, &c->gid);
  release(c, &c->xz);
  c->gid = gid2;
  c->xz = xz2;
  free_color(c);
  free_build(c);
  free_assign(c);
  // next palette base and remaining vertices of every set
  for (int k = 0; k < c->nsets; ++k) c->set_base[k] = c->sets[k].base + c->sets[k].P;
  if (c->nsets == 1) {
    c->remaining[0] = m;
  } else {
    CK(launch_set_counts(c->gid, m, c->d_soff, c->nsets, c->d_hist, c->s));
    std::vector<uint32_t> h(c->nsets);
    CK(cudaMemcpyAsync(h.data(), c->d_hist, sizeof(uint32_t) * c->nsets, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    for (int k = 0; k < c->nsets; ++k) c->remaining[k] = h[k];
  }
  c->n = m;
  c->round += 1;
  return PICASSO_OK;
}

// Whether picasso_run hands the remaining rounds to the small-round engine.
bool small_eligible(const Ctx* c) {
  const picasso_config& cfg = c->cfg;
  const int64_t nmax = cfg.sched.engine_max_n > 0 ? cfg.sched.engine_max_n : kSmallRoundsMax;
  if (c->n < 1 || c->n > nmax || cfg.small_engine != PICASSO_SMALL_AUTO || c->qw > 2) return false;
  if (cfg.conflict_algo != PICASSO_CONFLICT_AUTO || cfg.color_algo != PICASSO_COLOR_AUTO ||
      cfg.csr_form != PICASSO_CSR_EARLIER)
    return false;
  if (c->small_off || c->round == c->small_skip_round || c->round > cfg.max_rounds) return false;
  const int64_t rounds_left = (int64_t)cfg.max_rounds - c->round + 1;
  for (int k = 0; k < c->nsets; ++k) {
    const int64_t m = c->remaining[k];
    if (m == 0) continue;
    int64_t P;
    int32_t L;
    params_for(cfg, m, &P, &L);
    if (L > kSmallLCap || m * (int64_t)L > kSmallMeanBucket * P) return false;
    // every color the engine can hand out still fits an int32 (the
    // per-round path checks base + P each round)
    if (c->set_base[k] + rounds_left * P > (int64_t)0x7fffffff) return false;
  }
  return true;
}

// The remaining rounds in one cooperative launch (kernels_small.cu); on
// return the context stands between rounds, at the round the engine stopped
// at (no vertex left, the round limit, or a round handed back).
int run_small(Ctx* c) {
  const int64_t n0 = c->n;
  const int ns = c->nsets;
  cudaStream_t s = c->s;
  // sizes at the start bound every later round (P and L grow with n):
  // vertices, bucket colors, list entries, and the words of the bit rows
  int64_t mmax = 0, P0 = 0, E0 = 0;
  for (int k = 0; k < ns; ++k) {
    const int64_t m = c->remaining[k];
    if (m == 0) continue;
    int64_t P;
    int32_t L;
    params_for(c->cfg, m, &P, &L);
    mmax = std::max(mmax, m);
    P0 += P;
    E0 += m * L;
  }
  // the bit rows of a round: a bucket of s <= kSmallBucketCap members has
  // 16 nwb (nwb + 1) <= 9.5 s + 32 words (nwb = ceil(s / 32)); a round's
  // buckets hold at most E0 entries over at most P0 colors
  const int64_t wcap = 10 * E0 + 32 * P0 + 1024;
  std::vector<int2> ptab((size_t)mmax + 1);
  ptab[0] = make_int2(0, 0);
  for (int64_t m = 1; m <= mmax; ++m) {
    int64_t P;
    int32_t L;
    params_for(c->cfg, m, &P, &L);
    ptab[m] = make_int2((int)P, L);
  }
  // per-set words: base, remaining, peak bytes | vertex, color and entry
  // offsets (nsets + 1 each) | seeds
  std::vector<int64_t> hs(7 * (size_t)ns + 3, 0);
  for (int k = 0; k < ns; ++k) {
    hs[k] = c->set_base[k];
    hs[ns + k] = c->remaining[k];
    hs[2 * ns + k] = c->set_peak_bytes[k];
    hs[6 * ns + 3 + k] = (int64_t)c->seed[k];
  }
  constexpr int kPartCap = 2048;
  SmallArgs a{};
  int2* d_ptab = nullptr;
  int64_t* d_sw = nullptr;
  int32_t *gid_a = nullptr, *gid_b = nullptr, *perm = nullptr, *gid_r = nullptr, *lists = nullptr;
  int32_t *err = nullptr, *bmem = nullptr, *brank = nullptr, *ibkt = nullptr, *sid = nullptr, *ent_v = nullptr;
  uint64_t* bxz = nullptr;
  int64_t* iboff = nullptr;
  uint64_t *xz_r = nullptr, *state = nullptr, *key = nullptr;
  int64_t *loff = nullptr, *rinfo = nullptr, *pos = nullptr, *part = nullptr, *ctl = nullptr, *boff = nullptr;
  int64_t *moff = nullptr, *snnz = nullptr;
  uint32_t *rmask = nullptr, *bcnt = nullptr, *bcur = nullptr, *cmask = nullptr, *sbar = nullptr;
  int st = PICASSO_OK;
  auto cleanup = [&]() {
    release(c, &d_ptab);
    release(c, &cmask);
    release(c, &d_sw);
    release(c, &gid_a);
    release(c, &gid_b);
    release(c, &perm);
    release(c, &gid_r);
    release(c, &sid);
    release(c, &lists);
    release(c, &ent_v);
    release(c, &rmask);
    release(c, &moff);
    release(c, &snnz);
    release(c, &err);
    release(c, &xz_r);
    release(c, &state);
    release(c, &key);
    release(c, &loff);
    release(c, &rinfo);
    release(c, &pos);
    release(c, &part);
    release(c, &ctl);
    release(c, &sbar);
    release(c, &bcnt);
    release(c, &bcur);
    release(c, &boff);
    release(c, &bmem);
    release(c, &brank);
    release(c, &ibkt);
    release(c, &bxz);
    release(c, &iboff);
  };
#define TRY(expr)           \
  do {                      \
    st = (expr);            \
    if (st != PICASSO_OK) { \
      cleanup();            \
      return st;            \
    }                       \
  } while (0)
#define TRYC(expr)                                \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) {                      \
      st = map_err(_e);                           \
      if (st == PICASSO_ERR_CUDA) c->sticky = st; \
      cleanup();                                  \
      return st;                                  \
    }                                             \
  } while (0)
  TRY(alloc(c, &d_ptab, mmax + 1));
  TRY(alloc(c, &d_sw, (int64_t)hs.size()));
  TRY(alloc(c, &gid_a, n0));
  TRY(alloc(c, &gid_b, n0));
  TRY(alloc(c, &perm, n0));
  TRY(alloc(c, &gid_r, n0));
  TRY(alloc(c, &sid, n0));
  TRY(alloc(c, &xz_r, 2 * (int64_t)c->qw * n0));
  TRY(alloc(c, &lists, E0));
  TRY(alloc(c, &ent_v, E0));
  TRY(alloc(c, &loff, n0 + 1));
  TRY(alloc(c, &rinfo, E0));
  TRY(alloc(c, &rmask, wcap));
  TRY(alloc(c, &moff, P0 + 1));
  TRY(alloc(c, &snnz, ns));
  TRY(alloc(c, &state, n0));
  TRY(alloc(c, &pos, n0 + 1));
  TRY(alloc(c, &key, n0));
  TRY(alloc(c, &bcnt, P0));
  TRY(alloc(c, &cmask, 32 * P0));
  TRY(alloc(c, &bcur, P0));
  TRY(alloc(c, &boff, P0 + 1));
  TRY(alloc(c, &bmem, E0));
  TRY(alloc(c, &brank, E0));
  TRY(alloc(c, &bxz, 2 * (int64_t)c->qw * E0));
  TRY(alloc(c, &iboff, P0 + 1));
  TRY(alloc(c, &ibkt, E0 / 32 + P0 + 1));
  TRY(alloc(c, &part, kPartCap));
  TRY(alloc(c, &err, 4));
  TRY(alloc(c, &ctl, kSmallCtlWords));
  TRY(alloc(c, &sbar, 2));
  TRYC(cudaMemcpyAsync(d_ptab, ptab.data(), sizeof(int2) * (mmax + 1), cudaMemcpyHostToDevice, s));
  TRYC(cudaMemcpyAsync(d_sw, hs.data(), sizeof(int64_t) * hs.size(), cudaMemcpyHostToDevice, s));
  if (c->gid)
    TRYC(cudaMemcpyAsync(gid_a, c->gid, sizeof(int32_t) * n0, cudaMemcpyDeviceToDevice, s));
  else
    TRYC(launch_iota(gid_a, n0, s));
  int64_t* h = c->h_buf;
  std::memset(h, 0, sizeof(int64_t) * kSmallCtlWords);
  h[0] = n0;
  TRYC(cudaMemcpyAsync(ctl, h, sizeof(int64_t) * kSmallCtlWords, cudaMemcpyHostToDevice, s));
  TRYC(cudaMemsetAsync(err, 0, sizeof(int32_t) * 4, s));
  TRYC(cudaMemsetAsync(sbar, 0, sizeof(uint32_t) * 2, s));
  a.n0 = n0;
  a.round0 = c->round;
  a.max_rounds = c->cfg.max_rounds;
  a.nsets = ns;
  a.soff = c->d_soff;
  a.sbase = d_sw;
  a.srem = d_sw + ns;
  a.speak = d_sw + 2 * ns;
  a.svoff = d_sw + 3 * ns;
  a.scof = d_sw + 4 * ns + 1;
  a.seoff = d_sw + 5 * ns + 2;
  a.sseed = reinterpret_cast<const uint64_t*>(d_sw + 6 * ns + 3);
  a.ptab = d_ptab;
  a.wcap = wcap;
  a.budget = c->cfg.byte_budget;
  a.xz = c->xz_user;
  a.gid_a = gid_a;
  a.gid_b = gid_b;
  a.perm = perm;
  a.gid_r = gid_r;
  a.sid = sid;
  a.xz_r = xz_r;
  a.qw = c->qw;
  a.max_polls = c->max_polls();
  a.lists = lists;
  a.ent_v = ent_v;
  a.loff = loff;
  a.rinfo = rinfo;
  a.rmask = rmask;
  a.moff = moff;
  a.snnz = snnz;
  a.state = state;
  a.pos = pos;
  a.color = c->color;
  a.key = key;
  a.bcnt = bcnt;
  a.bcur = bcur;
  a.cmask = cmask;
  a.boff = boff;
  a.iboff = iboff;
  a.ibkt = ibkt;
  a.bmem = bmem;
  a.brank = brank;
  a.bxz = bxz;
  a.part = part;
  a.err = err;
  a.ctl = ctl;
  a.bar = sbar;
  // rounds of at most cluster_max_n vertices run in one cluster of the
  // largest size that fits (or the schedule's, if smaller)
  static int cl_blocks[3] = {-1, -1, -1};
  if (cl_blocks[c->qw] < 0) cl_blocks[c->qw] = small_cluster_blocks(c->qw);
  const picasso_schedule& sc = c->cfg.sched;
  a.handoff = sc.cluster_max_n == 0 ? kSmallClusterMaxN : sc.cluster_max_n < 0 ? 0 : sc.cluster_max_n;
  // and rounds of at most block_max_n vertices in one block
  a.handoff2 = sc.block_max_n == 0 ? kSmallBlockMaxN : sc.block_max_n < 0 ? 0 : sc.block_max_n;
  int clb = cl_blocks[c->qw];
  if (sc.cluster_blocks > 0) clb = std::min(clb, (int)sc.cluster_blocks);
  TRYC(launch_small_rounds(a, kPartCap, a.handoff > 0 ? clb : 0, sc.engine_blocks_per_sm, s));
  TRYC(cudaMemcpyAsync(h, ctl, sizeof(int64_t) * kSmallCtlWords, cudaMemcpyDeviceToHost, s));
  TRYC(cudaMemcpyAsync(h + kSmallCtlWords, err, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, s));
  TRYC(cudaMemcpyAsync(hs.data(), d_sw, sizeof(int64_t) * 3 * ns, cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  if (reinterpret_cast<const int32_t*>(h + kSmallCtlWords)[3] != 0) {
    // a grid barrier of the engine timed out: the launch ended in the middle
    // of a round, so the context cannot go on
    c->barrier_timeout[0] = 1;
    c->barrier_timeout[1] = (int32_t)h[9];
    c->barrier_timeout[2] = (int32_t)h[10];
    c->barrier_timeout[3] = (int32_t)h[11];
    c->sticky = PICASSO_ERR_TIMEOUT;
    cleanup();
    return PICASSO_ERR_TIMEOUT;
  }
  const int64_t nleft = h[0], rounds = h[1], stop = h[2], parity = h[4];
  const int64_t sum_nnz = h[6], sum_pairs = h[7];
  // V_l of the round the engine stopped at, and its words
  int32_t* gid2 = nullptr;
  uint64_t* xz2 = nullptr;
  if (nleft > 0) {
    TRY(alloc(c, &gid2, nleft));
    st = alloc(c, &xz2, 2 * (int64_t)c->qw * nleft);
    if (st != PICASSO_OK) {
      release(c, &gid2);
      cleanup();
      return st;
    }
    cudaError_t e = cudaMemcpyAsync(gid2, parity ? gid_b : gid_a, sizeof(int32_t) * nleft, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_gather_xz(c->xz_user, gid2, nleft, xz2, 2 * c->qw, s);
    if (e != cudaSuccess) {
      release(c, &gid2);
      release(c, &xz2);
    }
    TRYC(e);
  }
  release(c, &c->gid);
  release(c, &c->xz);
  c->gid = gid2;
  c->xz = xz2;
  c->n = nleft;
  for (int k = 0; k < ns; ++k) {
    c->set_base[k] = hs[k];
    c->remaining[k] = hs[ns + k];
    c->set_peak_bytes[k] = hs[2 * ns + k];
  }
  c->round += (int32_t)rounds;
  c->rounds_done += (int32_t)rounds;
  c->small_rounds += (int32_t)rounds;
  c->nnz_total += sum_nnz;
  c->logical_pairs += sum_pairs;
  if (stop == kSmallTimeout || stop == kSmallOverflow) {
    c->small_stops += 1;
    c->small_skip_round = c->round;
    c->small_off = stop == kSmallOverflow;
  }
  cleanup();
#undef TRY
#undef TRYC
  return PICASSO_OK;
}

// A round whose CSR exceeds the byte budget (chunk mode): the vertices in
// coloring order are cut into chunks whose own CSR rows fit the budget (8
// bytes per row + 1, 4 per run entry); chunk by chunk the rows are emitted
// and colored, earlier chunks' colors already final.  In the EARLIER form a
// row only lists earlier neighbours, so each chunk's coloring is exact.
int color_chunked(Ctx* c) {
  const int64_t n = c->n;
  const int64_t budget = c->cfg.byte_budget;
  cudaStream_t s = c->s;
  uint16_t* kcur = nullptr;
  uint32_t *rcur = nullptr, *blkw = nullptr, *clist = nullptr;
  int32_t *blk = nullptr, *ctl = nullptr, *colk = nullptr;
  void* tmp = nullptr;
  int st = PICASSO_OK;
  auto cleanup = [&]() {
    release(c, &kcur);
    release(c, &rcur);
    release(c, &blkw);
    release(c, &clist);
    release(c, &blk);
    release(c, &ctl);
    release(c, &colk);
    release(c, (uint8_t**)&tmp);
  };
#define TRY(expr)           \
  do {                      \
    st = (expr);            \
    if (st != PICASSO_OK) { \
      cleanup();            \
      return st;            \
    }                       \
  } while (0)
#define TRYC(expr)                                \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) {                      \
      st = map_err(_e);                           \
      if (st == PICASSO_ERR_CUDA) c->sticky = st; \
      cleanup();                                  \
      return st;                                  \
    }                                             \
  } while (0)
  // row offsets give every chunk's bytes: rows [lo, hi) take
  // 8 (hi - lo + 1) + 4 (off[hi] - off[lo])
  TRY(alloc(c, &c->off, n + 1));
  TRYC(launch_row_offsets(c->runoff, c->loff, n, c->off, s));
  std::vector<int64_t> off((size_t)n + 1);
  TRYC(cudaMemcpyAsync(off.data(), c->off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  free_color(c);
  TRY(alloc(c, &c->state, n));
  TRY(alloc(c, &kcur, n));
  TRY(alloc(c, &rcur, n));
  TRY(alloc(c, &blk, n));
  TRY(alloc(c, &blkw, n));
  TRY(alloc(c, &ctl, kCtlWords));
  TRY(alloc(c, &clist, kClistWords * c->Ptot));
  TRY(alloc(c, &c->flag, n));
  TRY(alloc(c, &c->pos, n + 1));
  TRY(alloc(c, (uint8_t**)&tmp, (int64_t)scan_tmp_bytes(n)));
  TRYC(cudaMemsetAsync(clist, 0, sizeof(uint32_t) * kClistWords * c->Ptot, s));
  TRYC(cudaMemsetAsync(ctl, 0, sizeof(int32_t) * kCtlWords, s));
  ColorArgs a{};
  a.n = n;
  a.lists = c->lists;
  a.loff = c->loff;
  a.runoff = c->runoff;
  a.state = c->state;
  a.kcur = kcur;
  a.rcur = rcur;
  a.blk = blk;
  a.blkw = blkw;
  a.ranked = 1;
  a.clist = clist;
  a.xz = c->xz_r;
  a.qw = c->qw;
  a.max_polls = c->max_polls();
  TRYC(launch_color_init(a, c->prio, ctl, s));
  ConflictArgs ca{};
  ca.n = n;
  ca.E = c->E;
  ca.Lmax = c->Lmax;
  ca.Lu = c->Lu;
  ca.P = c->Ptot;
  ca.xz = c->xz_r;
  ca.qw = c->qw;
  ca.lists = c->lists;
  ca.loff = c->loff;
  ca.ent_v = c->ent_v;
  ca.err = c->d_err;
  ca.lower = 1;
  ca.rmask = c->ck_rmask;
  ca.runoff = c->runoff;
  int64_t lo = 0;
  int64_t peak = 0;
  int32_t chunks = 0;
  while (lo < n) {
    int64_t hi = lo;
    while (hi < n && 8 * (hi + 1 - lo + 1) + 4 * (off[hi + 1] - off[lo]) <= budget) ++hi;
    if (hi == lo) {
      // one vertex's rows alone exceed the budget
      cleanup();
      return PICASSO_ERR_BUDGET;
    }
    const int64_t cnnz = off[hi] - off[lo];
    TRY(alloc(c, &colk, cnnz));
    ca.col = colk;
    TRYC(launch_bucket_emit(ca, c->ck_boff, c->ck_bmem, c->ck_moff, c->ck_jboff, c->ck_ibkt, c->d_err + 2, lo, hi,
                            off[lo], s));
    a.col = colk;
    a.cbase = off[lo];
    a.v0 = lo;
    a.n = hi - lo;
    TRYC(launch_color_ordered(a, nullptr, ctl + 5, s));
    TRYC(cudaMemcpyAsync(c->h_buf, ctl + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TRYC(cudaStreamSynchronize(s));
    if (*(int32_t*)c->h_buf != 0) {
      cleanup();
      return PICASSO_ERR_TIMEOUT;
    }
    release(c, &colk);
    peak = std::max(peak, 8 * (hi - lo + 1) + 4 * cnnz);
    ++chunks;
    lo = hi;
  }
  c->set_peak_bytes[0] = std::max(c->set_peak_bytes[0], peak);
  c->round_chunks += chunks;
  TRYC(launch_carry_flags(c->state, n, c->gid_r, c->perm, c->d_soff, c->nsets, c->d_sets, c->color, c->flag, s));
  TRYC(launch_scan_u32(c->flag, n, c->pos, tmp, s));
  TRYC(cudaMemcpyAsync(c->h_buf, c->pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  c->sweeps = 0;
  c->n_remaining = c->h_buf[0];
  c->n_colored = n - c->n_remaining;
  c->colored_done = true;
  cleanup();
#undef TRY
#undef TRYC
  return PICASSO_OK;
}

int validate_cfg(const picasso_config* cfg) {
  if (cfg->palette_num < 1 || cfg->palette_den < 1 || cfg->palette_num > (int64_t(1) << 32) ||
      cfg->palette_den > (int64_t(1) << 32) || !(cfg->alpha > 0.0) || !std::isfinite(cfg->alpha) ||
      cfg->max_rounds < 1 || cfg->byte_budget < 0 || cfg->conflict_algo < 0 || cfg->conflict_algo > 2 ||
      cfg->color_algo < 0 || cfg->color_algo > 2 || cfg->csr_form < 0 || cfg->csr_form > 1 ||
      cfg->small_engine < 0 || cfg->small_engine > 1 || cfg->budget_mode < 0 || cfg->budget_mode > 2 ||
      cfg->wait_polls < 0 || cfg->wait_polls > (1 << 30))
    return PICASSO_ERR_INVALID_ARG;
  const picasso_schedule& sc = cfg->sched;
  const int cb = sc.cluster_blocks;
  if (sc.engine_blocks_per_sm < 0 || sc.engine_blocks_per_sm > 2 || sc.cluster_max_n < -1 ||
      sc.cluster_max_n > kSmallRoundsMax || !(cb == 0 || cb == 2 || cb == 4 || cb == 8 || cb == 16) ||
      sc.bits_blocks_per_sm < 0 || sc.bits_blocks_per_sm > 4 || sc.color_blocks_per_sm < 0 ||
      sc.color_blocks_per_sm > 8 || sc.engine_max_n < 0 || sc.engine_max_n > kSmallRoundsMax ||
      sc.block_max_n < -1 || sc.block_max_n > kSmallRoundsMax)
    return PICASSO_ERR_INVALID_ARG;
  return PICASSO_OK;
}

int init_common(void** out, const picasso_config* cfg, const uint64_t* d_xz, const int64_t* h_soff, int32_t nsets,
                const uint64_t* h_seeds, int32_t q, void* stream) {
  if (!out || !cfg || !d_xz || !h_soff || nsets < 1) return PICASSO_ERR_INVALID_ARG;
  *out = nullptr;
  const int64_t n = h_soff[nsets];
  if (h_soff[0] != 0 || n < 1 || n >= (int64_t(1) << 30) || q < 1) return PICASSO_ERR_INVALID_ARG;
  for (int k = 0; k < nsets; ++k)
    if (h_soff[k + 1] < h_soff[k]) return PICASSO_ERR_INVALID_ARG;
  if (q > kMaxQ) return PICASSO_ERR_UNSUPPORTED;
  ST(validate_cfg(cfg));
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return PICASSO_ERR_OOM;
  c->cfg = *cfg;
  c->s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e == cudaSuccess) e = pool_for(c->dev, &c->pool);
  if (e != cudaSuccess) {
    delete c;
    return map_err(e);
  }
  c->N = n;
  c->q = q;
  c->qw = (q + 63) / 64;
  c->xz_user = d_xz;
  c->n = n;
  c->nsets = nsets;
  c->soff.assign(h_soff, h_soff + nsets + 1);
  c->seed.resize(nsets);
  c->remaining.resize(nsets);
  c->set_base.assign(nsets, 0);
  c->set_peak_bytes.assign(nsets, 0);
  c->sets.assign(nsets, SetRound{});
  for (int k = 0; k < nsets; ++k) {
    c->seed[k] = h_seeds ? h_seeds[k] : cfg->seed + (uint64_t)k;
    c->remaining[k] = h_soff[k + 1] - h_soff[k];
  }
  e = pinned_get(&c->h_buf);
  if (e != cudaSuccess) {
    delete c;
    return map_err(e);
  }
  int st = PICASSO_OK;
  for (int i = 0; i < Ctx::kEvents && st == PICASSO_OK; ++i) st = map_err(cudaEventCreate(&c->ev[i]));
  if (st == PICASSO_OK) st = alloc(c, &c->color, n);
  if (st == PICASSO_OK) st = alloc(c, &c->d_err, 4);
  if (st == PICASSO_OK) st = alloc(c, &c->d_soff, nsets + 1);
  if (st == PICASSO_OK) st = alloc(c, &c->d_sets, nsets);
  if (st == PICASSO_OK) st = alloc(c, &c->d_hist, nsets);
  if (st == PICASSO_OK) st = alloc(c, &c->d_set_bytes, nsets);
  if (st == PICASSO_OK)
    st = map_err(cudaMemcpyAsync(c->d_soff, c->soff.data(), sizeof(int64_t) * (nsets + 1), cudaMemcpyHostToDevice,
                                 c->s));
  if (st == PICASSO_OK) st = map_err(launch_fill_i32(c->color, n, -1, c->s));
  if (st == PICASSO_OK) st = map_err(cudaStreamSynchronize(c->s));
  if (st != PICASSO_OK) {
    release(c, &c->color);
    release(c, &c->d_err);
    release(c, &c->d_soff);
    release(c, &c->d_sets);
    release(c, &c->d_hist);
    release(c, &c->d_set_bytes);
    for (int i = 0; i < Ctx::kEvents; ++i)
      if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    pinned_put(c->h_buf);
    delete c;
    return st;
  }
  *out = c;
  return PICASSO_OK;
}

}  // namespace

namespace picasso {
// *diff (zeroed here) = 1 if a and b differ somewhere in [0, n).
__global__ void k_count_diff(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t n,
                             int32_t* __restrict__ diff) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) *diff = 1;
}
cudaError_t launch_count_diff(const int32_t* a, const int32_t* b, int64_t n, int32_t* diff, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(diff, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 8);
  k_count_diff<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a, b, n, diff);
  count_launches(1);
  return cudaGetLastError();
}
int64_t debug_grid(int64_t blocks) {
  static const int64_t div = [] {
    const char* e = std::getenv("PICASSO_GRID_DIVISOR");
    const long long d = e ? std::atoll(e) : 1;
    return (int64_t)(d > 1 ? d : 1);
  }();
  const int64_t b = blocks / div;
  return b > 0 ? b : 1;
}
}  // namespace picasso

extern "C" {

int picasso_config_default(picasso_config* cfg) {
  if (!cfg) return PICASSO_ERR_INVALID_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->seed = 0;
  cfg->palette_num = 1;
  cfg->palette_den = 8;
  cfg->alpha = 2.0;
  cfg->conflict_algo = PICASSO_CONFLICT_AUTO;
  cfg->max_rounds = 100000;
  cfg->byte_budget = 0;
  cfg->color_algo = PICASSO_COLOR_AUTO;
  return PICASSO_OK;
}

int picasso_pack(const uint8_t* d_codes, int64_t n, int32_t q, uint64_t* d_xz, void* stream) {
  if (n < 0 || q < 1 || q > kMaxQ) return q > kMaxQ ? PICASSO_ERR_UNSUPPORTED : PICASSO_ERR_INVALID_ARG;
  if (n > 0 && (!d_codes || !d_xz)) return PICASSO_ERR_INVALID_ARG;
  return map_err(launch_pack(d_codes, n, q, d_xz, (cudaStream_t)stream));
}

int picasso_philox_draws(uint64_t seed, int32_t round, int64_t gid, uint32_t tag, uint32_t i0, int32_t count,
                         uint32_t* d_out, void* stream) {
  if (count < 0 || (count > 0 && !d_out) || tag > 255u) return PICASSO_ERR_INVALID_ARG;
  return map_err(launch_philox_draws(seed, round, gid, tag, i0, count, d_out, (cudaStream_t)stream));
}

int picasso_init(void** out, const picasso_config* cfg, const uint64_t* d_xz, int64_t n, int32_t q, void* stream) {
  if (!cfg) return PICASSO_ERR_INVALID_ARG;
  const int64_t soff[2] = {0, n};
  const uint64_t seed = cfg->seed;
  return init_common(out, cfg, d_xz, soff, 1, &seed, q, stream);
}

int picasso_init_batch(void** out, const picasso_config* cfg, const uint64_t* d_xz, const int64_t* h_set_offsets,
                       int32_t nsets, const uint64_t* h_seeds, int32_t q, void* stream) {
  return init_common(out, cfg, d_xz, h_set_offsets, nsets, h_seeds, q, stream);
}

int picasso_round_params(void* ctx, int64_t* P, int32_t* L, int64_t* base) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (c->n == 0) return PICASSO_ERR_STATE;
  if (c->nsets != 1) return PICASSO_ERR_STATE;
  int64_t p;
  int32_t l;
  params_for(c->cfg, c->n, &p, &l);
  if (P) *P = p;
  if (L) *L = l;
  if (base) *base = c->set_base[0];
  return PICASSO_OK;
}

int picasso_assign_lists(void* ctx, int64_t P, int32_t L, int64_t base) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (c->n == 0 || c->nsets != 1) return PICASSO_ERR_STATE;
  if (P < 1 || L < 1 || L > P || base < 0 || base + P > (int64_t)0x7fffffff) return PICASSO_ERR_INVALID_ARG;
  if (L > kMaxL || P >= (int64_t(1) << 30)) return PICASSO_ERR_UNSUPPORTED;
  SetRound& sr = c->sets[0];
  sr.seed = c->seed[0];
  sr.P = P;
  sr.L = L;
  sr.base = base;
  phase_begin(c, "assign");
  ST(assign_round(c));
  CK(phase_end(c, &c->t_assign));
  return PICASSO_OK;
}

int picasso_build_conflicts(void* ctx, picasso_csr* out) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!c->assigned) return PICASSO_ERR_STATE;
  free_color(c);
  free_build(c);
  phase_begin(c, "build");
  ST(build_conflicts(c, false));
  CK(phase_end(c, &c->t_build));
  if (out) {
    ST(canonical_csr(c));
    out->d_off = c->off;
    out->d_col = c->col;
    out->n_rows = c->n;
    out->nnz = c->nnz;
  }
  return PICASSO_OK;
}

int picasso_color(void* ctx, int64_t* n_colored) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!c->built) return PICASSO_ERR_STATE;
  phase_begin(c, "color");
  ST(color_round(c));
  CK(phase_end(c, &c->t_color));
  if (n_colored) *n_colored = c->n_colored;
  return PICASSO_OK;
}

int picasso_carry(void* ctx, int64_t* n_remaining) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!c->colored_done) return PICASSO_ERR_STATE;
  phase_begin(c, "carry");
  ST(carry_round(c));
  CK(phase_end(c, &c->t_carry));
  c->rounds_done += 1;
  if (n_remaining) *n_remaining = c->n;
  return PICASSO_OK;
}

int picasso_round(void* ctx, int64_t* n_remaining) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (c->n == 0) {
    if (n_remaining) *n_remaining = 0;
    return PICASSO_OK;
  }
  plan_round(c);
  phase_begin(c, "assign");
  ST(assign_round(c));
  CK(phase_end(c, &c->t_assign));
  free_color(c);
  free_build(c);
  phase_begin(c, "build");
  ST(build_conflicts(c, true));
  CK(phase_end(c, &c->t_build));
  if (c->chunk_pending) {
    phase_begin(c, "color");
    ST(color_chunked(c));
    CK(phase_end(c, &c->t_color));
  } else {
    ST(picasso_color(ctx, nullptr));
  }
  return picasso_carry(ctx, n_remaining);
}

int picasso_run(void* ctx, int32_t* d_color_out, int32_t* n_rounds) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  while (c->n > 0) {
    if (c->round > c->cfg.max_rounds) return PICASSO_ERR_INTERNAL;
    if (small_eligible(c)) {
      phase_begin(c, "small");
      ST(run_small(c));
      CK(phase_end(c, &c->t_small));
      continue;
    }
    ST(picasso_round(ctx, nullptr));
  }
  if (d_color_out) ST(picasso_get_colors(ctx, d_color_out));
  if (n_rounds) *n_rounds = c->round - 1;
  return PICASSO_OK;
}

int picasso_color_host(const picasso_config* cfg, const uint8_t* h_codes, int64_t n, int32_t q,
                       int32_t* h_colors, int32_t* n_rounds, void* stream) {
  if (!cfg || !h_codes || !h_colors || n < 1 || n >= (int64_t(1) << 30) || q < 1) return PICASSO_ERR_INVALID_ARG;
  if (q > kMaxQ) return PICASSO_ERR_UNSUPPORTED;
  ST(validate_cfg(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaMemPool_t pool;
  {
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = pool_for(dev, &pool);
    if (ce != cudaSuccess) return map_err(ce);
  }
  const int64_t words = 2 * (int64_t)((q + 63) / 64);
  uint8_t* d_codes = nullptr;
  uint64_t* d_xz = nullptr;
  int32_t* d_colors = nullptr;
  void* ctx = nullptr;
  auto done = [&](int st) {
    if (ctx) picasso_destroy(ctx);
    if (d_codes) cudaFreeAsync(d_codes, s);
    if (d_xz) cudaFreeAsync(d_xz, s);
    if (d_colors) cudaFreeAsync(d_colors, s);
    cudaStreamSynchronize(s);
    return st;
  };
  cudaError_t e = cudaMallocFromPoolAsync((void**)&d_codes, (size_t)n * q, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&d_xz, sizeof(uint64_t) * words * n, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&d_colors, sizeof(int32_t) * n, pool, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_codes, h_codes, (size_t)n * q, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_pack(d_codes, n, q, d_xz, s);
  if (e != cudaSuccess) return done(map_err(e));
  int st = picasso_init(&ctx, cfg, d_xz, n, q, stream);
  if (st == PICASSO_OK) st = picasso_run(ctx, d_colors, n_rounds);
  if (st != PICASSO_OK) return done(st);
  e = cudaMemcpyAsync(h_colors, d_colors, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return done(map_err(e));
}

int picasso_autotune(const picasso_config* cfg, const uint64_t* d_xz, const int64_t* h_set_offsets,
                     int32_t nsets, const uint64_t* h_seeds, int32_t q, int32_t reps, picasso_schedule* best,
                     double* best_ms, double* start_ms, void* stream) {
  if (!cfg || !d_xz || !h_set_offsets || nsets < 1 || reps < 1 || reps > 64) return PICASSO_ERR_INVALID_ARG;
  ST(validate_cfg(cfg));
  const int64_t n = h_set_offsets[nsets];
  if (h_set_offsets[0] != 0 || n < 1 || n >= (int64_t(1) << 30)) return PICASSO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaMemPool_t pool;
  {
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = pool_for(dev, &pool);
    if (ce != cudaSuccess) return map_err(ce);
  }
  int32_t *ref = nullptr, *out = nullptr, *diff = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](int st) {
    if (ref) cudaFreeAsync(ref, s);
    if (out) cudaFreeAsync(out, s);
    if (diff) cudaFreeAsync(diff, s);
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
  };
  cudaError_t e = cudaMallocFromPoolAsync((void**)&ref, sizeof(int32_t) * n, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&out, sizeof(int32_t) * n, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&diff, sizeof(int32_t), pool, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return done(map_err(e));
  bool have_ref = false;
  // one whole run under `sc` into `dst`, its time on the stream in *ms
  auto run = [&](const picasso_schedule& sc, int32_t* dst, float* ms) -> int {
    picasso_config cf = *cfg;
    cf.sched = sc;
    void* ctx = nullptr;
    cudaError_t ce = cudaEventRecord(e0, s);
    if (ce != cudaSuccess) return map_err(ce);
    int st = init_common(&ctx, &cf, d_xz, h_set_offsets, nsets, h_seeds, q, stream);
    if (st == PICASSO_OK) st = picasso_run(ctx, dst, nullptr);
    if (ctx) {
      const int st2 = picasso_destroy(ctx);
      if (st == PICASSO_OK) st = st2;
    }
    if (st != PICASSO_OK) return st;
    ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, e0, e1);
    return map_err(ce);
  };
  // median time of `reps` runs after one untimed run; every run's colors
  // must equal the first run's (a schedule never changes a result)
  auto measure = [&](const picasso_schedule& sc, double* med) -> int {
    float ms = 0.f;
    std::vector<float> t;
    for (int r = 0; r <= reps; ++r) {
      ST(run(sc, have_ref ? out : ref, &ms));
      if (have_ref) {
        int32_t h = 0;
        cudaError_t ce = launch_count_diff(ref, out, n, diff, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, diff, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return map_err(ce);
        if (h != 0) return PICASSO_ERR_INTERNAL;
      }
      have_ref = true;
      if (r > 0) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *med = t[t.size() / 2];
    return PICASSO_OK;
  };
  picasso_schedule cur = cfg->sched;
  double t_cur = 0;
  int st = measure(cur, &t_cur);
  if (st != PICASSO_OK) return done(st);
  if (start_ms) *start_ms = t_cur;
  // coordinate descent: one field at a time over its candidates; a
  // candidate replaces the best only if it is at least 1 % faster
  struct Field {
    int32_t picasso_schedule::*f;
    int32_t cand[4];
    int nc;
  };
  const Field fields[] = {{&picasso_schedule::engine_max_n, {16384, 8192, 4096}, 3},
                          {&picasso_schedule::engine_blocks_per_sm, {1, 2}, 2},
                          {&picasso_schedule::cluster_max_n, {-1, 512, 2048, 8192}, 4},
                          {&picasso_schedule::cluster_blocks, {16, 8}, 2},
                          {&picasso_schedule::block_max_n, {-1, 64, 256, 1024}, 4},
                          {&picasso_schedule::bits_blocks_per_sm, {4, 3, 2}, 3},
                          {&picasso_schedule::color_blocks_per_sm, {6, 4, 3}, 3}};
  for (const Field& fd : fields) {
    picasso_schedule base = cur;
    for (int k = 0; k < fd.nc; ++k) {
      if (base.*(fd.f) == fd.cand[k]) continue;
      picasso_schedule trial = base;
      trial.*(fd.f) = fd.cand[k];
      double t = 0;
      st = measure(trial, &t);
      if (st != PICASSO_OK) return done(st);
      if (t < 0.99 * t_cur) {
        cur = trial;
        t_cur = t;
      }
    }
  }
  if (best) *best = cur;
  if (best_ms) *best_ms = t_cur;
  return done(PICASSO_OK);
}

int picasso_get_colors(void* ctx, int32_t* d_out) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!d_out) return PICASSO_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(d_out, c->color, sizeof(int32_t) * c->N, cudaMemcpyDeviceToDevice, c->s));
  return PICASSO_OK;
}

int picasso_get_round(void* ctx, int32_t* d_gid, int32_t* d_lists, uint32_t* d_prio) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (d_gid && c->n > 0) {
    if (c->assigned)
      CK(cudaMemcpyAsync(d_gid, c->gid_r, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->s));
    else if (c->gid)
      CK(cudaMemcpyAsync(d_gid, c->gid, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->s));
    else
      CK(launch_iota(d_gid, c->n, c->s));
  }
  if (d_lists || d_prio) {
    if (!c->assigned) return PICASSO_ERR_STATE;
    if (d_lists) CK(cudaMemcpyAsync(d_lists, c->lists, sizeof(int32_t) * c->E, cudaMemcpyDeviceToDevice, c->s));
    if (d_prio) CK(cudaMemcpyAsync(d_prio, c->prio, sizeof(uint32_t) * c->n, cudaMemcpyDeviceToDevice, c->s));
  }
  return PICASSO_OK;
}

int picasso_get_runs(void* ctx, const int64_t** d_runoff) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!c->built) return PICASSO_ERR_STATE;
  ST(canonical_csr(c));
  if (d_runoff) *d_runoff = c->runoff;
  return PICASSO_OK;
}

int picasso_copy_csr(void* ctx, int64_t* d_off, int32_t* d_col) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!c->built) return PICASSO_ERR_STATE;
  ST(canonical_csr(c));
  if (d_off) CK(cudaMemcpyAsync(d_off, c->off, sizeof(int64_t) * (c->n + 1), cudaMemcpyDeviceToDevice, c->s));
  if (d_col && c->nnz > 0)
    CK(cudaMemcpyAsync(d_col, c->col, sizeof(int32_t) * c->nnz, cudaMemcpyDefault, c->s));
  return PICASSO_OK;
}

int picasso_copy_runs(void* ctx, int64_t* d_runoff) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!c->built) return PICASSO_ERR_STATE;
  ST(canonical_csr(c));
  if (d_runoff)
    CK(cudaMemcpyAsync(d_runoff, c->runoff, sizeof(int64_t) * (c->E + 1), cudaMemcpyDeviceToDevice, c->s));
  return PICASSO_OK;
}

int picasso_get_stats(void* ctx, picasso_stats* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out) return PICASSO_ERR_INVALID_ARG;
  phase_resolve_all(c);
  std::memset(out, 0, sizeof(*out));
  out->round = c->round;
  out->n_total = c->N;
  out->n_round = c->n;
  out->P = c->Ptot;
  out->L = c->Lmax;
  out->base = c->sets.empty() ? 0 : c->sets[0].base;
  out->nnz = c->nnz;
  out->colored = c->n_colored;
  int64_t used = 0;
  for (int k = 0; k < c->nsets; ++k) used += c->set_base[k];
  out->colors_used = used;
  out->peak_bytes = c->peak_bytes;
  out->conflict_algo_used = c->algo_used;
  out->jp_sweeps = c->sweeps;
  out->ordered_fallbacks = c->ordered_fallbacks;
  out->max_bucket = c->max_bucket;
  out->rounds_done = c->rounds_done;
  out->t_assign_ms = c->t_assign;
  out->t_build_ms = c->t_build;
  out->t_color_ms = c->t_color;
  out->t_carry_ms = c->t_carry;
  out->t_pairs_ms = c->t_pairs;
  out->pairs_launches = c->pairs_launches;
  out->logical_pairs = c->logical_pairs;
  out->tested_pairs = c->tested_pairs;
  out->t_emit_ms = c->t_emit;
  out->emit_launches = c->emit_launches;
  out->emit_bytes = c->emit_bytes;
  out->nnz_total = c->nnz_total;
  out->small_rounds = c->small_rounds;
  out->small_stops = c->small_stops;
  for (int i = 0; i < 4; ++i) out->barrier_timeout[i] = c->barrier_timeout[i];
  out->t_small_ms = c->t_small;
  out->round_chunks = c->round_chunks;
  out->host_csr_rounds = c->host_rounds;
  const int ns = c->sweeps < kSweepLog ? c->sweeps : kSweepLog;
  const unsigned long long* t = reinterpret_cast<const unsigned long long*>(c->sweep_log + 8 + kSweepLog);
  for (int i = 0; i < ns; ++i) {
    out->sweep_pending[i] = c->sweep_log[8 + i];
    out->sweep_active[i] = c->sweep_log[8 + 3 * kSweepLog + i];
    out->sweep_us[i] = (float)((i + 1 < ns ? (double)(t[i + 1] - t[i]) : 0.0) / 1000.0);
  }
  return PICASSO_OK;
}

// Between-round state: header, per-set arrays, the colors of all strings and
// the global ids of the round's vertices.  Layout (little-endian, host):
//   int64 magic, version, N, nsets, round, n, rounds_done, seed0, num, den
//   double alpha
//   int64 soff[nsets+1], seed[nsets], set_base[nsets], remaining[nsets],
//         set_peak_bytes[nsets]
//   int32 color[N], gid[n]
namespace {
constexpr int64_t kStateMagic = 0x5049434153534f31ll;  // "PICASSO1"

int64_t state_bytes(const Ctx* c) {
  return 8 * 10 + 8 + 8 * (int64_t)(c->nsets + 1) + 8 * 4 * (int64_t)c->nsets + 4 * c->N + 4 * c->n;
}

bool between_rounds(const Ctx* c) { return !c->assigned && !c->built && !c->colored_done; }
}  // namespace

int picasso_save_state(void* ctx, void* h_buf, int64_t capacity, int64_t* bytes_out) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!bytes_out) return PICASSO_ERR_INVALID_ARG;
  if (!between_rounds(c)) return PICASSO_ERR_STATE;
  const int64_t need = state_bytes(c);
  *bytes_out = need;
  if (!h_buf) return PICASSO_OK;
  if (capacity < need) return PICASSO_ERR_INVALID_ARG;
  uint8_t* p = (uint8_t*)h_buf;
  auto put64 = [&](int64_t v) { std::memcpy(p, &v, 8); p += 8; };
  put64(kStateMagic);
  put64(1);
  put64(c->N);
  put64(c->nsets);
  put64(c->round);
  put64(c->n);
  put64(c->rounds_done);
  put64((int64_t)c->cfg.seed);
  put64(c->cfg.palette_num);
  put64(c->cfg.palette_den);
  std::memcpy(p, &c->cfg.alpha, 8);
  p += 8;
  for (int k = 0; k <= c->nsets; ++k) put64(c->soff[k]);
  for (int k = 0; k < c->nsets; ++k) put64((int64_t)c->seed[k]);
  for (int k = 0; k < c->nsets; ++k) put64(c->set_base[k]);
  for (int k = 0; k < c->nsets; ++k) put64(c->remaining[k]);
  for (int k = 0; k < c->nsets; ++k) put64(c->set_peak_bytes[k]);
  CK(cudaMemcpyAsync(p, c->color, 4 * c->N, cudaMemcpyDeviceToHost, c->s));
  p += 4 * c->N;
  if (c->n > 0) {
    if (c->gid) {
      CK(cudaMemcpyAsync(p, c->gid, 4 * c->n, cudaMemcpyDeviceToHost, c->s));
      CK(cudaStreamSynchronize(c->s));
    } else {
      CK(cudaStreamSynchronize(c->s));
      int32_t* g = (int32_t*)p;
      for (int64_t v = 0; v < c->n; ++v) g[v] = (int32_t)v;  // round 1: identity
    }
  } else {
    CK(cudaStreamSynchronize(c->s));
  }
  return PICASSO_OK;
}

int picasso_load_state(void* ctx, const void* h_buf, int64_t bytes) {
  Ctx* c = (Ctx*)ctx;
  ST(check(c));
  if (!h_buf || bytes < 8 * 11) return PICASSO_ERR_INVALID_ARG;
  if (!between_rounds(c)) return PICASSO_ERR_STATE;
  const uint8_t* p = (const uint8_t*)h_buf;
  auto get64 = [&]() {
    int64_t v;
    std::memcpy(&v, p, 8);
    p += 8;
    return v;
  };
  const int64_t magic = get64(), version = get64(), N = get64(), nsets = get64(), round = get64(), n = get64(),
                rounds_done = get64(), seed0 = get64(), num = get64(), den = get64();
  double alpha;
  std::memcpy(&alpha, p, 8);
  p += 8;
  if (magic != kStateMagic || version != 1 || N != c->N || nsets != c->nsets || (uint64_t)seed0 != c->cfg.seed ||
      num != c->cfg.palette_num || den != c->cfg.palette_den || alpha != c->cfg.alpha || n < 0 || n > N ||
      round < 1)
    return PICASSO_ERR_INVALID_ARG;
  const int64_t need = 8 * 10 + 8 + 8 * (nsets + 1) + 8 * 4 * nsets + 4 * N + 4 * n;
  if (bytes < need) return PICASSO_ERR_INVALID_ARG;
  for (int k = 0; k <= c->nsets; ++k)
    if (get64() != c->soff[k]) return PICASSO_ERR_INVALID_ARG;
  for (int k = 0; k < c->nsets; ++k)
    if ((uint64_t)get64() != c->seed[k]) return PICASSO_ERR_INVALID_ARG;
  std::vector<int64_t> base(c->nsets), rem(c->nsets), peak(c->nsets);
  for (int k = 0; k < c->nsets; ++k) base[k] = get64();
  for (int k = 0; k < c->nsets; ++k) rem[k] = get64();
  for (int k = 0; k < c->nsets; ++k) peak[k] = get64();
  int64_t rem_sum = 0;
  for (int k = 0; k < c->nsets; ++k) rem_sum += rem[k];
  if (rem_sum != n) return PICASSO_ERR_INVALID_ARG;
  const int32_t* color = (const int32_t*)p;
  const int32_t* gid = color + N;
  for (int64_t v = 0; v < n; ++v)
    if (gid[v] < 0 || gid[v] >= N || (v > 0 && gid[v] <= gid[v - 1])) return PICASSO_ERR_INVALID_ARG;
  int32_t* gid2 = nullptr;
  uint64_t* xz2 = nullptr;
  if (n > 0) {
    ST(alloc(c, &gid2, n));
    int st = alloc(c, &xz2, 2 * (int64_t)c->qw * n);
    if (st != PICASSO_OK) {
      release(c, &gid2);
      return st;
    }
    CK(cudaMemcpyAsync(gid2, gid, 4 * n, cudaMemcpyHostToDevice, c->s));
    CK(launch_gather_xz(c->xz_user, gid2, n, xz2, 2 * c->qw, c->s));
  }
  CK(cudaMemcpyAsync(c->color, color, 4 * N, cudaMemcpyHostToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  release(c, &c->gid);
  release(c, &c->xz);
  c->gid = gid2;
  c->xz = xz2;
  c->round = (int32_t)round;
  c->n = n;
  c->rounds_done = (int32_t)rounds_done;
  c->set_base = base;
  c->remaining = rem;
  c->set_peak_bytes = peak;
  return PICASSO_OK;
}

int picasso_get_set_stats(void* ctx, int64_t* h_colors, int64_t* h_peak_bytes, int64_t* h_remaining) {
  Ctx* c = (Ctx*)ctx;
  if (!c) return PICASSO_ERR_INVALID_ARG;
  for (int k = 0; k < c->nsets; ++k) {
    if (h_colors) h_colors[k] = c->set_base[k];
    if (h_peak_bytes) h_peak_bytes[k] = c->set_peak_bytes[k];
    if (h_remaining) h_remaining[k] = c->remaining[k];
  }
  return PICASSO_OK;
}

int picasso_features(const uint64_t* d_xz, int64_t n, int32_t q, uint64_t seed, int64_t samples,
                     double budget_bytes, int64_t* d_counts, float* d_feat, void* stream) {
  if (!d_xz || !d_counts || !d_feat || n < 1 || n >= (int64_t(1) << 31) || q < 1 || samples < 0 ||
      !(budget_bytes > 0.0) || !std::isfinite(budget_bytes))
    return PICASSO_ERR_INVALID_ARG;
  if (q > kMaxQ) return PICASSO_ERR_UNSUPPORTED;
  return map_err(launch_features(d_xz, n, q, seed, samples, std::log2(budget_bytes),
                                 reinterpret_cast<unsigned long long*>(d_counts), d_feat, (cudaStream_t)stream));
}

int picasso_features_beta(const uint64_t* d_xz, int64_t n, int32_t q, uint64_t seed, int64_t samples, double beta,
                          int64_t* d_counts, float* d_feat, void* stream) {
  if (!d_xz || !d_counts || !d_feat || n < 1 || n >= (int64_t(1) << 31) || q < 1 || samples < 0 ||
      !(beta >= 0.0 && beta <= 1.0))
    return PICASSO_ERR_INVALID_ARG;
  if (q > kMaxQ) return PICASSO_ERR_UNSUPPORTED;
  return map_err(launch_features(d_xz, n, q, seed, samples, 0.0, reinterpret_cast<unsigned long long*>(d_counts),
                                 d_feat, (cudaStream_t)stream, beta));
}

int32_t picasso_mlp_param_count(void) { return mlp_param_count(); }

int picasso_mlp_forward(const uint16_t* d_w, const float* d_x, int32_t batch, float* d_y, void* stream) {
  if (batch < 0 || (batch > 0 && (!d_w || !d_x || !d_y))) return PICASSO_ERR_INVALID_ARG;
  return map_err(launch_mlp_forward(d_w, d_x, batch, d_y, (cudaStream_t)stream));
}

int picasso_mlp_backward(const uint16_t* d_w, const float* d_x, const float* d_t, float weight0, float weight1,
                         int32_t batch, float* d_grad, float* d_loss, void* stream) {
  if (batch < 1 || !d_w || !d_x || !d_t || !d_grad || !std::isfinite(weight0) || !std::isfinite(weight1))
    return PICASSO_ERR_INVALID_ARG;
  return map_err(launch_mlp_backward(d_w, d_x, d_t, weight0, weight1, batch, d_grad, d_loss, (cudaStream_t)stream));
}

int picasso_mlp_adamw(float* d_master, uint16_t* d_w, const float* d_grad, float* d_m, float* d_v, float lr,
                      float beta1, float beta2, float eps, float weight_decay, int32_t step, void* stream) {
  if (!d_master || !d_w || !d_grad || !d_m || !d_v || step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) || !(weight_decay >= 0.f))
    return PICASSO_ERR_INVALID_ARG;
  return map_err(launch_mlp_adamw(d_master, d_w, d_grad, d_m, d_v, lr, beta1, beta2, eps, weight_decay, step,
                                  (cudaStream_t)stream));
}

int picasso_mlp_to_bf16(const float* d_src, uint16_t* d_dst, int32_t count, void* stream) {
  if (count < 0 || (count > 0 && (!d_src || !d_dst))) return PICASSO_ERR_INVALID_ARG;
  return map_err(launch_to_bf16(d_src, d_dst, count, (cudaStream_t)stream));
}

int picasso_trim_memory(int64_t keep_bytes) {
  if (keep_bytes < 0) return PICASSO_ERR_INVALID_ARG;
  pinned_trim();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return map_err(e);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (dev >= 0 && dev < 128) pool = g_pool[dev];
  }
  if (!pool) return PICASSO_OK;
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, (size_t)keep_bytes);
  return map_err(e);
}

int picasso_kernel_launches(int64_t* out) {
  if (!out) return PICASSO_ERR_INVALID_ARG;
  *out = (int64_t)g_launches.load();
  return PICASSO_OK;
}

int picasso_memory_requests(int64_t* out) {
  if (!out) return PICASSO_ERR_INVALID_ARG;
  *out = (int64_t)g_mem_requests.load();
  return PICASSO_OK;
}

int picasso_destroy(void* ctx) {
  Ctx* c = (Ctx*)ctx;
  if (!c) return PICASSO_ERR_INVALID_ARG;
  cudaSetDevice(c->dev);
  free_color(c);
  free_build(c);
  free_assign(c);
  release(c, &c->gid);
  release(c, &c->xz);
  release(c, &c->color);
  release(c, &c->d_err);
  release(c, &c->d_soff);
  release(c, &c->d_sets);
  release(c, &c->d_hist);
  release(c, &c->d_set_bytes);
  cudaStreamSynchronize(c->s);
  hostcol_put(c->hcol, c->hcol_cap);
  for (int i = 0; i < Ctx::kEvents; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  pinned_put(c->h_buf);
  delete c;
  return PICASSO_OK;
}

const char* picasso_strerror(int status) {
  switch (status) {
    case PICASSO_OK: return "ok";
    case PICASSO_ERR_INVALID_ARG: return "invalid argument";
    case PICASSO_ERR_OOM: return "device out of memory";
    case PICASSO_ERR_CUDA: return "CUDA error";
    case PICASSO_ERR_BUDGET: return "conflict graph exceeds the byte budget";
    case PICASSO_ERR_TIMEOUT: return "bounded device wait expired";
    case PICASSO_ERR_INTERNAL: return "internal consistency check failed";
    case PICASSO_ERR_UNSUPPORTED: return "outside this build's limits";
    case PICASSO_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

}  // extern "C"
