// capi_static.cu -- picasso_run_small_static: a whole Picasso run for small
// string sets that performs no device allocation.
//
// Some callers cannot allocate device memory while they work: plugins and
// services that hand every byte of the GPU to their own fixed pool, code that
// runs between a pool's reservation and its release, or hosts that forbid
// cudaMalloc/cudaFree on their hot path because those calls synchronise the
// device.  This entry point serves them for sets of at most kStaticMaxN
// strings: every temporary buffer of the run is carved out of one file-scope
// __device__ array of kStaticBytes bytes.  The caller still passes the packed
// strings and the color output.
//
// The array is owned by the library: once it has been used on a GPU (or at
// module load, if lazy module loading is off) that GPU holds it until the
// process exits.  All calls on a device share it and it keeps the last call's
// contents, so every region that must start at zero is cleared here.  Two
// calls whose work overlaps on the GPU (e.g. on two streams) race on the
// array; callers must serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"

using namespace picasso;

namespace {

constexpr int64_t kStaticMaxN = 2048;
constexpr int32_t kStaticMaxL = 32;
constexpr int64_t kStaticMaxNnz = 2560 * 1024;      // run entries in one round
constexpr int64_t kStaticNL = kStaticMaxN * kStaticMaxL;
constexpr size_t kScanTmpReserve = 64 * 1024;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// region offsets inside the array
constexpr size_t kOffGid = 0;                                              // 2 x [N] int32
constexpr size_t kOffXz = kOffGid + al(2 * kStaticMaxN * 4);               // 2 x [N][2] u64
constexpr size_t kOffLists = kOffXz + al(2 * kStaticMaxN * 16);            // [N*L] int32
constexpr size_t kOffPrio = kOffLists + al(kStaticNL * 4);                 // [N] u32
constexpr size_t kOffCnt = kOffPrio + al(kStaticMaxN * 4);                 // [N*L] u32
constexpr size_t kOffRunoff = kOffCnt + al(kStaticNL * 4);                 // [N*L+1] i64
constexpr size_t kOffCol = kOffRunoff + al((kStaticNL + 1) * 8);           // [maxnnz] i32
constexpr size_t kOffState = kOffCol + al(kStaticMaxNnz * 4);              // [N] u64
constexpr size_t kOffRcur = kOffState + al(kStaticMaxN * 8);               // [N] u32
constexpr size_t kOffBlk = kOffRcur + al(kStaticMaxN * 4);                 // [N] i32
constexpr size_t kOffBlkw = kOffBlk + al(kStaticMaxN * 4);                 // [N] u32
constexpr size_t kOffHist = kOffBlkw + al(kStaticMaxN * 4);                // [N] u32 (prio bins)
constexpr size_t kOffHoff = kOffHist + al(kStaticMaxN * 4);                // [N+1] i64
constexpr size_t kOffKcur = kOffHoff + al((kStaticMaxN + 1) * 8);          // [N] u16
constexpr size_t kOffWork = kOffKcur + al(kStaticMaxN * 2);                // 3 x [N] i32
constexpr size_t kOffCounts = kOffWork + al(3 * kStaticMaxN * 4);          // [kCtlWords] i32
constexpr size_t kOffFlag = kOffCounts + al(kCtlWords * 4);                // [N] u32
constexpr size_t kOffPos = kOffFlag + al(kStaticMaxN * 4);                 // [N+1] i64
constexpr size_t kOffTmp = kOffPos + al((kStaticMaxN + 1) * 8);            // scan temp
constexpr size_t kOffErr = kOffTmp + al(kScanTmpReserve);                  // [1] i32
constexpr size_t kOffLoff = kOffErr + 256;                                 // [N+1] i64
constexpr size_t kOffEnt = kOffLoff + al((kStaticMaxN + 1) * 8);           // [N*L] i32
constexpr size_t kOffLen = kOffEnt + al(kStaticNL * 4);                    // [N] u32
constexpr size_t kOffSoff = kOffLen + al(kStaticMaxN * 4);                 // [2] i64
constexpr size_t kOffSet = kOffSoff + 256;                                 // [1] SetRound
constexpr size_t kStaticBytes = kOffSet + 256;                             // about 12.1 MB

}  // namespace

// The scratch.  In host code this name is only a host-side stand-in: the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

std::mutex g_setup_mu;
void* g_scratch_addr[128] = {};

// Per-device set-up: look up the array's device address once, with that
// device current.
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return PICASSO_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) return PICASSO_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return PICASSO_OK;
}

void static_params(const picasso_config& cfg, int64_t n, int64_t* P, int32_t* L) {
  int64_t p = (n * cfg.palette_num + cfg.palette_den - 1) / cfg.palette_den;
  if (p < 1) p = 1;
  int64_t li = (int64_t)std::ceil(cfg.alpha * std::log((double)n));
  if (li < 1) li = 1;
  if (li > p) li = p;
  *P = p;
  *L = (int32_t)li;
}

int err_of(cudaError_t e) {
  if (e == cudaSuccess) return PICASSO_OK;
  return e == cudaErrorMemoryAllocation ? PICASSO_ERR_OOM : PICASSO_ERR_CUDA;
}

#define SCK(expr)                            \
  do {                                       \
    int _st = err_of(expr);                  \
    if (_st != PICASSO_OK) return _st;       \
  } while (0)

int read_i64(const void* d_src, int64_t* h, cudaStream_t s) {
  SCK(cudaMemcpyAsync(h, d_src, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCK(cudaStreamSynchronize(s));
  return PICASSO_OK;
}

}  // namespace

extern "C" int picasso_run_small_static(const uint64_t* d_xz, int64_t n, int32_t q, const picasso_config* cfg,
                                        int32_t* d_color_out, int32_t* n_rounds, void* stream) {
  if (!d_xz || !cfg || !d_color_out || q < 1 || n < 1) return PICASSO_ERR_INVALID_ARG;
  if (q > 64 || n > kStaticMaxN) return PICASSO_ERR_UNSUPPORTED;
  if (cfg->palette_num < 1 || cfg->palette_den < 1 || cfg->palette_num > (int64_t(1) << 32) ||
      cfg->palette_den > (int64_t(1) << 32) || !(cfg->alpha > 0.0) || !std::isfinite(cfg->alpha) ||
      cfg->max_rounds < 1 || cfg->byte_budget < 0 || cfg->color_algo < 0 || cfg->color_algo > 2 ||
      cfg->csr_form < 0 || cfg->csr_form > 1 || cfg->budget_mode < 0 || cfg->budget_mode > 2 ||
      cfg->wait_polls < 0 || cfg->wait_polls > (1 << 30))
    return PICASSO_ERR_INVALID_ARG;
  // Alg. 2's dynamic order and the budget fallbacks (chunks, host CSR) are
  // not built here
  if (cfg->color_algo == PICASSO_COLOR_DYNAMIC) return PICASSO_ERR_UNSUPPORTED;
  if (cfg->byte_budget > 0 && cfg->budget_mode != PICASSO_BUDGET_FAIL) return PICASSO_ERR_UNSUPPORTED;
  {
    int64_t P;
    int32_t L;
    static_params(*cfg, n, &P, &L);  // L never grows in later rounds
    if (L > kStaticMaxL) return PICASSO_ERR_UNSUPPORTED;
  }
  if (scan_tmp_bytes(kStaticNL + 1) > kScanTmpReserve) return PICASSO_ERR_INTERNAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base_ptr = nullptr;
  {
    int st = scratch_for_current_device(&base_ptr);
    if (st != PICASSO_OK) return st;
  }
  int32_t* gid_buf[2] = {(int32_t*)(base_ptr + kOffGid), (int32_t*)(base_ptr + kOffGid) + kStaticMaxN};
  uint64_t* xz_buf[2] = {(uint64_t*)(base_ptr + kOffXz), (uint64_t*)(base_ptr + kOffXz) + 2 * kStaticMaxN};
  int32_t* lists = (int32_t*)(base_ptr + kOffLists);
  uint32_t* prio = (uint32_t*)(base_ptr + kOffPrio);
  uint32_t* cnt = (uint32_t*)(base_ptr + kOffCnt);
  int64_t* runoff = (int64_t*)(base_ptr + kOffRunoff);
  int32_t* col = (int32_t*)(base_ptr + kOffCol);
  uint64_t* state = (uint64_t*)(base_ptr + kOffState);
  uint32_t* rcur = (uint32_t*)(base_ptr + kOffRcur);
  int32_t* blk = (int32_t*)(base_ptr + kOffBlk);
  uint32_t* blkw = (uint32_t*)(base_ptr + kOffBlkw);
  uint32_t* hist = (uint32_t*)(base_ptr + kOffHist);
  int64_t* hoff = (int64_t*)(base_ptr + kOffHoff);
  uint16_t* kcur = (uint16_t*)(base_ptr + kOffKcur);
  int32_t* work[2] = {(int32_t*)(base_ptr + kOffWork), (int32_t*)(base_ptr + kOffWork) + kStaticMaxN};
  int32_t* wact = (int32_t*)(base_ptr + kOffWork) + 2 * kStaticMaxN;
  int32_t* counts = (int32_t*)(base_ptr + kOffCounts);
  uint32_t* flag = (uint32_t*)(base_ptr + kOffFlag);
  int64_t* pos = (int64_t*)(base_ptr + kOffPos);
  void* tmp = (void*)(base_ptr + kOffTmp);
  int32_t* derr = (int32_t*)(base_ptr + kOffErr);
  int64_t* loff = (int64_t*)(base_ptr + kOffLoff);
  int32_t* ent_v = (int32_t*)(base_ptr + kOffEnt);
  uint32_t* len = (uint32_t*)(base_ptr + kOffLen);
  int64_t* soff = (int64_t*)(base_ptr + kOffSoff);
  SetRound* dset = (SetRound*)(base_ptr + kOffSet);
  static_assert(sizeof(SetRound) <= 256, "set table slot");

  SCK(launch_fill_i32(d_color_out, n, -1, s));
  SCK(cudaMemsetAsync(derr, 0, sizeof(int32_t), s));
  {
    const int64_t h_soff[2] = {0, n};
    SCK(cudaMemcpyAsync(soff, h_soff, sizeof(h_soff), cudaMemcpyHostToDevice, s));
  }

  const int32_t* gid = nullptr;         // round 1: identity
  const uint64_t* xz = d_xz;            // round 1: the caller's strings
  int cur = 0;
  int64_t m = n, base = 0;
  int32_t round = 1;
  while (m > 0) {
    if (round > cfg->max_rounds) return PICASSO_ERR_INTERNAL;
    int64_t P;
    int32_t L;
    static_params(*cfg, m, &P, &L);
    if (P >= (int64_t(1) << 30) || base + P > (int64_t)0x7fffffff) return PICASSO_ERR_UNSUPPORTED;
    const int64_t nl = m * L;
    SetRound sr{};
    sr.seed = cfg->seed;
    sr.P = P;
    sr.cofs = 0;
    sr.base = base;
    sr.L = L;
    SCK(cudaMemcpyAsync(dset, &sr, sizeof(sr), cudaMemcpyHostToDevice, s));
    SCK(launch_list_offsets(gid, m, soff, 1, dset, len, loff, tmp, s));
    SCK(launch_entry_owner(loff, m, ent_v, s));
    SCK(launch_assign_lists(round, gid, m, soff, 1, dset, L, loff, lists, prio, nullptr, s));

    ConflictArgs a{};
    a.n = m;
    a.E = nl;
    a.Lmax = L;
    a.Lu = L;
    a.P = P;
    a.xz = xz;
    a.lists = lists;
    a.loff = loff;
    a.ent_v = ent_v;
    a.cnt = cnt;
    a.err = derr;
    SCK(launch_allpairs(a, false, s));
    SCK(launch_scan_u32(cnt, nl, runoff, tmp, s));
    int64_t nnz = 0;
    {
      int st = read_i64(runoff + nl, &nnz, s);
      if (st != PICASSO_OK) return st;
    }
    if (nnz > kStaticMaxNnz) return PICASSO_ERR_UNSUPPORTED;
    // the byte budget counts the CSR picasso_run would build: both directions
    // (FULL) or each pair once (EARLIER, half of the two-sided count here)
    const int64_t csr_nnz = cfg->csr_form == PICASSO_CSR_FULL ? nnz : nnz / 2;
    if (cfg->byte_budget > 0 && 8 * (m + 1) + 4 * csr_nnz > cfg->byte_budget) return PICASSO_ERR_BUDGET;
    a.runoff = runoff;
    a.col = col;
    SCK(launch_allpairs(a, true, s));

    ColorArgs ca{};
    ca.n = m;
    ca.lists = lists;
    ca.loff = loff;
    ca.runoff = runoff;
    ca.col = col;
    ca.state = state;
    ca.kcur = kcur;
    ca.rcur = rcur;
    ca.blk = blk;
    ca.blkw = blkw;
    ca.ranked = 0;  // ids in ascending global id; the order list gives the coloring order
    ca.max_polls = cfg->wait_polls > 0 ? cfg->wait_polls : kMaxPolls;
    SCK(cudaMemsetAsync(counts, 0, sizeof(int32_t) * kCtlWords, s));
    SCK(launch_prio_order(prio, m, prio_bins_for(m), hist, hoff, tmp, work[0], s));
    SCK(launch_color_init(ca, prio, counts, s));
    const bool sweep_only = cfg->color_algo == PICASSO_COLOR_SWEEP;
    if (!sweep_only) SCK(launch_color_ordered(ca, work[0], counts + 5, s));
    {
      int32_t h[8];
      SCK(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s));
      SCK(cudaStreamSynchronize(s));
      if (sweep_only || h[5] != 0) {  // SWEEP, or a bounded wait ran out: the sweep kernel
        SCK(cudaMemsetAsync(counts, 0, sizeof(int32_t) * kCtlWords, s));
        SCK(launch_color_init(ca, prio, counts, s));
        SCK(launch_color_all(ca, work[0], work[1], wact, counts, s));
        int32_t ab = 0;
        SCK(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s));
        SCK(cudaMemcpyAsync(&ab, counts + kCtlAbort, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SCK(cudaStreamSynchronize(s));
        if (ab != 0) return PICASSO_ERR_TIMEOUT;  // a grid barrier of the sweep kernel gave up
        if (h[4] != 0 || h[0] != 0) return PICASSO_ERR_INTERNAL;
      }
    }
    SCK(launch_carry_flags(state, m, gid, nullptr, soff, 1, dset, d_color_out, flag, s));
    SCK(launch_scan_u32(flag, m, pos, tmp, s));
    int64_t rem = 0;
    {
      int st = read_i64(pos + m, &rem, s);
      if (st != PICASSO_OK) return st;
    }
    if (rem > 0) {
      SCK(launch_carry_gather(flag, pos, m, gid, xz, gid_buf[cur], xz_buf[cur], 2, s));
      gid = gid_buf[cur];
      xz = xz_buf[cur];
      cur = 1 - cur;
    }
    base += P;
    m = rem;
    ++round;
  }
  SCK(cudaStreamSynchronize(s));
  if (n_rounds) *n_rounds = round - 1;
  return PICASSO_OK;
}
