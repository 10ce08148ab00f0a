// C ABI of libphmm: plans, workspace layout, the forward launch sequence and CUDA graphs.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>
#include <nvtx3/nvToolsExt.h>
#include "fwd_inst.cuh"
#include "phmm_internal.cuh"

namespace phmm {

int launch_validate(const phmm_batch &b, int64_t sum_m, int64_t sum_n, unsigned *err,
                    unsigned long long *cells, cudaStream_t s);
int launch_prep(const phmm_batch &b, int64_t sum_m, float beta32, RowParams *rp,
                uint8_t *rcode, uint8_t *hcode, float2 *rgap, cudaStream_t s, int *launches);
int launch_binning(const phmm_batch &b, const CfgTable &tab, int32_t *key, int32_t *counts,
                   int32_t *offsets, int32_t *cursor, int32_t *grp_begin, int32_t *grp_count,
                   int32_t *order, cudaStream_t s, int *launches);
int bwd_enqueue_impl(phmm_plan *pl, char *ws, const double *dL, float *dbq, float *diq,
                     float *ddq, float *dgq, double *dgcp, cudaStream_t s, int *launches,
                     cudaEvent_t *ev3);
int bwd_sweep_impl(phmm_plan *pl, char *ws, const double *dL, double *out, uint8_t *oflags,
                   cudaStream_t s, int *launches, cudaEvent_t *ev2);
int bwd_reduce_impl(phmm_plan *pl, char *ws, const double *dL, float *dbq, float *diq,
                    float *ddq, float *dgq, double *dgcp, cudaStream_t s, int *launches,
                    cudaEvent_t ev1);
size_t bwd_workspace_bytes(const phmm_plan *pl);
std::vector<size_t> bwd_guard_offsets(const phmm_plan *pl);
int bwd_default_cfg(int m);
int bwd_cfg_supported(int cfg);

static thread_local int g_last_cuda = 0;

// Result words of plan-time validation: kValidateSlots static 64-byte device slots, one per
// plan creation in progress on this device (taken and given back under a lock); a creation
// that finds every slot taken allocates its own.
constexpr int kValidateSlots = 64;
__device__ unsigned long long g_validate_slot[kValidateSlots][8];
struct ValidateSlot {
  static std::mutex &mu() {
    static std::mutex m;
    return m;
  }
  static uint64_t &busy(int dev) {  // bit i: slot i in use on device dev
    static uint64_t b[64] = {};
    return b[dev & 63];
  }
  int dev = 0, idx = -1;
  void *p = nullptr;
  cudaError_t err = cudaSuccess;
  bool owned = false;
  ValidateSlot() {
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return;
    {
      std::lock_guard<std::mutex> lock(mu());
      uint64_t &b = busy(dev);
      for (int i = 0; i < kValidateSlots; ++i)
        if (!(b >> i & 1)) {
          b |= 1ull << i;
          idx = i;
          break;
        }
    }
    if (idx >= 0) {
      void *base = nullptr;
      err = cudaGetSymbolAddress(&base, g_validate_slot);
      if (err == cudaSuccess) p = (char *)base + (size_t)idx * 64;
    } else {
      err = cudaMalloc(&p, 64);
      owned = err == cudaSuccess;
      if (!owned) p = nullptr;
    }
  }
  ~ValidateSlot() {
    if (owned) cudaFree(p);
    if (idx >= 0) {
      std::lock_guard<std::mutex> lock(mu());
      busy(dev) &= ~(1ull << idx);
    }
  }
  void *ptr() const { return p; }
  cudaError_t error() const { return err == cudaSuccess ? cudaErrorUnknown : err; }
};

static int cuda_fail(cudaError_t e) {
  g_last_cuda = (int)e;
  return PHMM_ECUDA;
}
#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

static size_t table_warp_bytes(int K, int elem) {
  const int vw = 16 / elem, KV = (K + vw - 1) / vw * vw, units = KV / vw;
  const int LS = (units % 2 == 1) ? KV : KV + vw;
  return (size_t)kCodes * 32 * LS * elem;
}

static FwdKernel get32(int cfg, bool ext, bool gq = false) {
  const int L = cfg_lanes(cfg), K = cfg_rows(cfg);
  if (gq) return ext ? fwd32_gq(L, K) : nullptr;
  if (L <= 8) return ext ? fwd32_ext_lo(L, K) : fwd32_plain_lo(L, K);
  return ext ? fwd32_ext_hi(L, K) : fwd32_plain_hi(L, K);
}
static FwdKernel get64(int cfg64, bool ext, bool gq = false) {
  return gq ? fwd64_gq(rows64(cfg64), ext) : fwd64_table(rows64(cfg64), ext);
}

size_t fwd32_smem(int cfg, int block) { return (block / 32) * table_warp_bytes(cfg_rows(cfg), 4); }
// 1 if the FP32 forward kernels (both first lines) are built for group `cfg`.
int fwd_cfg_supported(int cfg) {
  return cfg >= 0 && cfg < kNumCfg32 && get32(cfg, true) != nullptr &&
         get32(cfg, false) != nullptr;
}
size_t fwd64_smem(int cfg64, int block) {
  return (block / 32) * table_warp_bytes(rows64(cfg64), 8);
}

static std::once_flag g_attr_once;
static void set_attrs() {
  for (int g = 0; g < 2; ++g) {
    for (int cfg = 0; cfg < kNumCfg32; ++cfg)
      for (int e = 0; e < 2; ++e) {
        FwdKernel k = get32(cfg, e, g);
        if (k) cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024);
      }
    for (int c = 0; c < kNumCfg64; ++c)
      for (int e = 0; e < 2; ++e) {
        FwdKernel k = get64(c, e, g);
        if (k) cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024);
      }
  }
}

int fwd32_blocks_per_sm(int cfg, bool ext, int block, bool gq) {
  std::call_once(g_attr_once, set_attrs);
  FwdKernel k = get32(cfg, ext, gq);
  int nb = 0;
  if (k) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, fwd32_smem(cfg, block));
  return nb;
}
int fwd64_blocks_per_sm(int cfg64, bool ext, int block, bool gq) {
  std::call_once(g_attr_once, set_attrs);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, get64(cfg64, ext, gq), block,
                                                fwd64_smem(cfg64, block));
  return nb;
}

// The kernel of a launch follows its arguments: a batch with a per-base gap-continuation
// track (a.gq) runs the kernels with per-row gap continuation.
int launch_fwd32(int cfg, bool ext, int grid, int block, cudaStream_t s, const FwdArgs &a) {
  std::call_once(g_attr_once, set_attrs);
  FwdKernel k = get32(cfg, ext, a.gq != nullptr);
  if (!k) return (int)cudaErrorInvalidValue;
  k<<<grid, block, fwd32_smem(cfg, block), s>>>(a);
  return (int)cudaGetLastError();
}
int launch_fwd64(int cfg64, bool ext, int grid, int block, cudaStream_t s, const FwdArgs &a) {
  std::call_once(g_attr_once, set_attrs);
  FwdKernel k = get64(cfg64, ext, a.gq != nullptr);
  if (!k) return (int)cudaErrorInvalidValue;
  k<<<grid, block, fwd64_smem(cfg64, block), s>>>(a);
  return (int)cudaGetLastError();
}

// Default read-length -> group table: the lanes x rows group with the fewest pad rows,
// fewer lanes on a tie (shorter wavefront ramp, more rows to amortise each step's exchange).
int default_cfg_of_m(int m) {
  int best = -1, best_cap = 1 << 30;
  for (int L = 4; L <= 32; L *= 2) {
    int K = (m + L - 1) / L;
    K = K < 4 ? 4 : (K + 1) / 2 * 2;
    if (K > 20) continue;
    if (L * K < best_cap) {
      best_cap = L * K;
      best = cfg_index(L, K);
    }
  }
  return best < 0 ? cfg_index(32, 16) : best;
}

}  // namespace phmm

using namespace phmm;

// Debug builds (PHMM_DEBUG): a guard region of kGuardBytes after every workspace region, filled
// with kGuardByte before each call and checked after it.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
#ifdef PHMM_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

struct WsLayout {
  std::vector<size_t> guards;  // guard offsets (debug builds)
  size_t tile = 0;  // row-tile buffers (plans holding reads longer than one group)
  size_t rgap = 0;  // per-position (eps_i, beta_i) (plans with a gap-continuation track)
  size_t rp, rcode, hcode, key, order, zero, zero_bytes, counts, ctr32, ctr64, ctrx, rcnt, xcnt,
      offsets, cursor, grp_begin, grp_count, rlist, xlist, bwd, total, why;
};

struct phmm_plan {
  phmm_batch b;
  phmm_options o;
  int64_t sum_m = 0, sum_n = 0, cells = 0, pair_rows = 0, n_max = 0;
  int max_m = 0;
  bool gq = false;  // the batch has a per-base gap-continuation track
  int cfg_of_m[PHMM_MAX_READ_LEN + 1];
  int bwd_cfg_of_m[PHMM_MAX_READ_LEN + 1];
  std::vector<int> used_cfgs, bwd_used;
  WsLayout L;
  int sms = 0;
  float eps32 = 0, beta32 = 0;
  double eps64 = 0, beta64 = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  void *g_ws = nullptr, *g_out = nullptr, *g_flags = nullptr;
  // the fused training step's two calls, captured on small batches (pointer sets as keys)
  cudaGraphExec_t gexec_fp = nullptr, gexec_bp = nullptr;
  const void *gfp_key[3] = {nullptr, nullptr, nullptr};
  const void *gbp_key[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // the previous call's pointers: a graph is captured only when a pointer set repeats
  const void *gfp_prev[3] = {nullptr, nullptr, nullptr};
  const void *gbp_prev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int gfp_launches = 0, gbp_launches = 0;
  // forward: FP32 kernels start/end, rescue end; adjoint: start, end, reduction end;
  // reduction start of the fused path
  cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int red_from = 4;   // the event the latest reduction started after
  bool bwd_timed = false;
  bool fwd_done = false;
  bool partials_done = false;  // the workspace holds the partials of log10 L (fused forward)
  bool timed = false;  // the latest forward recorded the timing events
  int launches_fwd = 0, launches_bwd = 0;
  void *bwd_state = nullptr;  // owned by the backward translation unit
  unsigned *dbg_word = nullptr;  // debug builds: failed guard and index checks (device)
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static void make_layout(phmm_plan *pl) {
  WsLayout &L = pl->L;
  const int64_t P = std::max<int64_t>(pl->b.n_pairs, 1);
  const size_t nkeys = (size_t)kNumCfg32 * kNBuckets;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    if (kDebug) {
      L.guards.push_back(o);
      o += kGuardBytes;
    }
    return at;
  };
  L.rp = take(sizeof(RowParams) * std::max<int64_t>(pl->sum_m, 1));
  if (pl->gq) L.rgap = take(sizeof(float2) * std::max<int64_t>(pl->sum_m, 1));
  L.rcode = take(std::max<int64_t>(pl->sum_m, 1));
  L.hcode = take((size_t)hap_code_bytes(pl->sum_n, pl->b.n_haps));
  L.key = take(4 * P);
  L.order = take(4 * P);
  // region zeroed at the start of every forward
  L.zero = o;
  L.counts = o;
  o += 4 * nkeys;
  L.ctr32 = o;
  o += 4 * kNumCfg32;
  L.ctr64 = o;
  o += 4 * kNumCfg64;
  L.ctrx = o;
  o += 4 * kNumCfg64;
  L.rcnt = o;
  o += 4 * kNumCfg64;
  L.xcnt = o;
  o += 4 * kNumCfg64;
  L.why = o;  // adjoint hand-offs for the scale range / non-finite partials
  o += 4 * 4;
  o = align256(o);
  L.zero_bytes = o - L.zero;
  if (kDebug) {
    L.guards.push_back(o);
    o += kGuardBytes;
  }
  L.offsets = take(4 * nkeys);
  L.cursor = take(4 * nkeys);
  L.grp_begin = take(4 * kNumCfg32);
  L.grp_count = take(4 * kNumCfg32);
  L.rlist = take((size_t)4 * P * kNumCfg64);
  L.xlist = take((size_t)4 * P * kNumCfg64);
  if (pl->max_m > PHMM_MAX_READ_LEN) {
    // 2 buffers of n_max columns (32 B each, enough for FP64) per resident warp of the widest
    // persistent launch of the 32 x 16 group (FP32 or FP64, either tier)
    const int block = 32 * pl->o.warps_per_block, c16 = cfg_index(32, 16);
    int bps = 1;
    for (int e = 0; e < 2; ++e) {
      bps = std::max(bps, fwd32_blocks_per_sm(c16, e == 1, block, pl->gq));
      bps = std::max(bps, fwd64_blocks_per_sm(2, e == 1, block, pl->gq));
    }
    const size_t warps = (size_t)pl->sms * bps * (block / 32);
    L.tile = take(warps * 2 * (size_t)pl->n_max * 32);
  }
  L.bwd = o;
  L.total = o;
}

namespace phmm {
NvtxRange::NvtxRange(const char *name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }
}  // namespace phmm

extern "C" {

void phmm_options_default(phmm_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->first_line = PHMM_FIRST_EXT32;
  opt->rescue = 1;
  opt->binning = 1;
  opt->lanes = 8;
  opt->rows = 16;
  opt->persistent = 1;
  opt->use_graph = 1;
  opt->warps_per_block = 4;
  opt->bin_table_valid = 0;
  opt->adjoint_rescue = 1;
}

const char *phmm_status_str(int s) {
  switch (s) {
    case PHMM_OK: return "ok";
    case PHMM_EINVAL: return "invalid argument";
    case PHMM_ETOOLONG: return "read longer than PHMM_MAX_READ_LEN";
    case PHMM_ENOMEM: return "workspace too small";
    case PHMM_ECUDA: return "CUDA error";
    case PHMM_ESTATE: return "call out of order";
    case PHMM_EGUARD: return "debug build: a guard region or a kernel index check failed";
    default: return "unknown status";
  }
}

int phmm_last_cuda_error(void) { return g_last_cuda; }

static bool valid_group(int L, int K) {
  return (L == 4 || L == 8 || L == 16 || L == 32) && K >= 4 && K <= 20 && K % 2 == 0;
}

int phmm_plan_create(const phmm_batch *batch, const phmm_options *opt, void *stream,
                     phmm_plan **out) {
  const phmm::NvtxRange nvtx("phmm_plan_create");
  if (!batch || !out) return PHMM_EINVAL;
  *out = nullptr;
  const phmm_batch &b = *batch;
  phmm_options o;
  if (opt)
    o = *opt;
  else
    phmm_options_default(&o);
  if (b.n_reads < 1 || b.n_haps < 1 || b.n_pairs < 0) return PHMM_EINVAL;
  if (b.n_reads > INT32_MAX || b.n_haps > INT32_MAX || b.n_pairs > INT32_MAX) return PHMM_EINVAL;
  if (!b.read_bases || !b.base_q || !b.ins_q || !b.del_q || !b.read_off || !b.hap_bases ||
      !b.hap_off)
    return PHMM_EINVAL;
  if (b.n_pairs > 0 && (!b.pair_read || !b.pair_hap)) return PHMM_EINVAL;
  if (b.qual_dtype != PHMM_QUAL_U8 && b.qual_dtype != PHMM_QUAL_F32) return PHMM_EINVAL;
  if (b.alpha_mode != 0 && b.alpha_mode != 1) return PHMM_EINVAL;
  if (!(b.gcp > 0.0) || !std::isfinite(b.gcp)) return PHMM_EINVAL;
  if (o.first_line != PHMM_FIRST_PLAIN32 && o.first_line != PHMM_FIRST_EXT32) return PHMM_EINVAL;
  // a per-base gap-continuation track runs the extended-range FP32 first line only
  if (b.gcp_q && o.first_line != PHMM_FIRST_EXT32) return PHMM_EINVAL;
  if (b.gcp_q && !o.binning) return PHMM_EINVAL;
  if (o.adjoint_rescue < 0 || o.adjoint_rescue > 2) return PHMM_EINVAL;
  if (!o.binning && !valid_group(o.lanes, o.rows)) return PHMM_EINVAL;
  (void)cudaGetLastError();  // drop a stale error left by an unrelated call
  if (o.warps_per_block <= 0) o.warps_per_block = 4;
  if (o.warps_per_block > 4) return PHMM_EINVAL;  // the kernels are built for <= 128 threads
  if (o.bwd_warps_per_block <= 0) o.bwd_warps_per_block = o.warps_per_block;
  if (o.bwd_warps_per_block > 4) return PHMM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;

  // offsets to the host: monotone from 0, non-empty sequences, read length bound
  std::vector<int64_t> ro(b.n_reads + 1), ho(b.n_haps + 1);
  CK(cudaMemcpyAsync(ro.data(), b.read_off, 8 * ro.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ho.data(), b.hap_off, 8 * ho.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (ro[0] != 0 || ho[0] != 0) return PHMM_EINVAL;
  int max_m = 0;
  for (int64_t r = 0; r < b.n_reads; ++r) {
    const int64_t m = ro[r + 1] - ro[r];
    if (m <= 0) return PHMM_EINVAL;
    if (m > PHMM_MAX_READ_LEN_FWD) return PHMM_ETOOLONG;
    max_m = std::max<int>(max_m, (int)m);
  }
  for (int64_t h = 0; h < b.n_haps; ++h)
    if (ho[h + 1] - ho[h] <= 0 || ho[h + 1] - ho[h] > INT32_MAX / 2) return PHMM_EINVAL;
  const int64_t sum_m = ro[b.n_reads], sum_n = ho[b.n_haps];

  // device checks: bases, Phred values, pair ids; and the cell count of Eq. 5.  The result
  // words live in a static device slot: cudaFree would wait for the whole device, stalling
  // a caller that creates the next plan while another stream computes.
  ValidateSlot vs;
  void *dbuf = vs.ptr();
  if (!dbuf) return cuda_fail(vs.error());
  CK(cudaMemsetAsync(dbuf, 0, 64, s));
  unsigned *err = (unsigned *)dbuf;
  unsigned long long *cells = (unsigned long long *)((char *)dbuf + 8);
  int rc = launch_validate(b, sum_m, sum_n, err, cells, s);
  unsigned long long hbuf[3] = {0, 0, 0};
  cudaError_t e2 = rc ? (cudaError_t)rc : cudaMemcpyAsync(hbuf, dbuf, 24, cudaMemcpyDeviceToHost, s);
  if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
  if (e2 != cudaSuccess) return cuda_fail(e2);
  if ((unsigned)hbuf[0] != 0) return PHMM_EINVAL;

  phmm_plan *pl = new (std::nothrow) phmm_plan();
  if (!pl) return PHMM_ENOMEM;
  pl->b = b;
  pl->o = o;
  pl->sum_m = sum_m;
  pl->sum_n = sum_n;
  pl->cells = (int64_t)hbuf[1];
  pl->pair_rows = (int64_t)hbuf[2];
  pl->max_m = max_m;
  pl->gq = b.gcp_q != nullptr;
  for (int64_t h = 0; h < b.n_haps; ++h) pl->n_max = std::max<int64_t>(pl->n_max, ho[h + 1] - ho[h]);
  pl->eps64 = std::pow(10.0, -b.gcp / 10.0);
  pl->beta64 = 1.0 - pl->eps64;
  pl->eps32 = (float)pl->eps64;
  pl->beta32 = (float)pl->beta64;
  for (int m = 0; m <= PHMM_MAX_READ_LEN; ++m) {
    int c = default_cfg_of_m(std::max(m, 1));
    if (pl->gq) {  // the kernels with per-row gap continuation exist for these groups only
      pl->cfg_of_m[m] = gq_cfg_of_m(std::max(m, 1));
      continue;
    }
    if (o.bin_table_valid) {
      const int e = o.bin_rows[(std::max(m, 1) + 3) / 4];
      if (fwd_cfg_supported(e) && cfg_lanes(e) * cfg_rows(e) >= m) c = e;
    }
    pl->cfg_of_m[m] = c;
  }
  if (o.binning) {
    std::vector<char> used(kNumCfg32, 0);
    for (int64_t r = 0; r < b.n_reads; ++r)
      used[pl->cfg_of_m[std::min<int64_t>(ro[r + 1] - ro[r], PHMM_MAX_READ_LEN)]] = 1;
    for (int c = 0; c < kNumCfg32; ++c)
      if (used[c]) pl->used_cfgs.push_back(c);
  }
  {
    for (int m = 0; m <= PHMM_MAX_READ_LEN; ++m) {
      int c = bwd_default_cfg(std::max(m, 1));
      if (pl->gq) {
        pl->bwd_cfg_of_m[m] = gq_cfg_of_m(std::max(m, 1));
        continue;
      }
      if (o.bwd_table_valid) {
        const int e = o.bwd_rows[(std::max(m, 1) + 3) / 4];
        if (bwd_cfg_supported(e) && cfg_lanes(e) * cfg_rows(e) >= m) c = e;
      }
      pl->bwd_cfg_of_m[m] = c;
    }
    std::vector<char> used(kNumCfg32, 0);
    for (int64_t r = 0; r < b.n_reads; ++r)
      used[pl->bwd_cfg_of_m[std::min<int64_t>(ro[r + 1] - ro[r], PHMM_MAX_READ_LEN)]] = 1;
    for (int c = 0; c < kNumCfg32; ++c)
      if (used[c]) pl->bwd_used.push_back(c);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, dev);
  make_layout(pl);
  pl->L.total = pl->L.bwd + bwd_workspace_bytes(pl);
  if (kDebug) {
    for (size_t g : bwd_guard_offsets(pl)) pl->L.guards.push_back(pl->L.bwd + g);
    if (cudaMalloc((void **)&pl->dbg_word, 64) != cudaSuccess ||
        cudaMemset(pl->dbg_word, 0, 64) != cudaSuccess) {
      phmm_plan_destroy(pl);
      return PHMM_ECUDA;
    }
  }
  cudaError_t ce = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
  for (int i = 0; i < 7 && ce == cudaSuccess; ++i) ce = cudaEventCreate(&pl->ev[i]);
  if (ce != cudaSuccess) {
    phmm_plan_destroy(pl);
    return cuda_fail(ce);
  }
  *out = pl;
  return PHMM_OK;
}

size_t phmm_workspace_bytes(const phmm_plan *pl) { return pl ? pl->L.total : 0; }

int phmm_plan_info(const phmm_plan *pl, int64_t *sum_m, int64_t *sum_n, int64_t *cells) {
  if (!pl) return PHMM_EINVAL;
  if (sum_m) *sum_m = pl->sum_m;
  if (sum_n) *sum_n = pl->sum_n;
  if (cells) *cells = pl->cells;
  return PHMM_OK;
}

void phmm_plan_destroy(phmm_plan *pl) {
  if (!pl) return;
  if (pl->dbg_word) cudaFree(pl->dbg_word);
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  if (pl->gexec_fp) cudaGraphExecDestroy(pl->gexec_fp);
  if (pl->gexec_bp) cudaGraphExecDestroy(pl->gexec_bp);
  for (auto &e : pl->ev)
    if (e) cudaEventDestroy(e);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  delete pl;
}

}  // extern "C"

// The fused training step's calls on small batches (at most kGraphCells cells, e.g. one
// region) replay a captured CUDA graph: their 20-30 launches would otherwise cost more than
// the kernels.  Larger batches launch eagerly and keep the kernel-time events.  A graph is
// captured when a call repeats the previous call's pointers (capture costs more than one
// eager call) and replayed while they stay the same.
constexpr int64_t kGraphCells = (int64_t)1 << 30;

// Capture `enqueue` (a function of the capture stream returning a cudaError_t value) into
// *exec; returns PHMM_OK or a status.
template <typename F>
static int capture_graph(phmm_plan *pl, cudaGraphExec_t *exec, F enqueue) {
  if (*exec) {
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  CK(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue(pl->cap);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(pl->cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc > 0 ? cuda_fail((cudaError_t)rc) : rc;
  }
  if (ce != cudaSuccess) return cuda_fail(ce);
  ce = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) return cuda_fail(ce);
  return PHMM_OK;
}

// ---- debug builds: guard regions and the kernels' index checks --------------------------
struct GuardList {
  int n;
  unsigned long long off[64];
};

// Every byte of every guard region must still hold kGuardByte.
__global__ void k_check_guards(const unsigned char *ws, GuardList gl, unsigned *err) {
  unsigned bad = 0;
  for (int g = blockIdx.x; g < gl.n; g += gridDim.x)
    for (int k = threadIdx.x; k < (int)kGuardBytes; k += blockDim.x)
      if (ws[gl.off[g] + k] != kGuardByte) bad = 1;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kDbgGuard);
}

// Before a call (debug builds): fill the guard regions.
static int dbg_begin(phmm_plan *pl, void *ws, size_t ws_bytes, void *stream) {
  if constexpr (kDebug) {
    if (!pl || !ws || ws_bytes < pl->L.total || ((uintptr_t)ws & 255)) return PHMM_OK;
    for (size_t g : pl->L.guards)
      if (cudaMemsetAsync((char *)ws + g, kGuardByte, kGuardBytes, (cudaStream_t)stream) !=
          cudaSuccess)
        return PHMM_ECUDA;
  }
  return PHMM_OK;
}

// Checks the guards now; PHMM_EGUARD if a guard or a kernel's index check failed since the
// last check.  Waits for `stream`.
static int dbg_check(phmm_plan *pl, void *ws, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  GuardList gl;
  gl.n = (int)std::min<size_t>(pl->L.guards.size(), 64);
  for (int i = 0; i < gl.n; ++i) gl.off[i] = pl->L.guards[i];
  if (gl.n > 0) k_check_guards<<<gl.n, 128, 0, s>>>((const unsigned char *)ws, gl, pl->dbg_word);
  unsigned w = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&w, pl->dbg_word, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(pl->dbg_word, 0, 4, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return PHMM_ECUDA;
  return w ? PHMM_EGUARD : PHMM_OK;
}

// After a call (debug builds): check the guards and the kernels' index checks.
static int dbg_end(phmm_plan *pl, void *ws, void *stream, int rc) {
  if (!kDebug || rc != PHMM_OK || !pl || !ws) return rc;
  return dbg_check(pl, ws, stream);
}

// The kernels' debug fields (debug builds; otherwise no checks).
static void dbg_args(const phmm_plan *pl, FwdArgs &a) {
  if (!kDebug) return;
  a.dbg_err = pl->dbg_word;
  a.dbg_sum_m = pl->sum_m;
  a.dbg_hcode_bytes = (int64_t)hap_code_bytes(pl->sum_n, pl->b.n_haps);
}

// Zeroed counters and the per-row parameters and codes every sweep reads.
static int enqueue_prep(phmm_plan *pl, char *ws, cudaStream_t s, int *launches) {
  const WsLayout &L = pl->L;
  CK(cudaMemsetAsync(ws + L.zero, 0, L.zero_bytes, s));
  const int rc = launch_prep(pl->b, pl->sum_m, pl->beta32, (RowParams *)(ws + L.rp),
                             (uint8_t *)(ws + L.rcode), (uint8_t *)(ws + L.hcode),
                             pl->gq ? (float2 *)(ws + L.rgap) : nullptr, s, launches);
  if (rc) return cuda_fail((cudaError_t)rc);
  return PHMM_OK;
}

// The whole forward pass as a stream-ordered launch sequence (capturable).
// `timed`: record the plan's events around the FP32 and rescue kernels (not under capture).
static int enqueue_forward(phmm_plan *pl, char *ws, double *out, uint8_t *flags,
                           cudaStream_t s, bool timed) {
  const WsLayout &L = pl->L;
  const phmm_batch &b = pl->b;
  const phmm_options &o = pl->o;
  int launches = 0;
  int rc = enqueue_prep(pl, ws, s, &launches);
  if (rc) return rc;
  RowParams *rp = (RowParams *)(ws + L.rp);
  uint8_t *rcode = (uint8_t *)(ws + L.rcode), *hcode = (uint8_t *)(ws + L.hcode);
  int32_t *order = (int32_t *)(ws + L.order);
  int32_t *grp_begin = (int32_t *)(ws + L.grp_begin), *grp_count = (int32_t *)(ws + L.grp_count);
  if (o.binning && b.n_pairs > 0) {
    CfgTable tab;
    for (int m = 0; m <= PHMM_MAX_READ_LEN; ++m) tab.cfg[m] = (int8_t)pl->cfg_of_m[m];
    rc = launch_binning(b, tab, (int32_t *)(ws + L.key),
                        (int32_t *)(ws + L.counts), (int32_t *)(ws + L.offsets),
                        (int32_t *)(ws + L.cursor), grp_begin, grp_count, order, s, &launches);
    if (rc) return cuda_fail((cudaError_t)rc);
  }

  FwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.pair_read = b.pair_read;
  a.pair_hap = b.pair_hap;
  a.read_off = b.read_off;
  a.hap_off = b.hap_off;
  a.rp = rp;
  a.rcode = rcode;
  a.hcode = hcode;
  a.bq = b.base_q;
  a.iq = b.ins_q;
  a.dq = b.del_q;
  a.gq = b.gcp_q;
  a.rgap = pl->gq ? (const float2 *)(ws + L.rgap) : nullptr;
  a.qual_f32 = b.qual_dtype == PHMM_QUAL_F32;
  a.alpha_mode = b.alpha_mode;
  a.n_reads = b.n_reads;
  a.n_haps = b.n_haps;
  a.out = out;
  a.flags = flags;
  a.eps32 = pl->eps32;
  a.beta32 = pl->beta32;
  a.eps64 = pl->eps64;
  a.beta64 = pl->beta64;
  a.rescue = o.rescue;
  int32_t *rcnt = (int32_t *)(ws + L.rcnt), *xcnt = (int32_t *)(ws + L.xcnt);
  for (int k = 0; k < kNumCfg64; ++k) {
    a.rescue_list[k] = (int32_t *)(ws + L.rlist) + (size_t)k * std::max<int64_t>(b.n_pairs, 1);
  }
  a.rescue_count = rcnt;
  a.tilebuf = pl->L.tile ? (void *)(ws + L.tile) : nullptr;
  a.tile_cols = pl->n_max;
  dbg_args(pl, a);
  const bool ext = o.first_line == PHMM_FIRST_EXT32;
  a.mode = ext ? 1 : 0;
  const int block = 32 * o.warps_per_block;

  if (timed) CK(cudaEventRecord(pl->ev[0], s));
  if (b.n_pairs > 0) {
    if (o.binning) {
      for (int cfg : pl->used_cfgs) {
        FwdArgs c = a;
        c.list = order;
        c.offset_dev = grp_begin + cfg;
        c.count_dev = grp_count + cfg;
        c.counter = (int32_t *)(ws + L.ctr32) + cfg;
        c.persistent = 1;
        const int grid = pl->sms * std::max(1, fwd32_blocks_per_sm(cfg, ext, block, pl->gq));
        rc = launch_fwd32(cfg, ext, grid, block, s, c);
        if (rc) return cuda_fail((cudaError_t)rc);
        ++launches;
      }
    } else {
      const int cfg = cfg_index(o.lanes, o.rows);
      FwdArgs c = a;
      c.count = b.n_pairs;
      const int G = 32 / o.lanes;
      const int64_t items = (b.n_pairs + G - 1) / G;
      int grid;
      if (o.persistent) {
        c.persistent = 1;
        c.counter = (int32_t *)(ws + L.ctr32) + cfg;
        grid = pl->sms * std::max(1, fwd32_blocks_per_sm(cfg, ext, block));
      } else {
        grid = (int)((items + o.warps_per_block - 1) / o.warps_per_block);
        c.tilebuf = nullptr;  // buffers exist per resident warp of persistent launches only
      }
      rc = launch_fwd32(cfg, ext, grid, block, s, c);
      if (rc) return cuda_fail((cudaError_t)rc);
      ++launches;
    }
  }
  if (timed) CK(cudaEventRecord(pl->ev[1], s));
  if (o.rescue && b.n_pairs > 0) {
    // FP64 with K0 = 2^1020; failures go on to the per-lane-exponent FP64 kernel.
    for (int tier = 0; tier < 2; ++tier) {
      for (int k = 0; k < kNumCfg64; ++k) {
        FwdArgs c = a;
        c.mode = tier == 0 ? 2 : 3;
        c.list = (tier == 0 ? (int32_t *)(ws + L.rlist) : (int32_t *)(ws + L.xlist)) +
                 (size_t)k * std::max<int64_t>(b.n_pairs, 1);
        c.count_dev = (tier == 0 ? rcnt : xcnt) + k;
        c.counter = (int32_t *)(ws + (tier == 0 ? L.ctr64 : L.ctrx)) + k;
        c.persistent = 1;
        c.rescue = tier == 0 ? 1 : 0;
        for (int q = 0; q < kNumCfg64; ++q)
          c.rescue_list[q] = (int32_t *)(ws + L.xlist) + (size_t)q * std::max<int64_t>(b.n_pairs, 1);
        c.rescue_count = xcnt;
        const int grid = pl->sms * std::max(1, fwd64_blocks_per_sm(k, tier == 1, block, pl->gq));
        rc = launch_fwd64(k, tier == 1, grid, block, s, c);
        if (rc) return cuda_fail((cudaError_t)rc);
        ++launches;
      }
    }
  }
  if (timed) CK(cudaEventRecord(pl->ev[2], s));
  pl->launches_fwd = launches;
  return PHMM_OK;
}

extern "C" {

static int phmm_forward_body(phmm_plan *pl, void *ws, size_t ws_bytes, double *out, uint8_t *flags,
                 void *stream) {
  const phmm::NvtxRange nvtx("phmm_forward");
  if (!pl || !ws || (pl->b.n_pairs > 0 && (!out || !flags))) return PHMM_EINVAL;
  if (((uintptr_t)ws & 255) != 0) return PHMM_EINVAL;
  if (ws_bytes < pl->L.total) return PHMM_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();  // drop a stale error left by an unrelated call
  pl->timed = false;
  int rc;
  if (pl->o.use_graph) {
    if (!pl->gexec || pl->g_ws != ws || pl->g_out != out || pl->g_flags != flags) {
      if (pl->gexec) {
        cudaGraphExecDestroy(pl->gexec);
        pl->gexec = nullptr;
      }
      CK(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_forward(pl, (char *)ws, out, flags, pl->cap, false);
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamEndCapture(pl->cap, &g);
      if (rc != PHMM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ce != cudaSuccess) return cuda_fail(ce);
      ce = cudaGraphInstantiate(&pl->gexec, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return cuda_fail(ce);
      pl->g_ws = ws;
      pl->g_out = out;
      pl->g_flags = flags;
    }
    CK(cudaGraphLaunch(pl->gexec, s));
    rc = PHMM_OK;
  } else {
    rc = enqueue_forward(pl, (char *)ws, out, flags, s, true);
    pl->timed = rc == PHMM_OK;
  }
  if (rc == PHMM_OK) pl->fwd_done = true;
  return rc;
}

int phmm_forward(phmm_plan *pl, void *ws, size_t ws_bytes, double *out, uint8_t *flags,
                 void *stream) {
  int rc = dbg_begin(pl, ws, ws_bytes, stream);
  if (rc == PHMM_OK) rc = phmm_forward_body(pl, ws, ws_bytes, out, flags, stream);
  return dbg_end(pl, ws, stream, rc);
}

static int phmm_backward_body(phmm_plan *pl, void *ws, size_t ws_bytes, const double *dL, float *dbq,
                  float *diq, float *ddq, float *dgq, double *dgcp, void *stream) {
  const phmm::NvtxRange nvtx("phmm_backward");
  if (!pl || !ws || !dgcp) return PHMM_EINVAL;
  if (pl->sum_m > 0 && (!dbq || !diq || !ddq || (pl->gq && !dgq))) return PHMM_EINVAL;
  if (pl->b.n_pairs > 0 && !dL) return PHMM_EINVAL;
  if (((uintptr_t)ws & 255) != 0) return PHMM_EINVAL;
  if (ws_bytes < pl->L.total) return PHMM_ENOMEM;
  if (!pl->fwd_done) return PHMM_ESTATE;
  (void)cudaGetLastError();
  int launches = 0;
  pl->bwd_timed = false;
  pl->partials_done = false;  // the sweep overwrites the partials with scaled ones
  pl->red_from = 4;
  int rc = bwd_enqueue_impl(pl, (char *)ws, dL, dbq, diq, ddq, pl->gq ? dgq : nullptr, dgcp,
                            (cudaStream_t)stream, &launches, pl->ev + 3);
  pl->launches_bwd = launches;
  if (rc) return cuda_fail((cudaError_t)rc);
  pl->bwd_timed = true;
  return PHMM_OK;
}

int phmm_backward(phmm_plan *pl, void *ws, size_t ws_bytes, const double *dL, float *dbq,
                  float *diq, float *ddq, float *dgq, double *dgcp, void *stream) {
  int rc = dbg_begin(pl, ws, ws_bytes, stream);
  if (rc == PHMM_OK) rc = phmm_backward_body(pl, ws, ws_bytes, dL, dbq, diq, ddq, dgq, dgcp, stream);
  return dbg_end(pl, ws, stream, rc);
}

static int phmm_forward_partials_body(phmm_plan *pl, void *ws, size_t ws_bytes, double *out,
                          uint8_t *flags, void *stream) {
  const phmm::NvtxRange nvtx("phmm_forward_partials");
  if (!pl || !ws || (pl->b.n_pairs > 0 && (!out || !flags))) return PHMM_EINVAL;
  if (((uintptr_t)ws & 255) != 0) return PHMM_EINVAL;
  if (ws_bytes < pl->L.total) return PHMM_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  pl->bwd_timed = false;
  pl->partials_done = false;
  const void *key_fp[3] = {ws, out, flags};
  const bool repeat_fp = std::memcmp(key_fp, pl->gfp_prev, sizeof(key_fp)) == 0;
  std::memcpy(pl->gfp_prev, key_fp, sizeof(key_fp));
  const bool replay_fp = pl->gexec_fp && std::memcmp(key_fp, pl->gfp_key, sizeof(key_fp)) == 0;
  if (pl->o.use_graph && pl->cells <= kGraphCells && (replay_fp || repeat_fp)) {
    const void *(&key)[3] = key_fp;
    if (!replay_fp) {
      int n = 0;
      const int rc = capture_graph(pl, &pl->gexec_fp, [&](cudaStream_t cs) {
        int r = enqueue_prep(pl, (char *)ws, cs, &n);
        if (r) return r;
        return bwd_sweep_impl(pl, (char *)ws, nullptr, out, flags, cs, &n, pl->ev + 3);
      });
      if (rc) return rc;
      std::memcpy(pl->gfp_key, key, sizeof(key));
      pl->gfp_launches = n;
    }
    CK(cudaGraphLaunch(pl->gexec_fp, s));
    pl->launches_fwd = pl->gfp_launches;
  } else {
    int launches = 0;
    int rc = enqueue_prep(pl, (char *)ws, s, &launches);
    if (rc) return rc;
    rc = bwd_sweep_impl(pl, (char *)ws, nullptr, out, flags, s, &launches, pl->ev + 3);
    pl->launches_fwd = launches;
    if (rc) return cuda_fail((cudaError_t)rc);
  }
  pl->fwd_done = true;
  pl->partials_done = true;
  return PHMM_OK;
}

int phmm_forward_partials(phmm_plan *pl, void *ws, size_t ws_bytes, double *out,
                          uint8_t *flags, void *stream) {
  int rc = dbg_begin(pl, ws, ws_bytes, stream);
  if (rc == PHMM_OK) rc = phmm_forward_partials_body(pl, ws, ws_bytes, out, flags, stream);
  return dbg_end(pl, ws, stream, rc);
}

static int phmm_backward_partials_body(phmm_plan *pl, void *ws, size_t ws_bytes, const double *dL,
                           float *dbq, float *diq, float *ddq, float *dgq, double *dgcp,
                           void *stream) {
  const phmm::NvtxRange nvtx("phmm_backward_partials");
  if (!pl || !ws || !dgcp) return PHMM_EINVAL;
  if (pl->sum_m > 0 && (!dbq || !diq || !ddq || (pl->gq && !dgq))) return PHMM_EINVAL;
  if (pl->b.n_pairs > 0 && !dL) return PHMM_EINVAL;
  if (((uintptr_t)ws & 255) != 0) return PHMM_EINVAL;
  if (ws_bytes < pl->L.total) return PHMM_ENOMEM;
  if (!pl->partials_done) return PHMM_ESTATE;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  float *gq = pl->gq ? dgq : nullptr;
  const void *key_bp[7] = {ws, dL, dbq, diq, ddq, gq, dgcp};
  const bool repeat_bp = std::memcmp(key_bp, pl->gbp_prev, sizeof(key_bp)) == 0;
  std::memcpy(pl->gbp_prev, key_bp, sizeof(key_bp));
  const bool replay_bp = pl->gexec_bp && std::memcmp(key_bp, pl->gbp_key, sizeof(key_bp)) == 0;
  if (pl->o.use_graph && pl->cells <= kGraphCells && (replay_bp || repeat_bp)) {
    const void *(&key)[7] = key_bp;
    if (!replay_bp) {
      int n = 0;
      const int rc = capture_graph(pl, &pl->gexec_bp, [&](cudaStream_t cs) {
        return bwd_reduce_impl(pl, (char *)ws, dL, dbq, diq, ddq, gq, dgcp, cs, &n, pl->ev[5]);
      });
      if (rc) return rc;
      std::memcpy(pl->gbp_key, key, sizeof(key));
      pl->gbp_launches = n;
    }
    CK(cudaGraphLaunch(pl->gexec_bp, s));
    pl->launches_bwd = pl->gbp_launches;
    pl->bwd_timed = false;  // kernel times are recorded by eager calls only
    return PHMM_OK;
  }
  int launches = 0;
  pl->red_from = 6;
  CK(cudaEventRecord(pl->ev[6], s));
  const int rc = bwd_reduce_impl(pl, (char *)ws, dL, dbq, diq, ddq, gq, dgcp, s, &launches,
                                 pl->ev[5]);
  pl->launches_bwd = launches;
  if (rc) return cuda_fail((cudaError_t)rc);
  pl->bwd_timed = true;
  return PHMM_OK;
}

int phmm_backward_partials(phmm_plan *pl, void *ws, size_t ws_bytes, const double *dL,
                           float *dbq, float *diq, float *ddq, float *dgq, double *dgcp,
                           void *stream) {
  int rc = dbg_begin(pl, ws, ws_bytes, stream);
  if (rc == PHMM_OK) rc = phmm_backward_partials_body(pl, ws, ws_bytes, dL, dbq, diq, ddq, dgq, dgcp, stream);
  return dbg_end(pl, ws, stream, rc);
}

int phmm_plan_launch_count(const phmm_plan *pl, int which) {
  if (!pl) return -1;
  return which == 0 ? pl->launches_fwd : pl->launches_bwd;
}

int phmm_plan_wavefront_ms(phmm_plan *pl, float *ms_fp32, float *ms_rescue) {
  if (!pl) return PHMM_EINVAL;
  float a = -1.f, r = -1.f;
  if (pl->timed && cudaEventQuery(pl->ev[2]) == cudaSuccess) {
    if (cudaEventElapsedTime(&a, pl->ev[0], pl->ev[1]) != cudaSuccess) a = -1.f;
    if (cudaEventElapsedTime(&r, pl->ev[1], pl->ev[2]) != cudaSuccess) r = -1.f;
  }
  if (ms_fp32) *ms_fp32 = a;
  if (ms_rescue) *ms_rescue = r;
  return PHMM_OK;
}

int phmm_plan_rescue_counts(phmm_plan *pl, const void *ws, void *stream, int64_t *counts) {
  if (!pl || !ws || !counts) return PHMM_EINVAL;
  int32_t h[4 * kNumCfg64 + 4];
  const char *w = (const char *)ws;
  cudaStream_t s = (cudaStream_t)stream;
  // the forward's FP32->FP64 and FP64->extended counts, and the adjoint's FP32->FP64 count
  // (kept in the slot after the forward's work counters, see the backward launch sequence)
  CK(cudaMemcpyAsync(h, w + pl->L.rcnt, 4 * kNumCfg64, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h + kNumCfg64, w + pl->L.xcnt, 4 * kNumCfg64, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h + 2 * kNumCfg64, w + pl->L.ctr64, 4 * kNumCfg64, cudaMemcpyDeviceToHost,
                     s));
  CK(cudaMemcpyAsync(h + 3 * kNumCfg64, w + pl->L.why, 16, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  counts[0] = counts[1] = counts[2] = 0;
  counts[3] = h[3 * kNumCfg64];      // adjoint hand-offs for the scale range
  counts[4] = h[3 * kNumCfg64 + 1];  // adjoint hand-offs for non-finite partials
  counts[5] = 0;
  for (int k = 0; k < kNumCfg64; ++k) {
    counts[0] += h[k];
    counts[1] += h[kNumCfg64 + k];
    counts[2] += h[2 * kNumCfg64 + k];
  }
  return PHMM_OK;
}

int phmm_plan_backward_ms(phmm_plan *pl, float *ms_adjoint, float *ms_reduce) {
  if (!pl) return PHMM_EINVAL;
  float a = -1.f, r = -1.f;
  if (pl->bwd_timed && cudaEventQuery(pl->ev[5]) == cudaSuccess) {
    if (cudaEventElapsedTime(&a, pl->ev[3], pl->ev[4]) != cudaSuccess) a = -1.f;
    if (cudaEventElapsedTime(&r, pl->ev[pl->red_from], pl->ev[5]) != cudaSuccess) r = -1.f;
  }
  if (ms_adjoint) *ms_adjoint = a;
  if (ms_reduce) *ms_reduce = r;
  return PHMM_OK;
}

}  // extern "C"

extern "C" {

int phmm_debug_guard_offset(const phmm_plan *pl, int k, size_t *offset) {
  if (!kDebug) return PHMM_ESTATE;
  if (!pl || !offset || k < 0 || k >= (int)pl->L.guards.size()) return PHMM_EINVAL;
  *offset = pl->L.guards[k];
  return PHMM_OK;
}

int phmm_debug_check(phmm_plan *pl, void *ws, void *stream) {
  if (!kDebug) return PHMM_ESTATE;
  if (!pl || !ws) return PHMM_EINVAL;
  return dbg_check(pl, ws, stream);
}

}  // extern "C"

// Accessors used by the backward translation unit.
namespace phmm {
const phmm_batch &plan_batch(const phmm_plan *pl) { return pl->b; }
const phmm_options &plan_options(const phmm_plan *pl) { return pl->o; }
size_t plan_bwd_offset(const phmm_plan *pl) { return pl->L.bwd; }
int64_t plan_sum_m(const phmm_plan *pl) { return pl->sum_m; }
int plan_sms(const phmm_plan *pl) { return pl->sms; }
void **plan_bwd_state(phmm_plan *pl) { return &pl->bwd_state; }
size_t plan_layout_rp(const phmm_plan *pl) { return pl->L.rp; }
size_t plan_layout_rcode(const phmm_plan *pl) { return pl->L.rcode; }
size_t plan_layout_hcode(const phmm_plan *pl) { return pl->L.hcode; }
double plan_eps64(const phmm_plan *pl) { return pl->eps64; }
int64_t plan_n_max(const phmm_plan *pl) { return pl->n_max; }
int64_t plan_pair_rows(const phmm_plan *pl) { return pl->pair_rows; }
int plan_max_m(const phmm_plan *pl) { return pl->max_m; }
bool plan_gq(const phmm_plan *pl) { return pl->gq; }
unsigned *plan_dbg_word(const phmm_plan *pl) { return kDebug ? pl->dbg_word : nullptr; }
int64_t plan_hcode_bytes(const phmm_plan *pl) {
  return (int64_t)hap_code_bytes(pl->sum_n, pl->b.n_haps);
}
size_t plan_layout_rgap(const phmm_plan *pl) { return pl->L.rgap; }
const int *plan_bwd_cfg_of_m(const phmm_plan *pl) { return pl->bwd_cfg_of_m; }
const std::vector<int> &plan_bwd_used(const phmm_plan *pl) { return pl->bwd_used; }
// 0 counts, 1 key, 2 offsets, 3 cursor, 4 grp_begin, 5 grp_count, 6 order, 7 ctr32,
// 8 rescue lists, 9 (bytes the adjoint zeroes from counts on: up to the forward's rescue counts)
size_t plan_layout_bin(const phmm_plan *pl, int which) {
  const WsLayout &L = pl->L;
  const size_t v[11] = {L.counts,    L.key,   L.offsets, L.cursor,          L.grp_begin,
                        L.grp_count, L.order, L.ctr32,   L.rlist,           L.rcnt - L.counts,
                        L.why};
  return v[which];
}
}  // namespace phmm
