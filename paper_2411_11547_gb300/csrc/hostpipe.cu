// End-to-end scoring of a batch held in host memory: the host workflow of Sec. III-A
// (partition into subsets, transfer, score, transfer back), with the copies of one subset
// overlapping the scoring of the previous one; and the same pipeline for the gradient.
//
// Pairs are grouped by read (every pair of a read in one subset) and cut into subsets of
// about `subset_cells` cells.  Per subset the host packs the reads, the haplotypes the pairs
// use (renumbered) and the pairs into one pinned staging buffer, which goes to the device in
// one copy; the subset is then validated and scored through the library's own plan and
// forward on one of two streams, and its log10 L and flags come back by one copy each.  While
// the GPU scores subset k on one stream, the host packs subset k+1 and starts its copy on
// the other.  In the gradient mode the subset's dL travels with its inputs, the plan runs the
// fused step (forward with partials, then the reduction weighted by dL), and the subset's
// per-read gradients come back with its results: a subset holds whole reads, so their
// gradients are complete there, and the d/dgcp of the subsets are summed in subset order.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>
#include "phmm.h"
#include "phmm_internal.cuh"

namespace {

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Slot {
  cudaStream_t s = nullptr;
  unsigned char *stage = nullptr;  // pinned: packed inputs
  size_t stage_cap = 0;
  unsigned char *dev = nullptr;    // device: packed inputs, then log10 L and flags
  size_t dev_cap = 0;
  void *ws = nullptr;              // device: workspace
  size_t ws_cap = 0;
  unsigned char *hres = nullptr;   // pinned: log10 L and flags of the subset
  size_t hres_cap = 0;
  phmm_plan *plan = nullptr;
  std::vector<int64_t> pairs;      // global pair ids of the subset in flight (if scattered)
  bool contiguous = false;         // else: the pairs are p0 .. p0 + np - 1
  int64_t p0 = 0, np = 0;
  int64_t b0 = 0, sm = 0;          // the subset's reads: bases b0 .. b0 + sm - 1
  size_t res_off = 0;              // offset of the results in dev / hres
  size_t grad_off = 0;             // offset of the gradients within the results
  bool busy = false;
};

// Where a pipeline call writes (host memory); the gradient arrays are null when scoring only.
struct HostOut {
  double *log10;
  uint8_t *flags;
  float *gb, *gi, *gd;
  double *gg;
  float *gq;  // per-base gap-continuation gradients (batches with a track), else null
};

// memcpy split over host threads (large copies only)
void par_copy(void *dst, const void *src, size_t bytes) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t T = std::min<size_t>({(size_t)hw, (size_t)16, bytes / (4u << 20) + 1});
  if (T <= 1) {
    std::memcpy(dst, src, bytes);
    return;
  }
  std::vector<std::thread> th;
  const size_t chunk = (bytes + T - 1) / T;
  for (size_t i = 0; i < T; ++i) {
    const size_t a = i * chunk, b = std::min(bytes, a + chunk);
    if (a < b)
      th.emplace_back([=] { std::memcpy((char *)dst + a, (const char *)src + a, b - a); });
  }
  for (auto &t : th) t.join();
}

int grow_pinned(unsigned char **p, size_t *cap, size_t need) {
  if (need <= *cap) return 0;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost((void **)p, need) != cudaSuccess) return PHMM_ENOMEM;
  *cap = need;
  return 0;
}
int grow_device(void **p, size_t *cap, size_t need) {
  if (need <= *cap) return 0;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need) != cudaSuccess) return PHMM_ENOMEM;
  *cap = need;
  return 0;
}

// Wait for a slot's subset and scatter its results to the caller's arrays.
int drain(Slot &sl, const HostOut &o) {
  if (!sl.busy) return 0;
  if (cudaStreamSynchronize(sl.s) != cudaSuccess) return PHMM_ECUDA;
  const size_t np = (size_t)sl.np;
  const double *r = (const double *)sl.hres;
  const uint8_t *f = (const uint8_t *)(sl.hres + up(8 * np));
  if (sl.contiguous) {
    par_copy(o.log10 + sl.p0, r, 8 * np);
    std::memcpy(o.flags + sl.p0, f, np);
  } else {
    for (size_t i = 0; i < np; ++i) {
      o.log10[sl.pairs[i]] = r[i];
      o.flags[sl.pairs[i]] = f[i];
    }
  }
  if (o.gb) {
    const unsigned char *g = sl.hres + sl.grad_off;
    const size_t gbytes = 4 * (size_t)sl.sm;
    par_copy(o.gb + sl.b0, g, gbytes);
    par_copy(o.gi + sl.b0, g + up(gbytes), gbytes);
    par_copy(o.gd + sl.b0, g + 2 * up(gbytes), gbytes);
    if (o.gq) par_copy(o.gq + sl.b0, g + 3 * up(gbytes), gbytes);
    double gg;
    std::memcpy(&gg, g + (o.gq ? 4 : 3) * up(gbytes), 8);
    *o.gg += gg;
  }
  phmm_plan_destroy(sl.plan);
  sl.plan = nullptr;
  sl.busy = false;
  return 0;
}

// 1 if kernels on device `dev` may read pageable host memory in place (coherent host access
// through the host's page tables, as on Grace-Blackwell over NVLink-C2C).
bool host_direct(int dev) {
  static int cached[64] = {};  // 0 unknown, 1 no, 2 yes
  int &c = cached[dev & 63];
  if (!c) {
    int v = 0, w = 0;
    const bool ok =
        cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&w, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) ==
            cudaSuccess;
    c = ok && v && w ? 2 : 1;
  }
  return c == 2;
}

// Staging and device buffers kept between calls (pinned allocations are slow to make), for
// the device they were made on; one call at a time uses them.
struct Cache {
  std::mutex mu;
  int device = -1;
  Slot slot[2];
};
Cache &cache() {
  static Cache c;
  return c;
}
void release_slots(Slot (&slot)[2]) {
  for (auto &sl : slot) {
    if (sl.stage) cudaFreeHost(sl.stage);
    if (sl.hres) cudaFreeHost(sl.hres);
    if (sl.dev) cudaFree(sl.dev);
    if (sl.ws) cudaFree(sl.ws);
    if (sl.s) cudaStreamDestroy(sl.s);
    sl = Slot();
  }
}

}  // namespace

extern "C" void phmm_score_host_release(void) {
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  release_slots(c.slot);
  c.device = -1;
}

// The pipeline behind phmm_score_host (dL null) and phmm_grad_host.
static int host_pipeline(const phmm_batch *hb, const phmm_options *opt, int64_t subset_cells,
                         const double *dL, const HostOut &ho_) {
  double *out_log10 = ho_.log10;
  if (!hb || !out_log10 || !ho_.flags || subset_cells < 1) return PHMM_EINVAL;
  const bool grad = dL != nullptr;
  const phmm_batch &b = *hb;
  if (b.n_reads < 1 || b.n_haps < 1 || b.n_pairs < 0) return PHMM_EINVAL;
  if (!b.read_bases || !b.base_q || !b.ins_q || !b.del_q || !b.read_off || !b.hap_bases ||
      !b.hap_off || (b.n_pairs > 0 && (!b.pair_read || !b.pair_hap)))
    return PHMM_EINVAL;
  if (grad && (!ho_.gb || !ho_.gi || !ho_.gd || !ho_.gg)) return PHMM_EINVAL;
  const bool gqt = b.gcp_q != nullptr;  // per-base gap-continuation track
  if (grad && gqt && !ho_.gq) return PHMM_EINVAL;
  HostOut hout = ho_;
  if (!gqt) hout.gq = nullptr;
  const int64_t R = b.n_reads, H = b.n_haps, P = b.n_pairs;
  const int64_t *ro = b.read_off, *ho = b.hap_off;
  if (ro[0] != 0 || ho[0] != 0) return PHMM_EINVAL;
  for (int64_t r = 0; r < R; ++r)
    if (ro[r + 1] <= ro[r]) return PHMM_EINVAL;
  for (int64_t h = 0; h < H; ++h)
    if (ho[h + 1] <= ho[h]) return PHMM_EINVAL;
  if (grad) {  // reads without pairs keep zero gradients
    *ho_.gg = 0.0;
    const size_t sm_all = (size_t)ro[R] * 4;
    std::memset(ho_.gb, 0, sm_all);
    std::memset(ho_.gi, 0, sm_all);
    std::memset(ho_.gd, 0, sm_all);
    if (gqt) std::memset(ho_.gq, 0, sm_all);
  }
  if (P == 0) return PHMM_OK;
  // pairs grouped by read: already so when pair_read is non-decreasing (all-vs-all batches
  // list a read's pairs together), else by a counting sort
  std::vector<int64_t> rptr(R + 1, 0), rpairs;
  bool sorted = true;
  for (int64_t p = 0; p < P; ++p) {
    const int32_t r = b.pair_read[p], h = b.pair_hap[p];
    if (r < 0 || r >= R || h < 0 || h >= H) return PHMM_EINVAL;
    ++rptr[r + 1];
    if (p && r < b.pair_read[p - 1]) sorted = false;
  }
  for (int64_t r = 0; r < R; ++r) rptr[r + 1] += rptr[r];
  if (!sorted) {
    rpairs.resize(P);
    std::vector<int64_t> cur(rptr.begin(), rptr.end() - 1);
    for (int64_t p = 0; p < P; ++p) rpairs[cur[b.pair_read[p]]++] = p;
  }
  auto pair_at = [&](int64_t i) { return sorted ? i : rpairs[i]; };
  phmm_options o;
  if (opt) o = *opt; else phmm_options_default(&o);
  o.use_graph = 0;  // one forward per plan: no graph to replay
  const int qe = b.qual_dtype == PHMM_QUAL_F32 ? 4 : 1;

  Cache &cc = cache();
  std::lock_guard<std::mutex> lock(cc.mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PHMM_ECUDA;
  if (cc.device != dev) {  // buffers of another device: start afresh
    release_slots(cc.slot);
    cc.device = dev;
  }
  Slot(&slot)[2] = cc.slot;
  // Forward scoring with coherent host access: the kernels read the subset's bases, qualities
  // and (contiguous) haplotypes where they lie, and only offsets and pair ids are packed and
  // copied (host packing bounds this path).  The gradient keeps the copies: its subsets run
  // long adjoint kernels, and reading in place from kernels that must wait for SMs measured
  // slower than copy-engine transfers that overlap them.
  const bool direct = !grad && host_direct(dev);
  int rc = 0;
  for (auto &sl : slot)
    if (!sl.s && cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess)
      rc = PHMM_ECUDA;
  std::vector<int64_t> hmark(H, -1);
  std::vector<int32_t> hmap(H, 0);
  int64_t lo = 0, k = 0;
  // Gradient mode: subset sizes ramp up over the first subsets (1/8, 1/4, 1/2 of
  // subset_cells) and halve over the last ones (down to 1/8), so the copies and host packing
  // that nothing overlaps, the first subset's inputs and the last one's results, stay small.
  // A forward subset is short on the GPU (about 1/20 of a gradient subset's time per cell):
  // there the extra subsets' fixed costs outweigh that (measured), so its size is fixed.
  int64_t left = 0;
  for (int64_t r = 0; grad && r < R; ++r) {
    const int64_t m = ro[r + 1] - ro[r];
    for (int64_t i = rptr[r]; i < rptr[r + 1]; ++i) {
      const int32_t h = b.pair_hap[pair_at(i)];
      left += m * (ho[h + 1] - ho[h]);
    }
  }
  while (rc == 0 && lo < R) {
    // the next subset: whole reads up to about `target` cells
    int64_t target = subset_cells;
    if (grad) {
      if (k < 3) target = subset_cells >> (3 - k);
      if (left < 2 * target) target = std::max(left / 2, subset_cells / 8);
    }
    target = std::max<int64_t>(target, 1);
    int64_t hi = lo, cells = 0;
    int32_t hmin = INT32_MAX, hmax = -1;  // the haplotypes the subset's pairs use
    while (hi < R && (hi == lo || cells < target)) {
      const int64_t m = ro[hi + 1] - ro[hi];
      for (int64_t i = rptr[hi]; i < rptr[hi + 1]; ++i) {
        const int32_t h = b.pair_hap[pair_at(i)];
        cells += m * (ho[h + 1] - ho[h]);
        hmin = std::min(hmin, h);
        hmax = std::max(hmax, h);
      }
      ++hi;
    }
    left -= cells;
    Slot &sl = slot[k & 1];
    if ((rc = drain(sl, hout))) break;
    // the subset's pairs and haplotypes.  Fast path: the pairs are one contiguous range and
    // the haplotypes they use fill most of one contiguous range [hmin, hmax], which is then
    // copied whole and renumbered by offset; otherwise haplotypes are renumbered in
    // first-use order and gathered one by one.
    const int64_t p0 = rptr[lo], np = rptr[hi] - rptr[lo], nr = hi - lo;
    if (np == 0) {  // reads without pairs: nothing to score (their gradients stay zero)
      lo = hi;
      continue;
    }
    sl.contiguous = sorted;
    sl.p0 = p0;
    if (sorted) sl.pairs.clear();
    else sl.pairs.assign(rpairs.begin() + p0, rpairs.begin() + rptr[hi]);
    sl.np = np;
    std::vector<int32_t> haps;
    int64_t sn = 0;
    bool hrange = false;
    if ((int64_t)(hmax - hmin + 1) <= 2 * np + 16) {
      hrange = true;
      sn = ho[hmax + 1] - ho[hmin];
    } else {
      for (int64_t i = 0; i < np; ++i) {
        const int32_t h = b.pair_hap[pair_at(p0 + i)];
        if (hmark[h] != k) {
          hmark[h] = k;
          hmap[h] = (int32_t)haps.size();
          haps.push_back(h);
          sn += ho[h + 1] - ho[h];
        }
      }
    }
    const int64_t nh = hrange ? (int64_t)(hmax - hmin + 1) : (int64_t)haps.size();
    const int64_t sm = ro[hi] - ro[lo];
    // packed layout: bases, 3 quals, read offsets, haplotype bases and offsets, pair ids,
    // (gradient mode) the pairs' dL, and the gap-continuation track
    size_t off[11], tot = 0;
    const size_t rb = direct ? 0 : (size_t)sm;           // read bases / quals staged
    const size_t hb = direct && hrange ? 0 : (size_t)sn;   // haplotype bases staged
    const size_t sz[11] = {rb, rb * qe, rb * qe, rb * qe, (size_t)(nr + 1) * 8, hb,
                           (size_t)(nh + 1) * 8, (size_t)np * 4, (size_t)np * 4,
                           grad ? (size_t)np * 8 : 0, gqt ? rb * qe : 0};
    for (int i = 0; i < 11; ++i) {
      off[i] = tot;
      tot += up(sz[i]);
    }
    sl.res_off = tot;
    sl.b0 = ro[lo];
    sl.sm = sm;
    // results: log10 L, flags, and (gradient mode) the three per-base gradients and d/dgcp
    sl.grad_off = up(8 * (size_t)np) + up((size_t)np);
    const size_t res = sl.grad_off + (grad ? (gqt ? 4 : 3) * up(4 * (size_t)sm) + up(8) : 0);
    if ((rc = grow_pinned(&sl.stage, &sl.stage_cap, tot))) break;
    if ((rc = grow_pinned(&sl.hres, &sl.hres_cap, res))) break;
    if ((rc = grow_device((void **)&sl.dev, &sl.dev_cap, tot + res))) break;
    unsigned char *st = sl.stage;
    if (!direct) {
      par_copy(st + off[0], b.read_bases + ro[lo], sm);
      par_copy(st + off[1], (const unsigned char *)b.base_q + ro[lo] * qe, sm * qe);
      par_copy(st + off[2], (const unsigned char *)b.ins_q + ro[lo] * qe, sm * qe);
      par_copy(st + off[3], (const unsigned char *)b.del_q + ro[lo] * qe, sm * qe);
      if (gqt) par_copy(st + off[10], (const unsigned char *)b.gcp_q + ro[lo] * qe, sm * qe);
    }
    int64_t *sro = (int64_t *)(st + off[4]);
    for (int64_t r = 0; r <= nr; ++r) sro[r] = ro[lo + r] - ro[lo];
    int64_t *sho = (int64_t *)(st + off[6]);
    sho[0] = 0;
    if (hrange) {
      if (!direct) par_copy(st + off[5], b.hap_bases + ho[hmin], sn);
      for (int64_t i = 0; i <= nh; ++i) sho[i] = ho[hmin + i] - ho[hmin];
    } else {
      for (int64_t i = 0; i < nh; ++i) {
        const int32_t h = haps[i];
        const int64_t n = ho[h + 1] - ho[h];
        std::memcpy(st + off[5] + sho[i], b.hap_bases + ho[h], n);
        sho[i + 1] = sho[i] + n;
      }
    }
    int32_t *spr = (int32_t *)(st + off[7]), *sph = (int32_t *)(st + off[8]);
    double *sdl = (double *)(st + off[9]);
    for (int64_t i = 0; i < np; ++i) {
      const int64_t p = pair_at(p0 + i);
      spr[i] = (int32_t)(b.pair_read[p] - lo);
      sph[i] = hrange ? b.pair_hap[p] - hmin : hmap[b.pair_hap[p]];
    }
    if (grad) {
      if (sorted) par_copy(sdl, dL + p0, 8 * (size_t)np);
      else for (int64_t i = 0; i < np; ++i) sdl[i] = dL[pair_at(p0 + i)];
    }
    if (cudaMemcpyAsync(sl.dev, st, tot, cudaMemcpyHostToDevice, sl.s) != cudaSuccess) {
      rc = PHMM_ECUDA;
      break;
    }
    phmm_batch d = b;
    d.n_reads = nr;
    d.n_haps = nh;
    d.n_pairs = np;
    if (direct) {
      d.read_bases = b.read_bases + ro[lo];
      d.base_q = (const unsigned char *)b.base_q + ro[lo] * qe;
      d.ins_q = (const unsigned char *)b.ins_q + ro[lo] * qe;
      d.del_q = (const unsigned char *)b.del_q + ro[lo] * qe;
      if (gqt) d.gcp_q = (const unsigned char *)b.gcp_q + ro[lo] * qe;
    } else {
      d.read_bases = sl.dev + off[0];
      d.base_q = sl.dev + off[1];
      d.ins_q = sl.dev + off[2];
      d.del_q = sl.dev + off[3];
      if (gqt) d.gcp_q = sl.dev + off[10];
    }
    d.read_off = (const int64_t *)(sl.dev + off[4]);
    d.hap_bases = direct && hrange ? b.hap_bases + ho[hmin] : sl.dev + off[5];
    d.hap_off = (const int64_t *)(sl.dev + off[6]);
    d.pair_read = (const int32_t *)(sl.dev + off[7]);
    d.pair_hap = (const int32_t *)(sl.dev + off[8]);
    // validation waits for this stream only: the other stream's subset keeps the GPU busy
    if ((rc = phmm_plan_create(&d, &o, sl.s, &sl.plan))) break;
    const size_t wsb = phmm_workspace_bytes(sl.plan);
    if ((rc = grow_device(&sl.ws, &sl.ws_cap, wsb + 256))) break;
    double *dout = (double *)(sl.dev + sl.res_off);
    uint8_t *dfl = (uint8_t *)(sl.dev + sl.res_off + up(8 * (size_t)np));
    if (grad) {
      unsigned char *g = sl.dev + sl.res_off + sl.grad_off;
      const size_t gbytes = up(4 * (size_t)sm);
      if ((rc = phmm_forward_partials(sl.plan, sl.ws, wsb, dout, dfl, sl.s))) break;
      if ((rc = phmm_backward_partials(sl.plan, sl.ws, wsb, (const double *)(sl.dev + off[9]),
                                       (float *)g, (float *)(g + gbytes),
                                       (float *)(g + 2 * gbytes),
                                       gqt ? (float *)(g + 3 * gbytes) : nullptr,
                                       (double *)(g + (gqt ? 4 : 3) * gbytes), sl.s)))
        break;
    } else {
      if ((rc = phmm_forward(sl.plan, sl.ws, wsb, dout, dfl, sl.s))) break;
    }
    if (cudaMemcpyAsync(sl.hres, sl.dev + sl.res_off, res, cudaMemcpyDeviceToHost, sl.s) !=
        cudaSuccess) {
      rc = PHMM_ECUDA;
      break;
    }
    sl.busy = true;
    lo = hi;
    ++k;
  }
  for (auto &sl : slot) {
    const int r2 = rc ? (cudaStreamSynchronize(sl.s), 0) : drain(sl, hout);
    if (!rc) rc = r2;
    if (sl.plan) phmm_plan_destroy(sl.plan);
    sl.plan = nullptr;
    sl.busy = false;
  }
  if (rc) {  // after an error, give the buffers back
    release_slots(slot);
    cc.device = -1;
  }
  return rc;
}

extern "C" int phmm_score_host(const phmm_batch *hb, const phmm_options *opt,
                               int64_t subset_cells, double *out_log10, uint8_t *out_flags) {
  const phmm::NvtxRange nvtx("phmm_score_host");
  return host_pipeline(hb, opt, subset_cells, nullptr,
                       HostOut{out_log10, out_flags, nullptr, nullptr, nullptr, nullptr, nullptr});
}

extern "C" int phmm_grad_host(const phmm_batch *hb, const phmm_options *opt,
                              int64_t subset_cells, const double *dL, double *out_log10,
                              uint8_t *out_flags, float *d_base_q, float *d_ins_q,
                              float *d_del_q, float *d_gcp_q, double *d_gcp) {
  const phmm::NvtxRange nvtx("phmm_grad_host");
  if (!dL) return PHMM_EINVAL;
  return host_pipeline(hb, opt, subset_cells, dL,
                       HostOut{out_log10, out_flags, d_base_q, d_ins_q, d_del_q, d_gcp, d_gcp_q});
}
