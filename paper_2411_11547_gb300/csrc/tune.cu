// Autotuner of the read-length -> group tables (lanes per pair x rows per lane).
//
// The paper picks rows per thread by read length (Sec. III-C) from fixed bins; the best
// group for a length also depends on the haplotype lengths it meets (wavefront fill and
// drain, L - 1 idle steps per pair) and on register pressure, so here the tables are
// measured on the batch itself: for each 16-row read-length range that holds pairs, a
// strided sample of that range's pairs is gathered into a compact batch and every built
// group whose capacity covers the range is timed (CUDA events around the library's own
// forward or adjoint); the fastest wins the range's table entries.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>
#include "phmm.h"
#include "phmm_internal.cuh"

namespace phmm {
int bwd_cfg_supported(int cfg);
int fwd_cfg_supported(int cfg);
int bwd_default_cfg(int m);
int default_cfg_of_m(int m);
}

namespace {

using namespace phmm;

__global__ void k_gather_segments(const int64_t *__restrict__ src_off,
                                  const int64_t *__restrict__ dst_off,
                                  const int64_t *__restrict__ len, int64_t nseg,
                                  const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                  int elem) {
  for (int64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
    const int64_t a = src_off[s] * elem, b = dst_off[s] * elem, n = len[s] * elem;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[b + i] = src[a + i];
  }
}

// Stream-ordered device buffer, freed when it goes out of scope (move-only).
struct DevBuf {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), s(o.s) { o.p = nullptr; }
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

struct SubBatch {
  phmm_batch b{};
  std::vector<DevBuf> bufs;
  int64_t cells = 0;
};

static cudaError_t dev_alloc(std::vector<DevBuf> &bufs, size_t bytes, cudaStream_t s,
                             void **out) {
  bufs.emplace_back();
  bufs.back().s = s;
  cudaError_t e = cudaMallocAsync(&bufs.back().p, std::max<size_t>(bytes, 16), s);
  *out = bufs.back().p;
  return e;
}

// Compact copy of the pairs `sel` (reads and haplotypes renumbered, bases and qualities
// gathered on the device).
static cudaError_t make_sub(const phmm_batch &b, const std::vector<int64_t> &ro,
                            const std::vector<int64_t> &ho, const std::vector<int32_t> &pr,
                            const std::vector<int32_t> &ph, const std::vector<int64_t> &sel,
                            cudaStream_t s, SubBatch &out) {
  std::vector<int32_t> rmap(b.n_reads, -1), hmap(b.n_haps, -1), reads, haps;
  std::vector<int32_t> npr, nph;
  for (int64_t p : sel) {
    const int32_t r = pr[p], h = ph[p];
    if (rmap[r] < 0) {
      rmap[r] = (int32_t)reads.size();
      reads.push_back(r);
    }
    if (hmap[h] < 0) {
      hmap[h] = (int32_t)haps.size();
      haps.push_back(h);
    }
    npr.push_back(rmap[r]);
    nph.push_back(hmap[h]);
    out.cells += (ro[r + 1] - ro[r]) * (ho[h + 1] - ho[h]);
  }
  // segment lists: reads then haplotypes
  std::vector<int64_t> rso, rdo, rl, nro(reads.size() + 1, 0), hso, hdo, hl, nho(haps.size() + 1, 0);
  for (size_t i = 0; i < reads.size(); ++i) {
    rso.push_back(ro[reads[i]]);
    rl.push_back(ro[reads[i] + 1] - ro[reads[i]]);
    rdo.push_back(nro[i]);
    nro[i + 1] = nro[i] + rl.back();
  }
  for (size_t i = 0; i < haps.size(); ++i) {
    hso.push_back(ho[haps[i]]);
    hl.push_back(ho[haps[i] + 1] - ho[haps[i]]);
    hdo.push_back(nho[i]);
    nho[i + 1] = nho[i] + hl.back();
  }
  const int qe = b.qual_dtype == PHMM_QUAL_F32 ? 4 : 1;
  const int64_t sm = nro.back(), sn = nho.back();
  void *d_rb, *d_bq, *d_iq, *d_dq, *d_ro, *d_hb, *d_ho, *d_pr, *d_ph, *d_seg;
  cudaError_t e;
  auto &B = out.bufs;
  B.reserve(16);
  if ((e = dev_alloc(B, sm, s, &d_rb)) || (e = dev_alloc(B, sm * qe, s, &d_bq)) ||
      (e = dev_alloc(B, sm * qe, s, &d_iq)) || (e = dev_alloc(B, sm * qe, s, &d_dq)) ||
      (e = dev_alloc(B, 8 * nro.size(), s, &d_ro)) || (e = dev_alloc(B, sn, s, &d_hb)) ||
      (e = dev_alloc(B, 8 * nho.size(), s, &d_ho)) ||
      (e = dev_alloc(B, 4 * npr.size(), s, &d_pr)) ||
      (e = dev_alloc(B, 4 * nph.size(), s, &d_ph)))
    return e;
  const size_t nr = reads.size(), nh = haps.size();
  if ((e = dev_alloc(B, 8 * (3 * nr + 3 * nh), s, &d_seg))) return e;
  int64_t *seg = (int64_t *)d_seg;
  std::vector<int64_t> host_seg;
  host_seg.insert(host_seg.end(), rso.begin(), rso.end());
  host_seg.insert(host_seg.end(), rdo.begin(), rdo.end());
  host_seg.insert(host_seg.end(), rl.begin(), rl.end());
  host_seg.insert(host_seg.end(), hso.begin(), hso.end());
  host_seg.insert(host_seg.end(), hdo.begin(), hdo.end());
  host_seg.insert(host_seg.end(), hl.begin(), hl.end());
  // synchronous copies from pageable memory: the host vectors die with this function
  if ((e = cudaMemcpyAsync(seg, host_seg.data(), 8 * host_seg.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_ro, nro.data(), 8 * nro.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_ho, nho.data(), 8 * nho.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_pr, npr.data(), 4 * npr.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_ph, nph.data(), 4 * nph.size(), cudaMemcpyHostToDevice, s)))
    return e;
  const int grid = 1024;
  k_gather_segments<<<grid, 128, 0, s>>>(seg, seg + nr, seg + 2 * nr, (int64_t)nr,
                                         (const uint8_t *)b.read_bases, (uint8_t *)d_rb, 1);
  k_gather_segments<<<grid, 128, 0, s>>>(seg, seg + nr, seg + 2 * nr, (int64_t)nr,
                                         (const uint8_t *)b.base_q, (uint8_t *)d_bq, qe);
  k_gather_segments<<<grid, 128, 0, s>>>(seg, seg + nr, seg + 2 * nr, (int64_t)nr,
                                         (const uint8_t *)b.ins_q, (uint8_t *)d_iq, qe);
  k_gather_segments<<<grid, 128, 0, s>>>(seg, seg + nr, seg + 2 * nr, (int64_t)nr,
                                         (const uint8_t *)b.del_q, (uint8_t *)d_dq, qe);
  k_gather_segments<<<grid, 128, 0, s>>>(seg + 3 * nr, seg + 3 * nr + nh, seg + 3 * nr + 2 * nh,
                                         (int64_t)nh, (const uint8_t *)b.hap_bases,
                                         (uint8_t *)d_hb, 1);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  phmm_batch &o = out.b;
  o = b;
  o.n_reads = (int64_t)nr;
  o.n_haps = (int64_t)nh;
  o.n_pairs = (int64_t)npr.size();
  o.read_bases = (const uint8_t *)d_rb;
  o.base_q = d_bq;
  o.ins_q = d_iq;
  o.del_q = d_dq;
  o.read_off = (const int64_t *)d_ro;
  o.hap_bases = (const uint8_t *)d_hb;
  o.hap_off = (const int64_t *)d_ho;
  o.pair_read = (const int32_t *)d_pr;
  o.pair_hap = (const int32_t *)d_ph;
  return cudaSuccess;
}

// Time one candidate table on a sub-batch: forward (which == 1) or adjoint (which == 2).
// Returns milliseconds per call, or a negative value if the candidate could not run.
static float time_candidate(const SubBatch &sb, const phmm_options &opt, int which,
                            cudaStream_t s) {
  phmm_plan *plan = nullptr;
  if (phmm_plan_create(&sb.b, &opt, s, &plan) != PHMM_OK) return -1.f;
  std::vector<DevBuf> bufs;
  void *ws, *out, *flags, *dL = nullptr, *g = nullptr;
  const size_t wsb = phmm_workspace_bytes(plan);
  int64_t sm = 0, sn = 0, cells = 0;
  phmm_plan_info(plan, &sm, &sn, &cells);
  const int64_t P = sb.b.n_pairs;
  float ms = -1.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = !dev_alloc(bufs, wsb + 256, s, &ws) && !dev_alloc(bufs, 8 * P, s, &out) &&
            !dev_alloc(bufs, P, s, &flags) &&
            (which == 1 || (!dev_alloc(bufs, 8 * P, s, &dL) &&
                            !dev_alloc(bufs, 12 * sm + 64, s, &g))) &&
            !cudaEventCreate(&e0) && !cudaEventCreate(&e1);
  if (ok) {
    char *w = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    if (which == 2) {
      std::vector<double> ones(P, 1.0);
      ok = !cudaMemcpyAsync(dL, ones.data(), 8 * P, cudaMemcpyHostToDevice, s) &&
           !cudaStreamSynchronize(s);
    }
    float *gb = (float *)g, *gi = gb + sm, *gd = gi + sm;
    double *gg = (double *)(((uintptr_t)(gd + sm) + 7) & ~(uintptr_t)7);
    auto run = [&]() {
      if (which == 1) return phmm_forward(plan, w, wsb, (double *)out, (uint8_t *)flags, s);
      return phmm_backward(plan, w, wsb, (const double *)dL, gb, gi, gd, nullptr, gg, s);
    };
    ok = ok && phmm_forward(plan, w, wsb, (double *)out, (uint8_t *)flags, s) == PHMM_OK &&
         run() == PHMM_OK;  // warm-up (graph capture, caches)
    // one timed call sets the repetitions: at least ~10 ms of timed work per candidate
    int reps = 1;
    float ms1 = 0.f;
    ok = ok && !cudaEventRecord(e0, s) && run() == PHMM_OK && !cudaEventRecord(e1, s) &&
         !cudaEventSynchronize(e1) && !cudaEventElapsedTime(&ms1, e0, e1);
    if (ok) reps = std::max(2, std::min(50, (int)(10.f / std::max(ms1, 1e-3f)) + 1));
    ok = ok && !cudaEventRecord(e0, s);
    for (int i = 0; ok && i < reps; ++i) ok = run() == PHMM_OK;
    ok = ok && !cudaEventRecord(e1, s) && !cudaEventSynchronize(e1) &&
         !cudaEventElapsedTime(&ms, e0, e1);
    if (ok) ms /= reps;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  phmm_plan_destroy(plan);
  cudaGetLastError();
  return ok ? ms : -1.f;
}

}  // namespace

extern "C" int phmm_autotune(const phmm_batch *batch, phmm_options *opt, int which,
                             int64_t sample_pairs, void *stream) {
  const phmm::NvtxRange nvtx("phmm_autotune");
  if (!batch || !opt || which < 1 || which > 3 || sample_pairs < 1) return PHMM_EINVAL;
  cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const phmm_batch &b = *batch;
  {  // validate once (the candidates' plans validate their sub-batches again)
    phmm_plan *pl = nullptr;
    const int rc = phmm_plan_create(batch, opt, stream, &pl);
    if (rc != PHMM_OK) return rc;
    phmm_plan_destroy(pl);
  }
  // a batch with a per-base gap-continuation track runs a fixed group table: nothing to tune
  if (b.gcp_q) return PHMM_OK;
  if (b.n_pairs == 0) return PHMM_OK;
  std::vector<int64_t> ro(b.n_reads + 1), ho(b.n_haps + 1);
  std::vector<int32_t> pr(b.n_pairs), ph(b.n_pairs);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ro.data(), b.read_off, 8 * ro.size(), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(ho.data(), b.hap_off, 8 * ho.size(), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(pr.data(), b.pair_read, 4 * pr.size(), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(ph.data(), b.pair_hap, 4 * ph.size(), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return PHMM_ECUDA;
  constexpr int kRange = 16, kRanges = PHMM_MAX_READ_LEN / kRange;
  std::vector<std::vector<int64_t>> members(kRanges);
  for (int64_t p = 0; p < b.n_pairs; ++p) {
    const int64_t m = ro[pr[p] + 1] - ro[pr[p]];
    if (m <= PHMM_MAX_READ_LEN) members[(m - 1) / kRange].push_back(p);  // longer: row tiles
  }
  phmm_options work = *opt;  // ranges without pairs keep the caller's entries
  // A tuned choice replaces the built-in one only if it is at least this much faster: timings
  // of samples carry noise and some bias against the whole batch.
  constexpr float kMargin = 0.98f;
  for (int k = 0; k < kRanges; ++k) {
    const std::vector<int64_t> &mem = members[k];
    if (mem.empty()) continue;
    const int hi = kRange * (k + 1);
    for (int pass = 1; pass <= 2; ++pass) {
      if (!(which & pass)) continue;
      // the forward is cheap: it is timed on samples 8x larger
      const int64_t want = pass == 1 ? 8 * sample_pairs : sample_pairs;
      std::vector<int64_t> sel;
      const int64_t stride = std::max<int64_t>(1, (int64_t)mem.size() / want);
      for (size_t i = 0; i < mem.size() && (int64_t)sel.size() < want; i += stride)
        sel.push_back(mem[i]);
      SubBatch sb;
      if (make_sub(b, ro, ho, pr, ph, sel, s, sb) != cudaSuccess) return PHMM_ECUDA;
      const int builtin = pass == 1 ? default_cfg_of_m(hi) : bwd_default_cfg(hi);
      int best = -1;
      float best_ms = 0.f, builtin_ms = -1.f;
      for (int cfg = 0; cfg < kNumCfg32; ++cfg) {
        const int cap = cfg_lanes(cfg) * cfg_rows(cfg);
        if (cap < hi || cap > std::max(2 * hi, 64)) continue;
        if (pass == 1 && !fwd_cfg_supported(cfg)) continue;
        if (pass == 2 && !bwd_cfg_supported(cfg)) continue;
        phmm_options o = *opt;
        o.binning = 1;
        int32_t *tab = pass == 1 ? o.bin_rows : o.bwd_rows;
        for (int i = 0; i <= PHMM_MAX_READ_LEN / 4; ++i) tab[i] = cfg;
        if (pass == 1) o.bin_table_valid = 1; else o.bwd_table_valid = 1;
        const float ms = time_candidate(sb, o, pass, s);
        if (cfg == builtin) builtin_ms = ms;
        if (ms > 0.f && (best < 0 || ms < best_ms)) {
          best = cfg;
          best_ms = ms;
        }
      }
      if (best < 0) continue;  // no candidate ran: keep the built-in entries
      // not clearly faster than the built-in group: keep the built-in (per 4-row bucket) entries
      if (builtin_ms > 0.f && best_ms > kMargin * builtin_ms) continue;
      int32_t *tab = pass == 1 ? work.bin_rows : work.bwd_rows;
      const int32_t *valid = pass == 1 ? &work.bin_table_valid : &work.bwd_table_valid;
      if (!*valid) {  // first tuned range: fill the table with "no entry" (default)
        for (int i = 0; i <= PHMM_MAX_READ_LEN / 4; ++i) tab[i] = -1;
        if (pass == 1) work.bin_table_valid = 1; else work.bwd_table_valid = 1;
      }
      for (int bk = 4 * k + 1; bk <= 4 * k + 4; ++bk) tab[bk] = best;
    }
  }
  // Warps per block (pairs per block = warps x pairs per warp; the kernels take up to 4
  // warps per block) for the tuned tables, forward and adjoint separately: timed on a strided
  // sample of the whole batch.
  {
    std::vector<int64_t> sel;
    const int64_t want = std::min<int64_t>(b.n_pairs, 4 * sample_pairs);
    const int64_t stride = std::max<int64_t>(1, b.n_pairs / want);
    for (int64_t p = 0; p < b.n_pairs && (int64_t)sel.size() < want; p += stride)
      if (ro[pr[p] + 1] - ro[pr[p]] <= PHMM_MAX_READ_LEN) sel.push_back(p);
    if (!sel.empty()) {
      SubBatch sb;
      if (make_sub(b, ro, ho, pr, ph, sel, s, sb) != cudaSuccess) return PHMM_ECUDA;
      for (int pass = 1; pass <= 2; ++pass) {
        if (!(which & pass)) continue;
        int32_t &field = pass == 1 ? work.warps_per_block : work.bwd_warps_per_block;
        const int current = field > 0 ? field : (pass == 2 && work.warps_per_block > 0
                                                     ? work.warps_per_block : 4);
        int best = current;
        float best_ms = 0.f, current_ms = -1.f;
        for (int wpb : {1, 2, 4}) {
          phmm_options o = work;
          (pass == 1 ? o.warps_per_block : o.bwd_warps_per_block) = wpb;
          const float ms = time_candidate(sb, o, pass, s);
          if (wpb == current) current_ms = ms;
          if (ms > 0.f && (best_ms == 0.f || ms < best_ms)) {
            best = wpb;
            best_ms = ms;
          }
        }
        if (current_ms > 0.f && best_ms > kMargin * current_ms) best = current;
        field = best;
      }
    }
  }
  *opt = work;
  return PHMM_OK;
}
