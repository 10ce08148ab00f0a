// Adjoint (reverse sweep) of the Pair-HMM forward pass: d log10 L / d(Phred inputs).
//
// Not in the paper (which scores only): the gradient of log10 L with respect to the per-base
// base, insertion and deletion qualities and the gap-continuation penalty, for fitting error
// models.  With adjoints A^ = (dL/dA) / L, the reverse recurrences of Eq. 1-3 are
//   M^(i,j) = a'_{i+1} u(i+1,j+1) + delta_{i+1} I^(i+1,j) + zeta_i D^(i,j+1)   [+1/L, i = m]
//   I^(i,j) = u(i+1,j+1) + eps I^(i+1,j)                                       [+1/L, i = m]
//   D^(i,j) = u(i+1,j+1) + eps D^(i,j+1),        u(i,j) = beta lambda(i,j) M^(i,j)
// and each parameter's partial is a sum over cells of an adjoint times a forward value.
// Written so that every product pairs forward values of one column j with adjoints already
// at hand when the reverse sweep reaches column j (u and D^ of column j+1, I^ of column j):
//   alpha_{i+1}: sum_j u(i+1,j+1) M(i,j) / beta      beta: sum u(i+1,j+1) (I+D)(i,j) / beta
//   delta_{i+1}: sum_j I^(i+1,j) M(i,j)              zeta_i: sum_j D^(i,j+1) M(i,j)
//   eps: sum I^(i+1,j) I(i,j) + D^(i,j+1) D(i,j)     (minus the beta term: beta = 1 - eps)
//   Q_i: -A1/(1-Q_i) + A2/Q_i with A1, A2 = sum over match / mismatch columns of
//        M^(i,j) M(i,j)  (lambda = 1-Q on a match, Q/3 on a mismatch),
// followed by the chain rule through alpha = 1-(delta+zeta) (or 1-10^(-(iq+dq)/10)) and
// P = 10^(-q/10).
//
// GPU design.  The same lane/row decomposition as the forward wavefront, reversed: lane t
// owns K rows, walks the columns from right to left, and exchanges the top row's u and I^
// with the lane above by __shfl_down_sync.  Forward values are recomputed, not stored:
//   phase A  runs the per-lane-exponent FP32 forward and checkpoints every lane's register
//            state at each renormalisation point (every step of the ramp, then every
//            segment of 2..8 steps) into a per-warp scratch slot (streaming stores);
//   phase B  for each segment, last to first: restores the checkpoint, recomputes the
//            segment while recording the lane's rows after each step in the warp's shared
//            memory (M and D/zeta per row and the top row's I; the reverse step rebuilds
//            the other rows' I with Eq. 2), then runs the adjoint over the segment in
//            reverse.  Step records never leave the SM: written to global memory they
//            would move ~2.5 words per cell each way through the SM's L2 port, which
//            bounds the recompute well below the forward's arithmetic rate.
// Adjoints carry their own per-lane power-of-two exponent and the inverse of the forward's
// per-row bias, so a forward x adjoint product is a posterior-scale number times
// 2^-(E_fwd + E_adj).  The partial sums are held at the lane's current scale and re-based
// (by an exact power of two) when E_fwd + E_adj changes: no per-cell scaling.  Per-pair
// partials are written in FP32 and reduced per read in FP64 (grad_reduce.cu).
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <vector>
#include "bwd_kernel.cuh"

struct phmm_plan;

namespace phmm {

const phmm_batch &plan_batch(const phmm_plan *pl);
const phmm_options &plan_options(const phmm_plan *pl);
size_t plan_bwd_offset(const phmm_plan *pl);
int64_t plan_sum_m(const phmm_plan *pl);
int plan_sms(const phmm_plan *pl);
size_t plan_layout_rp(const phmm_plan *pl);
size_t plan_layout_rcode(const phmm_plan *pl);
size_t plan_layout_hcode(const phmm_plan *pl);
size_t plan_layout_bin(const phmm_plan *pl, int which);
double plan_eps64(const phmm_plan *pl);
int64_t plan_n_max(const phmm_plan *pl);
int64_t plan_pair_rows(const phmm_plan *pl);
int plan_max_m(const phmm_plan *pl);
unsigned *plan_dbg_word(const phmm_plan *pl);
int64_t plan_hcode_bytes(const phmm_plan *pl);
bool plan_gq(const phmm_plan *pl);
size_t plan_layout_rgap(const phmm_plan *pl);
const int *plan_bwd_cfg_of_m(const phmm_plan *pl);
const std::vector<int> &plan_bwd_used(const phmm_plan *pl);

int launch_binning(const phmm_batch &b, const CfgTable &tab, int32_t *key, int32_t *counts,
                   int32_t *offsets, int32_t *cursor, int32_t *grp_begin, int32_t *grp_count,
                   int32_t *order, cudaStream_t s, int *launches);
int pair_offsets(const phmm_batch &b, char *scratch, int64_t **poff, cudaStream_t s);
int reduce_gradients(const phmm_batch &b, char *scratch, const float *part_bq,
                     const float *part_iq, const float *part_dq, const float *part_gq,
                     const double *pair_dgcp, const double *dL, float *dbq, float *diq,
                     float *ddq, float *dgq, double *dgcp, cudaStream_t s, int *launches);
size_t reduce_scratch_bytes_aligned(int64_t P, int64_t R);

// ------------------------------------------------------------------------ host side ------

static BwdKernel bwd_kernel32(int L, int K, bool gq = false) {
  if (gq) return bwd32_gq(L, K);
  if (K % 2 == 1) return L <= 8 ? bwd32_odd_lo(L, K) : bwd32_odd_hi(L, K);
  switch (L) {
    case 4:
    case 8: return bwd32_lo(L, K);
    case 16: return bwd32_mid(L, K);
    case 32: return bwd32_hi(L, K);
    default: return nullptr;
  }
}
static BwdKernel bwd_kernel64(int K, bool gq = false) {
  return gq ? bwd64_gq(K) : bwd64_table(K);
}

// 1 if the FP32 adjoint is built for group `cfg`.
int bwd_cfg_supported(int cfg) {
  return cfg >= 0 && cfg < kNumCfg32 && bwd_kernel32(cfg_lanes(cfg), cfg_rows(cfg)) != nullptr;
}

static size_t bwd_smem(int K, int elem, int block, bool gq) {
  return (size_t)(block / 32) * bwd_warp_bytes(K, elem, gq);
}

// Threads per block of an adjoint launch: warps_per_block warps, fewer where the group's
// launch bounds allow fewer or their shared memory would exceed the per-block limit.
static int bwd_block(int K, int elem, int warps_per_block, bool gq) {
  const int fit = (int)((size_t)227 * 1024 / bwd_warp_bytes(K, elem, gq));
  return 32 * std::max(1, std::min({warps_per_block, bwd_max_wpb(K, elem, gq), fit}));
}

// Read length -> FP32 backward group (rows per lane <= 12 keeps the adjoint in registers).
int bwd_default_cfg(int m) {
  struct Gp { int cap, L, K; };
  static const Gp order[] = {{16, 4, 4},   {32, 4, 8},    {48, 4, 12},  {64, 8, 8},
                             {96, 8, 12},  {128, 16, 8},  {192, 16, 12}, {256, 32, 8},
                             {384, 32, 12}, {512, 32, 16}};
  for (const Gp &g : order)
    if (m <= g.cap) return cfg_index(g.L, g.K);
  return cfg_index(32, 16);
}

static int blocks_per_sm(BwdKernel k, size_t smem, int block) {
  if (!k) return 0;
  cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem);
  return nb < 1 ? 1 : nb;
}

// Checkpoints per pair group: one per ramp step, then one per segment.
static int64_t bwd_nchk(int L, int K, int elem, int64_t n_max, bool gq) {
  const int seg = bwd_seg_len(K, elem, gq);
  const int64_t steps = n_max + L - 1 + seg;
  const int64_t ramp = (L + 15) & ~15;
  return ramp + (steps + seg - 1) / seg + 2;
}

// Row tiles a slot of group (L, K) holds for a plan whose longest read is max_m: reads longer
// than one group are swept in tiles of 512 rows by the 32 x 16 group only.
static int ntile_cap(int L, int K, int max_m) {
  if (L != 32 || K != 16 || max_m <= 32 * 16) return 1;
  return (max_m + 32 * 16 - 1) / (32 * 16);
}

// A slot (elements of the kernel's type): the checkpoints of every row tile, then for tiled
// plans the last row of every tile but the last and two buffers of a tile's first-row
// adjoints, each n_max columns of 4 values.
static int64_t slot_elems(int L, int K, int elem, int64_t n_max, int ntile, bool gq) {
  int64_t e = (int64_t)ntile * bwd_nchk(L, K, elem, n_max, gq) * 32 * ck_w(K, elem);
  if (ntile > 1) e += (int64_t)(ntile - 1 + 2) * n_max * 4;
  return e;
}

struct BwdLayout {
  size_t part, pdgcp, red, slots, slots_bytes, total;
  std::vector<size_t> guards;  // debug builds: a guard region after every region
};

#ifdef PHMM_DEBUG
constexpr bool kDebugB = true;
#else
constexpr bool kDebugB = false;
#endif

static BwdLayout bwd_layout(const phmm_plan *pl) {
  const phmm_batch &b = plan_batch(pl);
  const int wpb = plan_options(pl).bwd_warps_per_block;
  BwdLayout Lo;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 255) & ~(size_t)255;
    if (kDebugB) {
      Lo.guards.push_back(o);
      o += 256;
    }
    return at;
  };
  const int64_t rows = plan_pair_rows(pl) + 1;
  Lo.part = take((plan_gq(pl) ? 4 : 3) * 4 * (size_t)rows);
  Lo.pdgcp = take(8 * (size_t)(b.n_pairs + 1));
  Lo.red = take(reduce_scratch_bytes_aligned(b.n_pairs, b.n_reads));
  size_t slots = 0;
  const int64_t nmax = plan_n_max(pl);
  const bool gq = plan_gq(pl);
  for (int cfg : plan_bwd_used(pl)) {
    const int L = cfg_lanes(cfg), K = cfg_rows(cfg);
    const int block = bwd_block(K, 4, wpb, gq);
    const size_t nslot = (size_t)plan_sms(pl) *
                         blocks_per_sm(bwd_kernel32(L, K, gq), bwd_smem(K, 4, block, gq),
                                       block) *
                         (block / 32);
    slots = std::max(slots, nslot * 4 * (size_t)slot_elems(L, K, 4, nmax,
                                                             ntile_cap(L, K, plan_max_m(pl)), gq));
  }
  for (int c = 0; c < kNumCfg64; ++c) {
    const int K = rows64(c);
    const int block = bwd_block(K, 8, wpb, gq);
    const size_t nslot = (size_t)plan_sms(pl) *
                         blocks_per_sm(bwd_kernel64(K, gq), bwd_smem(K, 8, block, gq),
                                       block) *
                         (block / 32);
    slots = std::max(slots, nslot * 8 * (size_t)slot_elems(32, K, 8, nmax,
                                                             ntile_cap(32, K, plan_max_m(pl)), gq));
  }
  Lo.slots = take(slots);
  Lo.slots_bytes = slots;
  Lo.total = o;
  return Lo;
}

size_t bwd_workspace_bytes(const phmm_plan *pl) { return bwd_layout(pl).total; }
std::vector<size_t> bwd_guard_offsets(const phmm_plan *pl) { return bwd_layout(pl).guards; }

#define CKB(x)                          \
  do {                                  \
    int rc_ = (int)(x);                 \
    if (rc_) return rc_;                \
  } while (0)

// The adjoint sweep over every pair: per-pair partials (times dL[p], or of log10 L itself
// when dL is null) into the workspace, and with `out` non-null log10 L and flags from the
// sweep's own forward pass.  Returns a cudaError_t value (0 on success).
// ev2: events recorded before and after the adjoint kernels.
int bwd_sweep_impl(phmm_plan *pl, char *ws, const double *dL, double *out, uint8_t *oflags,
                   cudaStream_t s, int *launches, cudaEvent_t *ev2) {
  const phmm_batch &b = plan_batch(pl);
  const phmm_options &o = plan_options(pl);
  const BwdLayout Lo = bwd_layout(pl);
  char *bw = ws + plan_bwd_offset(pl);
  float *part = (float *)(bw + Lo.part);
  const int64_t rows = plan_pair_rows(pl) + 1;
  float *part_bq = part, *part_iq = part + rows, *part_dq = part + 2 * rows;
  float *part_gq = plan_gq(pl) ? part + 3 * rows : nullptr;
  double *pdg = (double *)(bw + Lo.pdgcp);
  char *red = bw + Lo.red;
  int64_t *poff = nullptr;
  CKB(pair_offsets(b, red, &poff, s));
  *launches += 2;
  if (b.n_pairs > 0) {
    // bin pairs by backward group, reusing the forward's sort buffers; zero the counters
    int32_t *counts = (int32_t *)(ws + plan_layout_bin(pl, 0));
    CKB(cudaMemsetAsync(counts, 0, plan_layout_bin(pl, 9), s));
    CfgTable tab;
    const int *cm = plan_bwd_cfg_of_m(pl);
    for (int m = 0; m <= PHMM_MAX_READ_LEN; ++m) tab.cfg[m] = (int8_t)cm[m];
    int32_t *grp_begin = (int32_t *)(ws + plan_layout_bin(pl, 4));
    int32_t *grp_count = (int32_t *)(ws + plan_layout_bin(pl, 5));
    int32_t *order = (int32_t *)(ws + plan_layout_bin(pl, 6));
    CKB(launch_binning(b, tab, (int32_t *)(ws + plan_layout_bin(pl, 1)), counts,
                       (int32_t *)(ws + plan_layout_bin(pl, 2)),
                       (int32_t *)(ws + plan_layout_bin(pl, 3)), grp_begin, grp_count, order, s,
                       launches));
    BwdArgs a;
    std::memset(&a, 0, sizeof(a));
    FwdArgs &f = a.f;
    f.pair_read = b.pair_read;
    f.pair_hap = b.pair_hap;
    f.read_off = b.read_off;
    f.hap_off = b.hap_off;
    f.rp = (const RowParams *)(ws + plan_layout_rp(pl));
    f.rcode = (const uint8_t *)(ws + plan_layout_rcode(pl));
    f.hcode = (const uint8_t *)(ws + plan_layout_hcode(pl));
    f.bq = b.base_q;
    f.iq = b.ins_q;
    f.dq = b.del_q;
    f.gq = b.gcp_q;
    f.rgap = plan_gq(pl) ? (const float2 *)(ws + plan_layout_rgap(pl)) : nullptr;
    f.qual_f32 = b.qual_dtype == PHMM_QUAL_F32;
    f.alpha_mode = b.alpha_mode;
    f.n_reads = b.n_reads;
    f.n_haps = b.n_haps;
    const double eps64 = plan_eps64(pl);
    f.eps32 = (float)eps64;
    f.beta32 = (float)(1.0 - eps64);
    f.eps64 = eps64;
    f.beta64 = 1.0 - eps64;
    f.persistent = 1;
    f.dbg_err = plan_dbg_word(pl);  // debug builds only (else null: no checks)
    f.dbg_sum_m = plan_sum_m(pl);
    f.dbg_hcode_bytes = plan_hcode_bytes(pl);
    a.dL = dL;
    a.out = out;
    a.oflags = oflags;
    a.poff = poff;
    a.part_bq = part_bq;
    a.part_iq = part_iq;
    a.part_dq = part_dq;
    a.part_gq = part_gq;
    a.pair_dgcp = pdg;
    a.scratch = bw + Lo.slots;
    int32_t *rlist = (int32_t *)(ws + plan_layout_bin(pl, 8));
    int32_t *rcnt = counts + (size_t)kNumCfg32 * kNBuckets + kNumCfg32;  // in the zeroed region
    int32_t *rctr = rcnt + kNumCfg64;
    for (int k = 0; k < kNumCfg64; ++k)
      a.resc_list[k] = rlist + (size_t)k * std::max<int64_t>(b.n_pairs, 1);
    a.resc_count = rcnt;
    a.why = (int32_t *)(ws + plan_layout_bin(pl, 10));
    CKB(cudaMemsetAsync(a.why, 0, 16, s));
    const int64_t nmax = plan_n_max(pl);
    CKB(cudaEventRecord(ev2[0], s));
    for (int cfg : plan_bwd_used(pl)) {
      const int L = cfg_lanes(cfg), K = cfg_rows(cfg);
      BwdArgs c = a;
      c.f.list = order;
      c.f.offset_dev = grp_begin + cfg;
      c.f.count_dev = grp_count + cfg;
      c.f.counter = (int32_t *)(ws + plan_layout_bin(pl, 7)) + cfg;
      c.nchk = (int32_t)bwd_nchk(L, K, 4, nmax, plan_gq(pl));
      c.ntile_cap = ntile_cap(L, K, plan_max_m(pl));
      c.ck_tile = (int64_t)c.nchk * 32 * ck_w(K, 4);
      c.tile_cols = nmax;
      c.slot_elems = slot_elems(L, K, 4, nmax, c.ntile_cap, plan_gq(pl));
      c.rescue = o.adjoint_rescue ? 0 : 1;  // without the FP64 pass, failures write NaN
      c.all64 = o.adjoint_rescue == 2 ? 1 : 0;
      BwdKernel k = bwd_kernel32(L, K, plan_gq(pl));
      if (!k) return (int)cudaErrorInvalidValue;
      const int block = bwd_block(K, 4, o.bwd_warps_per_block, plan_gq(pl));
      const size_t sm = bwd_smem(K, 4, block, plan_gq(pl));
      const int grid = plan_sms(pl) * blocks_per_sm(k, sm, block);
      c.f.dbg_nslots = (int64_t)(Lo.slots_bytes / (4 * (size_t)c.slot_elems));
      k<<<grid, block, sm, s>>>(c);
      CKB(cudaGetLastError());
      ++*launches;
    }
    // FP64 pass over the pairs whose FP32 adjoint ran out of range
    for (int k64 = 0; k64 < kNumCfg64; ++k64) {
      const int K = rows64(k64);
      BwdArgs c = a;
      c.f.list = a.resc_list[k64];
      c.f.offset_dev = nullptr;
      c.f.count_dev = rcnt + k64;
      c.f.counter = rctr + k64;
      c.nchk = (int32_t)bwd_nchk(32, K, 8, nmax, plan_gq(pl));
      c.ntile_cap = ntile_cap(32, K, plan_max_m(pl));
      c.ck_tile = (int64_t)c.nchk * 32 * ck_w(K, 8);
      c.tile_cols = nmax;
      c.slot_elems = slot_elems(32, K, 8, nmax, c.ntile_cap, plan_gq(pl));
      c.rescue = 1;
      BwdKernel kk = bwd_kernel64(K, plan_gq(pl));
      const int block = bwd_block(K, 8, o.bwd_warps_per_block, plan_gq(pl));
      const size_t sm = bwd_smem(K, 8, block, plan_gq(pl));
      const int grid = plan_sms(pl) * blocks_per_sm(kk, sm, block);
      c.f.dbg_nslots = (int64_t)(Lo.slots_bytes / (8 * (size_t)c.slot_elems));
      kk<<<grid, block, sm, s>>>(c);
      CKB(cudaGetLastError());
      ++*launches;
    }
  } else {
    CKB(cudaEventRecord(ev2[0], s));
  }
  CKB(cudaEventRecord(ev2[1], s));
  return 0;
}

// The per-read FP64 reduction of the partials the latest sweep left in the workspace, each
// pair's weighted by dL[p] when given.  ev1: event recorded after it.
int bwd_reduce_impl(phmm_plan *pl, char *ws, const double *dL, float *dbq, float *diq,
                    float *ddq, float *dgq, double *dgcp, cudaStream_t s, int *launches,
                    cudaEvent_t ev1) {
  const phmm_batch &b = plan_batch(pl);
  const BwdLayout Lo = bwd_layout(pl);
  char *bw = ws + plan_bwd_offset(pl);
  float *part = (float *)(bw + Lo.part);
  const int64_t rows = plan_pair_rows(pl) + 1;
  const bool gq = plan_gq(pl) && dgq;
  CKB(reduce_gradients(b, bw + Lo.red, part, part + rows, part + 2 * rows,
                       gq ? part + 3 * rows : nullptr, (const double *)(bw + Lo.pdgcp), dL, dbq,
                       diq, ddq, gq ? dgq : nullptr, dgcp, s, launches));
  CKB(cudaEventRecord(ev1, s));
  return 0;
}

// The whole backward: sweep with the partials scaled by dL, then the reduction.
// ev3: events recorded before the adjoint kernels, after them, and after the reduction.
int bwd_enqueue_impl(phmm_plan *pl, char *ws, const double *dL, float *dbq, float *diq,
                     float *ddq, float *dgq, double *dgcp, cudaStream_t s, int *launches,
                     cudaEvent_t *ev3) {
  CKB(bwd_sweep_impl(pl, ws, dL, nullptr, nullptr, s, launches, ev3));
  return bwd_reduce_impl(pl, ws, nullptr, dbq, diq, ddq, dgq, dgcp, s, launches, ev3[2]);
}

}  // namespace phmm
