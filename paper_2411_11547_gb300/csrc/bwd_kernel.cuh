// Adjoint wavefront kernel (the reverse sweep of the Pair-HMM forward pass); the host side
// and the method are described in bwd.cu.  Explicit instantiations live in bwd32_*.cu and
// bwd64.cu so the build compiles them in parallel.
#pragma once
#include <cstdint>
#include <type_traits>
#include "phmm_internal.cuh"
#include "wavefront.cuh"

namespace phmm {

struct BwdArgs {
  FwdArgs f;               // pair list, inputs and prepared parameters (as the forward)
  const double *dL;        // d(loss)/d(log10 L_p); null: partials of log10 L_p itself
  double *out;             // non-null: also write log10 L_p and its flags from the sweep's
  uint8_t *oflags;         //   own forward pass (the fused forward-with-partials call)
  const int64_t *poff;     // partial-gradient offsets per pair
  float *part_bq, *part_iq, *part_dq;
  float *part_gq;          // per-base gap-continuation partials (plans with a track)
  double *pair_dgcp;
  void *scratch;           // per-warp slots (elements of the kernel's type)
  int64_t slot_elems;
  int32_t nchk;            // checkpoint capacity per slot and row tile
  int64_t ck_tile;         // elements of one row tile's checkpoints in a slot (nchk x 32 x width)
  int32_t ntile_cap;       // row tiles a slot holds (reads longer than one group: 32 x 16 only)
  int64_t tile_cols;       // columns of the row-tile buffers (the longest haplotype)
  int32_t rescue;          // 1: this is the FP64 pass (write NaN on failure)
  int32_t all64;           // FP32 pass: hand every valid pair to the FP64 pass untouched
  int32_t *resc_list[kNumCfg64];  // FP32 pass: pairs handed to the FP64 pass
  int32_t *resc_count;
  int32_t *why;                   // [2]: hand-offs for the scale range / non-finite partials
};

// Widths (elements, multiples of the 16-byte vector) of a checkpoint (K rows of M and D/zeta,
// the top row's I, the boundary values, the conversion factor and the exponent) and of a step
// record (K rows of M and D/zeta; the step's top-row I goes to a side array of one element
// per lane).  Both leave the other rows' I out: Eq. 2 gives them again from M and the top
// row's I.  Both start with the same values in the same order, so the lane's registers feed
// either store alike.
__host__ __device__ constexpr int vecw(int elem) { return 16 / elem; }
__host__ __device__ constexpr int ck_w(int K, int elem) {
  return (2 * K + 5 + vecw(elem) - 1) / vecw(elem) * vecw(elem);
}
__host__ __device__ constexpr int rec_w(int K, int elem) {
  return (2 * K + vecw(elem) - 1) / vecw(elem) * vecw(elem);
}
template <typename T>
__host__ __device__ constexpr int ck_width(int K) { return ck_w(K, (int)sizeof(T)); }
template <typename T>
__host__ __device__ constexpr int rec_width(int K) { return rec_w(K, (int)sizeof(T)); }

// Shared memory of one warp: the emission table (kCodes planes of 32 lanes x LS, as
// TableGeom) and the step records of one segment (every step, the last one included, so the
// reverse reads every step's forward values from shared memory and the forward state is dead
// while it runs), then the steps' top-row I.  The segment length follows from what fits next
// to the table at the occupancy the registers allow (warps per SM): 2 to 8 steps.
// gq: the kernels of batches with a per-base gap-continuation track (more registers per row;
// they share the scalar kernels' geometry).  More warps per SM for the 8- and 10-row groups
// (10 and 9, at shorter segments) measured 1-5% slower on the 2^22-pair batch.
__host__ __device__ constexpr int bwd_warps_per_sm(int K, int elem, bool gq = false) {
  return (void)gq, elem == 8 ? 4 : (K <= 4 ? 16 : (K <= 6 ? 12 : 8));
}
// Most warps per block of a group's launch: the largest divisor (up to 4) of its warps per SM,
// so that whole blocks fill the SM.
__host__ __device__ constexpr int bwd_max_wpb(int K, int elem, bool gq = false) {
  return bwd_warps_per_sm(K, elem, gq) % 4 == 0   ? 4
         : bwd_warps_per_sm(K, elem, gq) % 3 == 0 ? 3
         : bwd_warps_per_sm(K, elem, gq) % 2 == 0 ? 2
                                                  : 1;
}
__host__ __device__ constexpr size_t bwd_table_bytes(int K, int elem) {
  return (size_t)kCodes * 32 * elem *
         (((K + vecw(elem) - 1) / vecw(elem)) % 2 == 1
              ? (K + vecw(elem) - 1) / vecw(elem) * vecw(elem)
              : (K + vecw(elem) - 1) / vecw(elem) * vecw(elem) + vecw(elem));
}
// Shared memory of one step: its record and its top-row I.
__host__ __device__ constexpr size_t bwd_rec_bytes(int K, int elem) {
  return (size_t)32 * (rec_w(K, elem) + 1) * elem;
}
// Steps whose records fit next to the table.
__host__ __device__ constexpr int bwd_rec_fit(int K, int elem, bool gq = false) {
  return (int)(((size_t)227 * 1024 / bwd_warps_per_sm(K, elem, gq) - 256 -
                 bwd_table_bytes(K, elem)) /
                bwd_rec_bytes(K, elem));
}
__host__ __device__ constexpr int bwd_seg_len(int K, int elem, bool gq = false) {
  return bwd_rec_fit(K, elem, gq) > 8   ? 8
         : bwd_rec_fit(K, elem, gq) < 2 ? 2
                                        : bwd_rec_fit(K, elem, gq);
}
__host__ __device__ constexpr size_t bwd_warp_bytes(int K, int elem, bool gq = false) {
  return bwd_table_bytes(K, elem) + (size_t)bwd_seg_len(K, elem, gq) * bwd_rec_bytes(K, elem);
}

// Records are stored as [record][16-byte group][lane], so one warp-wide 128-bit access
// covers 512 contiguous bytes.  STREAM: checkpoints, written once and read once much later,
// bypass the caches' keep-alive (evict-first) so the short-lived step records stay in L2.
template <typename T, int W, bool STREAM = false>
__device__ __forceinline__ void rec_store(T *base, int lane, const T (&v)[W]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int g = 0; g < W / 4; ++g) {
      const float4 x = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
      if constexpr (STREAM) __stcs(reinterpret_cast<float4 *>(base) + g * 32 + lane, x);
      else reinterpret_cast<float4 *>(base)[g * 32 + lane] = x;
    }
  } else {
#pragma unroll
    for (int g = 0; g < W / 2; ++g) {
      const double2 x = make_double2(v[2 * g], v[2 * g + 1]);
      if constexpr (STREAM) __stcs(reinterpret_cast<double2 *>(base) + g * 32 + lane, x);
      else reinterpret_cast<double2 *>(base)[g * 32 + lane] = x;
    }
  }
}
template <typename T, int W, bool STREAM = false>
__device__ __forceinline__ void rec_load(const T *base, int lane, T (&v)[W]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int g = 0; g < W / 4; ++g) {
      const float4 x = STREAM ? __ldcs(reinterpret_cast<const float4 *>(base) + g * 32 + lane)
                              : reinterpret_cast<const float4 *>(base)[g * 32 + lane];
      v[4 * g] = x.x;
      v[4 * g + 1] = x.y;
      v[4 * g + 2] = x.z;
      v[4 * g + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int g = 0; g < W / 2; ++g) {
      const double2 x = STREAM ? __ldcs(reinterpret_cast<const double2 *>(base) + g * 32 + lane)
                               : reinterpret_cast<const double2 *>(base)[g * 32 + lane];
      v[2 * g] = x.x;
      v[2 * g + 1] = x.y;
    }
  }
}

// Ask the copy engine to bring `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// A lane's share of a record ([16-byte group][lane] layout, W elements) copied from global to
// shared memory asynchronously (16 bytes per copy, bypassing L1); cp_async_wait waits for
// every copy the thread has issued.
template <typename T, int W>
__device__ __forceinline__ void rec_copy_async(T *dst, const T *src, int lane) {
  constexpr int V = 16 / (int)sizeof(T);
#pragma unroll
  for (int g = 0; g < W / V; ++g) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + (size_t)(g * 32 + lane) * V);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d),
                 "l"(src + (size_t)(g * 32 + lane) * V)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Small integers (exponents, base codes) ride in the records as exact floating values.
template <typename T>
__device__ __forceinline__ T int_bits(int e) {
  return (T)e;
}
template <typename T>
__device__ __forceinline__ int bits_int(T x) {
  return (int)x;
}

// Adjoint state of one lane.
template <typename T, int K>
struct AdjState {
  T u[K];      // u(i, j+1) = beta lambda M^ of the lane's rows at the column to the right,
               // with the sign of the signed emission (+ match, - mismatch)
  T Db[K];     // D^(i, j+1)
  T Itop;      // I^ of the lane's top row at its current column (read by the lane above)
  T diagU;     // u of the lower lane's top row one column to the right (own scale, signed)
  T fB;        // 2^(E_low - E_own) and the row bias, for values from the lane below
  T seed;      // 1/L in the stored scale of the last row (last lane only)
  int EB;      // per-lane exponent of the adjoints
  bool nz;     // the lane held a nonzero adjoint at the latest renormalisation
};

// Renormalise the adjoints of a lane by a power of two; a lane that holds only zeros takes
// the exponent that makes the next values from the lane below arrive near 1.
// `apply` selects the lanes that renormalise now (the exchange runs on every lane).
// keep: the lane prefers the exponent Ek (which keeps its posterior scale, and so the scale
// of its partial sums, unchanged) whenever that leaves its largest adjoint within 2^+-24;
// otherwise it normalises the largest to [1, 2).
// ovr: the last lane of a row tile above another takes the lane below's exponent and size
// from (Eo, xo), the tile below's first-row adjoints about to arrive, for its adoption.
// rS: 1/S with L = S 2^(ES - kBias (K-1)), for the lane that seeds row m (else 0).
template <typename T, int L, int K, int kBias>
__device__ __forceinline__ void adj_rescale(AdjState<T, K> &as, int t, T rS, int ES,
                                            bool apply = true, bool keep = false, int Ek = 0,
                                            bool ovr = false, int Eo = 0, T xo = 0) {
  constexpr unsigned FULL = 0xffffffffu;
  T mx = fmax(as.Itop, fabs(as.diagU));
#pragma unroll
  for (int r = 0; r < K; ++r) mx = fmax(mx, fmax(fabs(as.u[r]), as.Db[r]));
  const bool zero = !(mx > (T)0);
  if (apply) as.nz = !zero;
  if (apply && !zero) {
    int En = as.EB + Num<T>::ilog2(mx);
    if (keep && Ek - En <= 24 && En - Ek <= 24) En = Ek;
    const T sc = Num<T>::exp2i(as.EB - En);
#pragma unroll
    for (int r = 0; r < K; ++r) {
      as.u[r] *= sc;
      as.Db[r] *= sc;
    }
    as.Itop *= sc;
    as.diagU *= sc;
    as.EB = En;
  }
  const T xb = fmax(fabs(as.u[0]), as.Itop);
  int Elow = __shfl_down_sync(FULL, as.EB, 1, L);
  T xbl = __shfl_down_sync(FULL, xb, 1, L);
  const bool last_ovr = ovr && t == L - 1;
  if (last_ovr) {
    Elow = Eo;
    xbl = xo;
  }
  if (apply && zero && (t < L - 1 || last_ovr))
    as.EB = Elow - kBias * (K - 1) + (xbl > (T)0 ? Num<T>::ilog2(xbl) : 0);
  as.fB = t < L - 1 ? Num<T>::exp2i(Elow - as.EB - kBias * (K - 1)) : (T)0;
  as.seed = (t == L - 1 && rS > (T)0) ? Num<T>::exp2i(-ES - as.EB) * rS : (T)0;
}

// Register cap per thread for the group's warps per SM (the per-row registers: forward
// state, adjoints, coefficients, four partial sums, grow with the rows per lane).
__host__ __device__ constexpr int bwd_max_regs(int K, int elem, bool gq) {
  return 65536 / (32 * bwd_warps_per_sm(K, elem, gq)) / 8 * 8 > 255
             ? 255
             : 65536 / (32 * bwd_warps_per_sm(K, elem, gq)) / 8 * 8;
}

// GQ: the batch has a per-base gap-continuation track: row r takes eps_r and beta_r, and the
// gap-continuation partials are kept per row (three more sums per row) for d/dgcp_r.
template <typename T, int L, int K, bool GQ = false>
__global__ void __maxnreg__(bwd_max_regs(K, sizeof(T), GQ)) wf_backward(const BwdArgs a) {
  using G_ = TableGeom<T, K>;
  constexpr int G = 32 / L, VW = G_::VW, LS = G_::LS, CS = G_::CS;
  constexpr int kBias = 2;
  constexpr int CKW = ck_width<T>(K), RW = rec_width<T>(K);
  constexpr int kSeg = bwd_seg_len(K, sizeof(T), GQ);
  // Range of the posterior scale exponent h = E_fwd + E_adj over which the raw products of
  // stored forward and adjoint values are accumulated: below kHmin a product is at most
  // 2^(16 + kHmin) of a posterior (dropped); above kHmax the products a lane needs can fall
  // under the type's range, and the pair is finished in FP64.
  constexpr int kHmax = sizeof(T) == 4 ? 100 : 900;
  constexpr int kHmin = sizeof(T) == 4 ? -100 : -900;
  constexpr int kNoScale = -(1 << 30);
  constexpr unsigned FULL = 0xffffffffu;
  // Row tiles (Sec. III-C handles reads up to 1,024 bases): the 32 x 16 group sweeps reads
  // longer than its 512 rows in tiles of 512 rows, as the forward does.  One pair per warp,
  // so every tile loop is warp-uniform.  Phase A runs the tiles top to bottom, each tile's
  // last lane handing its last row (per column) to the next tile's lane 0; phase B runs them
  // bottom to top, each tile's lane 0 handing its first row's adjoints (per column) to the
  // tile above's last lane, which also forms the partials that pair the two rows.
  constexpr bool TILED = L == 32 && K == 16;
  constexpr int LK = L * K;
  const FwdArgs &fa = a.f;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane % L, sub = lane / L;
  // per warp: the table of signed emissions beta * lambda (+ for a match, - for a mismatch)
  // and the segment's step records
  static_assert(bwd_table_bytes(K, sizeof(T)) == (size_t)kCodes * CS * sizeof(T), "table");
  unsigned char *wsm = smem_raw + (size_t)warp * bwd_warp_bytes(K, sizeof(T), GQ);
  T *tblE = reinterpret_cast<T *>(wsm) + lane * LS;
  T *recS = reinterpret_cast<T *>(wsm + bwd_table_bytes(K, sizeof(T)));
  T *recI = recS + (size_t)kSeg * 32 * RW;  // [step][lane]: the step's top-row I
  static_assert(RW % vecw(sizeof(T)) == 0, "records of whole 16-byte groups");
  const int wpb = blockDim.x >> 5;
  T *slot = reinterpret_cast<T *>(a.scratch) + (size_t)(blockIdx.x * wpb + warp) * a.slot_elems;
  T *ckb = slot;
  // after the tiles' checkpoints: the last row of every tile but the last (forward values
  // and the last lane's exponent, per column) and two alternating buffers of a tile's first
  // row adjoints (u, I^ and lane 0's exponent, per column)
  TileCol<T> *fbuf = nullptr, *abuf = nullptr;
  if constexpr (TILED) {
    fbuf = reinterpret_cast<TileCol<T> *>(slot + (size_t)a.ntile_cap * a.ck_tile);
    abuf = fbuf + (size_t)(a.ntile_cap - 1) * a.tile_cols;
  }
  const T eps = sizeof(T) == 4 ? (T)fa.eps32 : (T)fa.eps64;
  const T beta = sizeof(T) == 4 ? (T)fa.beta32 : (T)fa.beta64;

  const int64_t count = *fa.count_dev;
  const int64_t base = fa.offset_dev ? *fa.offset_dev : 0;
  const int64_t nitems = (count + G - 1) / G;
#ifdef PHMM_DEBUG
  // the warp's scratch slot inside the workspace's slot region
  if (fa.dbg_err && (int64_t)blockIdx.x * wpb + warp >= fa.dbg_nslots) {
    if (lane == 0) atomicOr(fa.dbg_err, kDbgSlot);
    return;
  }
#endif

  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(fa.counter, 1);
    const int64_t item = __shfl_sync(FULL, it, 0);
    if (item >= nitems) break;

    // ---- pair and per-row constants ------------------------------------------------------
    const int64_t idx = item * G + sub;
    const bool valid = idx < count;
    int32_t p = -1;
    bool bad = false;
    int m = 0;
    int64_t n = 0, r0 = 0, hs = 0;
    if (valid) {
      p = fa.list[base + idx];
      const int32_t ri = fa.pair_read[p], hi = fa.pair_hap[p];
      if (ri >= 0 && ri < fa.n_reads && hi >= 0 && hi < fa.n_haps) {
        r0 = fa.read_off[ri];
        m = (int)(fa.read_off[ri + 1] - r0);
        hs = hap_start(fa.hap_off[hi], hi);
        n = fa.hap_off[hi + 1] - fa.hap_off[hi];
        const int cap = TILED ? LK * a.ntile_cap : LK;
        if (m <= 0 || m > cap || n <= 0 || (TILED && m > LK && n > a.tile_cols)) bad = true;
#ifdef PHMM_DEBUG
        // the pair's read positions and haplotype codes (with their guards) inside the
        // buffers, and its columns inside the row-tile buffers (sized by the longest one)
        if (!bad && fa.dbg_err &&
            (r0 + m > fa.dbg_sum_m || hs < kHapGuard ||
             hs + ((n + 15) & ~(int64_t)15) + kHapGuard > fa.dbg_hcode_bytes)) {
          atomicOr(fa.dbg_err, kDbgPairIndex);
          bad = true;
        }
        if (!bad && fa.dbg_err && n > a.tile_cols) {
          atomicOr(fa.dbg_err, kDbgCheckpoints);
          bad = true;
        }
#endif
      } else {
        bad = true;
      }
      if (bad) {
        m = 0;
        n = 0;
      }
    }
    if (a.all64) {  // warp-uniform: every pair of the item goes to the FP64 pass as it is
      if (valid && !bad && t == 0) {
        const int bin = bin64_of_m(m);
        a.resc_list[bin][atomicAdd(&a.resc_count[bin], 1)] = p;
      }
      continue;
    }
    const int ntile = (TILED && m > LK) ? (m + LK - 1) / LK : 1;
    const int npad = ntile * LK - m;  // pad rows above row 1, all in the first tile
    const T bnd = n > 0 ? (T)1 / (T)n : (T)0;
    T ap[K], dl[K], zt[K], ei[K];
    T er[GQ ? K : 1];  // per-row gap continuation (track only)
    WfState<T, K> st;
    // per-row constants and the emission table of one tile's rows; the lane's rows start at
    // zero, pad rows carrying the row-0 boundary down in I
    auto setup_tile = [&](int tile) {
#pragma unroll
      for (int rv = 0; rv < K; rv += VW) {
        T ev[kCodes][VW];
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          const int rr = rv + u;
          if (rr >= K) {  // table padding past the lane's rows
#pragma unroll
            for (int c = 0; c < kCodes; ++c) ev[c][u] = 0;
            continue;
          }
          const int pos = tile * LK + t * K + rr - npad;
          const T bias = rr ? (T)(1 << kBias) : (T)1;
          st.M[rr] = 0;
          st.D[rr] = 0;
          T epr = eps, ber = beta;
          if constexpr (GQ) {
            if (pos >= 0) row_gap<T>(fa, r0 + pos, epr, ber);
            er[rr] = epr;
          }
          if (pos >= 0) {
            T Q;
            row_params<T>(fa, r0 + pos, ap[rr], dl[rr], zt[rr], Q, GQ ? (double)ber : 0.0);
            const int code = fa.rcode[r0 + pos];
            ei[rr] = pos == 0 ? (T)0 : epr * bias;
            dl[rr] *= bias;
            st.I[rr] = 0;
            const T em = bias * (ber * ((T)1 - Q)), ex = bias * (ber * (Q / (T)3));
#pragma unroll
            for (int c = 0; c < kNull; ++c) {
              const bool mt = c == code || c == kN || code == kN;
              ev[c][u] = mt ? em : -ex;
            }
            ev[kNull][u] = 0;
          } else {
            ap[rr] = 0;
            dl[rr] = 0;
            zt[rr] = 0;
            ei[rr] = bias;
            st.I[rr] = bnd * (T)(1ll << (kBias * rr));
#pragma unroll
            for (int c = 0; c < kCodes; ++c) ev[c][u] = 0;
          }
        }
#pragma unroll
        for (int c = 0; c < kCodes; ++c) store_vec<T, VW>(tblE + c * CS + rv, ev[c]);
      }
    };

    int steps = n > 0 ? (int)n + L - 1 : 0;
    steps = __reduce_max_sync(FULL, steps);
    // The wavefront enters the lanes one per step over the first roundup16(L) steps (the
    // ramp): there the lanes renormalise after every step, so an empty lane adopts the
    // exponent of the values about to reach it (two-step ramp segments measured wrong
    // gradients); then every kSeg steps.  Segment q < ramp is step q; regular segments start
    // at step ramp.
    const int ramp = steps < ((L + 15) & ~15) ? steps : ((L + 15) & ~15);
    const int nq = ramp + (steps - ramp + kSeg - 1) / kSeg;
    auto seg_begin = [&](int qq) { return qq < ramp ? qq : ramp + kSeg * (qq - ramp); };
    auto seg_len = [&](int qq) { return qq < ramp ? 1 : kSeg; };
    const int fin = n > 0 ? (int)n + L - 1 : 0;
#ifdef PHMM_DEBUG
    // every checkpoint of the warp's longest pair inside the slot (warp-uniform)
    if (fa.dbg_err && nq > a.nchk) {
      if (lane == 0) atomicOr(fa.dbg_err, kDbgCheckpoints);
      continue;
    }
#endif
    // Haplotype codes of the lane's columns over segment qq's steps, one byte per step (at
    // step s lane t is at column s + 1 - t; columns outside 1..n take the null code).  Every
    // lane reads its own 8-byte window, one segment ahead: no code exchange and no load on
    // the steps' dependency chain.  The reverse sweep reuses them.  The window starts at most
    // 31 columns before column 1 and is clamped to start at column n + 1 at the latest, so it
    // stays inside the NULLC guards around the haplotype's codes: no per-step bounds checks.
    static_assert(kSeg <= 8 && kHapGuard >= 32 + 4, "codes of a segment: one 8-byte window");
    constexpr uint64_t kNullCodes = 0x0505050505050505ull;
    auto seg_codes = [&](int qq) -> uint64_t {
      if (qq < 0 || qq >= nq || n <= 0) return kNullCodes;
      const int bb = seg_begin(qq);
      int64_t i0 = (int64_t)bb - t;  // 0-based haplotype position of the window's first step
      if (i0 > n) i0 = n;
      const uintptr_t addr = (uintptr_t)(fa.hcode + hs + i0);
      const uint32_t *w = reinterpret_cast<const uint32_t *>(addr & ~(uintptr_t)3);
      const uint32_t sh = 8u * (uint32_t)(addr & 3);
      const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
      const uint32_t lo = __funnelshift_r(w0, w1, sh), hi = __funnelshift_r(w1, w2, sh);
      return ((uint64_t)hi << 32) | lo;
    };
    auto code_at = [](uint64_t cs, int u) { return (int)((cs >> (8 * u)) & 0xff); };
    // the row above a lower tile, at the columns of the steps b .. b + kSeg - 1 of lane 0
    // (lane u holds column b + u + 1), read once per segment
    auto load_above = [&](const TileCol<T> *above, int b) {
      TileCol<T> cb = {0, 0, 0, 0};
      const int64_t c = (int64_t)b + lane;
      if (above && lane < kSeg && c < n) cb = above[c];
      return cb;
    };
    // one forward step (phase A or the recompute): lane 0 takes the row above its strip from
    // the row-0 boundary (first tile) or from the tile above (its u-th column in cb)
    auto fstep = [&](int code, int u, const TileCol<T> &cb, bool above) {
      T in3[3];
      if constexpr (TILED) {
        T tM = 0, tI = bnd * st.f, tT = bnd * st.f;  // K0 D(0, j), in lane 0's scale
        if (above) {  // warp-uniform (one pair per warp)
          const T bM = __shfl_sync(FULL, cb.M, u), bI = __shfl_sync(FULL, cb.I, u);
          const T bX = __shfl_sync(FULL, cb.X, u), bE = __shfl_sync(FULL, cb.E, u);
          const T cv = Num<T>::exp2i((int)bE - st.E - kBias * (K - 1));
          tM = bM * cv;
          tI = bI * cv;
          tT = bX * cv;
        }
        wf_step<T, L, K, true, true, true, true, true, GQ>(st, code, t, bnd, eps, tblE, ap, dl,
                                                           zt, ei, in3, tM, tI, tT, er);
      } else {
        wf_step<T, L, K, true, true, true, false, true, GQ>(st, code, t, bnd, eps, tblE, ap, dl,
                                                            zt, ei, in3, 0, 0, 0, er);
      }
    };

    // ---- phase A: forward with checkpoints, tile by tile from the top ---------------------
    T Sfin = 0;
    int Efin = 0;
    uint32_t nz_end = 0;  // bit per tile: the lane's state is nonzero after its last segment
    for (int tile = 0; tile < ntile; ++tile) {
      const bool last_tile = tile == ntile - 1;
      if constexpr (TILED) __syncwarp();  // the tile above's last row is in memory
      setup_tile(tile);
      T *ckt = ckb + (size_t)tile * a.ck_tile;
      const TileCol<T> *above = nullptr;
      TileCol<T> *below_out = nullptr;
      if constexpr (TILED) {
        if (tile > 0) above = fbuf + (size_t)(tile - 1) * a.tile_cols;
        if (!last_tile) below_out = fbuf + (size_t)tile * a.tile_cols;
      }
      st.c = kNull;
      st.Md = 0;
      st.Sd = (t == 0 && tile == 0) ? bnd : (T)0;
      st.acc = 0;
      st.f = t == 0 ? (T)1 : Num<T>::exp2i(-kBias * (K - 1));
      st.E = 0;
      if constexpr (TILED) {
        // lane 0 of a lower tile starts at the exponent that brings column 1 of the row above
        // near 1 (its own state is still zero, so this changes nothing else)
        if (above && t == 0) {
          const TileCol<T> c1 = above[0];
          const T mx = fmax(c1.M, fmax(c1.I, c1.X));
          st.E = mx > (T)0 ? (int)c1.E - kBias * (K - 1) + Num<T>::ilog2(mx) : 0;
          st.f = Num<T>::exp2i(-st.E);
        }
      }
      bool done = false;
      // whether the lane's forward state is nonzero at the current checkpoint (kept with the
      // checkpoint's exponent, so the reverse knows which segments hold forward values)
      bool nzA;
      {
        T mx = fmax(st.Md, st.Sd);
#pragma unroll
        for (int r = 0; r < K; ++r) mx = fmax(mx, st.I[r]);  // M and D start at zero
        nzA = mx > (T)0;
      }
      uint64_t segc = seg_codes(0);
      for (int q = 0; q < nq; ++q) {
        const int b = seg_begin(q);
        const int len = seg_len(q);
        const uint64_t cur = segc;
        segc = seg_codes(q + 1);
        {
          T ck[CKW];
#pragma unroll
          for (int r = 0; r < K; ++r) {
            ck[r] = st.M[r];
            ck[K + r] = st.D[r];
          }
          ck[2 * K] = st.I[0];
          ck[2 * K + 1] = st.Md;
          ck[2 * K + 2] = st.Sd;
          ck[2 * K + 3] = st.f;
          ck[2 * K + 4] = int_bits<T>(2 * st.E + (nzA ? 1 : 0));
#pragma unroll
          for (int k = 2 * K + 5; k < CKW; ++k) ck[k] = 0;
          rec_store<T, CKW, true>(ckt + (size_t)q * 32 * CKW, lane, ck);
        }
        TileCol<T> cb = {0, 0, 0, 0};
        if constexpr (TILED) cb = load_above(above, b);
        for (int u = 0; u < len; ++u) {
          fstep(code_at(cur, u), u, cb, above != nullptr);
          if constexpr (TILED) {
            // the tile's last row, column by column, for the tile below
            const int64_t j = (int64_t)b + u + 1 - (L - 1);  // the last lane's column
            if (below_out && t == L - 1 && j >= 1 && j <= n) {
              TileCol<T> o;
              o.M = st.M[K - 1];
              o.I = st.I[K - 1];
              o.X = st.I[K - 1] + zt[K - 1] * st.D[K - 1];
              o.E = (T)st.E;
              below_out[j - 1] = o;
            }
          }
        }
        if (last_tile && !done && b + len >= fin) {
          Sfin = st.acc;
          Efin = st.E;
          done = true;
        }
        nzA = wf_rescale<T, L, K, kBias>(st, t);
      }
      if (last_tile && !done) {
        Sfin = st.acc;
        Efin = st.E;
      }
      if (nzA) nz_end |= 1u << tile;
    }
    // L = S * 2^(ES - kBias (K-1)), held by the last lane of the group (last tile)
    const T S = __shfl_sync(FULL, Sfin, sub * L + L - 1);
    const int ES = __shfl_sync(FULL, Efin, sub * L + L - 1);
    const bool okS = S > (T)0 && S < (sizeof(T) == 4 ? (T)3.0e38f : (T)1.7e308);
    bool hard = !okS;

    // ---- phase B: adjoint, tile by tile from the bottom, segment by segment from the right
    const double dy = (valid && !bad && a.dL) ? a.dL[p] : 1.0;
    const int64_t po = (valid && !bad) ? a.poff[p] : 0;
    const float nanv = __int_as_float(0x7fc00000);
    int hs_pair = 0, why_h = 0, why_f = 0;
    T dgcp_pair = 0;  // d log10 L / d gcp, summed over the tiles
    // the adjoint enters the pair's lanes one per step from its last column on: renormalise
    // after every one of the first ramp_b such steps (a window set by the pair alone, so the
    // result does not depend on which pairs share the warp), then at segment boundaries
    const int ramp_b = 16 + ((L + 15) & ~15);
    for (int tile = ntile - 1; tile >= 0; --tile) {
      const bool last_tile = tile == ntile - 1;
      // the tile below's partials and first-row adjoints (and phase A's rows) are in memory
      __syncwarp();
      setup_tile(tile);
      T *ckt = ckb + (size_t)tile * a.ck_tile;
      // pad rows: the rows above row 1 (their partials are never used)
      const int first = npad - tile * LK - t * K;  // local index of the lane's first real row
      // lanes whose products can matter: those holding a real row, and the pad lane just
      // above a first real row that starts a lane (its last row's S feeds that row's beta
      // partial)
      const bool real_lane = first <= K;
      // Coefficients of the row just below the strip (the lower lane's row 0, unbiased); the
      // last lane of a tile above another takes the next tile's first row
      T apb = __shfl_down_sync(FULL, ap[0], 1, L);
      T dlb = __shfl_down_sync(FULL, dl[0], 1, L);
      T eib = __shfl_down_sync(FULL, ei[0], 1, L);
      const TileCol<T> *above = nullptr, *ain = nullptr;
      TileCol<T> *aout = nullptr;
      if constexpr (TILED) {
        if (tile > 0) {
          above = fbuf + (size_t)(tile - 1) * a.tile_cols;
          aout = abuf + (size_t)(tile & 1) * a.tile_cols;
        }
        if (!last_tile) {
          ain = abuf + (size_t)((tile + 1) & 1) * a.tile_cols;
          if (t == L - 1) {
            const int64_t gb = r0 + (int64_t)(tile + 1) * LK - npad;
            T zdum, Qdum, epb = eps, beb = beta;
            if constexpr (GQ) row_gap<T>(fa, gb, epb, beb);
            row_params<T>(fa, gb, apb, dlb, zdum, Qdum, GQ ? (double)beb : 0.0);
            eib = epb;
          }
        }
      }
      AdjState<T, K> as;
#pragma unroll
      for (int r = 0; r < K; ++r) as.u[r] = as.Db[r] = 0;
      as.Itop = as.diagU = 0;
      as.EB = (last_tile && t == L - 1) ? -ES : 0;
      as.fB = 0;
      as.seed = 0;
      as.nz = false;
      // the seed 1/L enters at row m only (the last tile's last lane)
      // 1/L in the stored scale: 2^(-ES - EB) / S, formed as 2^(-ES - EB) (1/S) (the same
      // value: scaling by a power of two does not change the rounding)
      const T Sseed = (last_tile && okS) ? (T)1 / S : (T)0;
      adj_rescale<T, L, K, kBias>(as, t, Sseed, ES);
      // Partial sums, each held as (true value) x 2^-H, the lane's accumulator scale.
      // Per row r: gA (alpha_r: u(r,j+1) M(r-1,j)), gD (delta_r: I^(r,j) M(r-1,j)),
      // gZ (zeta_r: D^(r,j+1) M(r,j)), gX (the mismatch-column part of M^(r,j) M(r,j),
      // times -e_mismatch).  gAl / gDl: the products for the lower lane's row 0.
      // Lane scalars: gEI (eps via I: I^(r+1,j) I(r,j) over the lane's rows, the lower
      // lane's row 0 apart in gEIe), gED (eps via D), gMe (M at row m: seed x M(m,j)).
      // The M occupancy per row (sum_j M^ M) and the beta sum are not accumulated: flow
      // conservation of the posterior gives them from the sums above (phase C).
      // With a per-base track the beta and eps sums are kept per row instead: gSr (beta_r),
      // gEIr and gEDr (eps_r), with gSl / gEIl the lower lane's row 0.
      T gA[K], gD[K], gZ[K], gX[K];
#pragma unroll
      for (int r = 0; r < K; ++r) gA[r] = gD[r] = gZ[r] = gX[r] = 0;
      T gAl = 0, gDl = 0, gEI = 0, gEIe = 0, gED = 0, gMe = 0;
      T gSr[GQ ? K : 1], gEIr[GQ ? K : 1], gEDr[GQ ? K : 1], gSl = 0, gEIl = 0;
#pragma unroll
      for (int r = 0; r < (GQ ? K : 1); ++r) gSr[r] = gEIr[r] = gEDr[r] = 0;
      int H = kNoScale;
      // lane 0's row above its strip (row 0 of the DP, or a pad row): S = K0 D(0, j); below
      // the first tile that row is the tile above's last row, whose lane forms the product
      // (per-base track only: the scalar beta sum follows from flow conservation)
      const T bndS = (GQ && t == 0 && tile == 0) ? bnd : (T)0;
      // a lane holding pad rows: its forward I there (the row-0 boundary passed down) is
      // taken as zero in the reverse, so products across pad rows vanish without a per-row
      // test (the per-base track's beta_r sums keep the boundary)
      const bool padl = !GQ && first > 0;
      // the last lane of a tile above another: the tile below's first-row adjoints of the
      // segment's columns (lane u: the column of reverse step b + u), and the exponent and
      // size of the next ones to arrive (for the lane's renormalisation)
      TileCol<T> ab = {0, 0, 0, 0};
      int Eo = 0;
      T xo = 0;
      // until the first nonzero adjoint arrives from the tile below, that lane's state is all
      // zero: it then takes the exponent that brings the arriving values near 1
      bool got_in = false;

      // the lanes' codes of each segment's steps, loaded one segment ahead as in phase A
      uint64_t segc = seg_codes(nq - 1);
      bool nz_next = (nz_end >> tile) & 1;  // the state after the last segment
      // A segment's closing renormalisation is applied at the start of the next segment's
      // reverse, when that segment's forward exponent EF is known: a lane then keeps
      // EF + EB = H where it can, so its partial sums need no re-basing.
      bool pend = false;
      // The checkpoint of the segment to the left is copied (cp.async) into the last two
      // step-record slots once the reverse has read them, so the next restore reads shared
      // memory.  Every record access is lane-private ([group][lane] layout, each lane its own
      // 16-byte groups), so no warp synchronisation is needed.
      static_assert(CKW <= 2 * RW, "a checkpoint fits in two record slots");
      constexpr bool kPf = kSeg >= 3;
      T *const ckS = recS + (size_t)(kSeg - 2) * 32 * RW;
      bool ck_smem = false;
      for (int q = nq - 1; q >= 0; --q) {
        const int b = seg_begin(q);
        const int len = seg_len(q);
        const uint64_t codes = segc;
        segc = seg_codes(q - 1);
        bool nzq;
        {
          T ck[CKW];
          if (ck_smem) {  // copied into the record slots during the previous segment's reverse
            cp_async_wait();
            rec_load<T, CKW>(ckS, lane, ck);
          } else {
            rec_load<T, CKW, true>(ckt + (size_t)q * 32 * CKW, lane, ck);
          }
          ck_smem = false;
#pragma unroll
          for (int r = 0; r < K; ++r) {
            st.M[r] = ck[r];
            st.D[r] = ck[K + r];
          }
          st.I[0] = ck[2 * K];
          // the other rows' I by Eq. 2, as the forward step formed them (power-of-two
          // renormalisation commutes with it)
#pragma unroll
          for (int r = 1; r < K; ++r) st.I[r] = dl[r] * st.M[r - 1] + ei[r] * st.I[r - 1];
          st.Md = ck[2 * K + 1];
          st.Sd = ck[2 * K + 2];
          st.f = ck[2 * K + 3];
          const int ef = bits_int<T>(ck[2 * K + 4]);
          st.E = ef >> 1;
          nzq = (ef & 1) != 0;
        }
        // bring the next (left) segment's checkpoint from DRAM towards L2 while this one runs
        if (q > 0 && lane == 0)
          prefetch_l2(ckt + (size_t)(q - 1) * 32 * CKW, 32 * CKW * sizeof(T));
        // forward values in the lane over this segment: nonzero at its start or at its end (a
        // lane's state turns nonzero once and stays so; power-of-two rescaling keeps zeros)
        const bool nzF = nzq || nz_next;
        nz_next = nzq;
        TileCol<T> cb = {0, 0, 0, 0};
        if constexpr (TILED) {
          cb = load_above(above, b);
          if (ain) {
            // reverse step b + u of the last lane is at column b + u + 2 - L
            const int64_t c = (int64_t)b + lane + 1 - L;
            ab = (lane < kSeg && c >= 0 && c < n) ? ain[c] : TileCol<T>{0, 0, 0, 0};
            const T nM = __shfl_sync(FULL, ab.M, len - 1), nI = __shfl_sync(FULL, ab.I, len - 1);
            Eo = (int)__shfl_sync(FULL, ab.E, len - 1);
            xo = fmax(fabs(nM), nI);
          }
        }
        // recompute the segment, recording the lane's rows after each step (column b+u2+1-t)
        for (int u2 = 0; u2 < len; ++u2) {
          fstep(code_at(codes, u2), u2, cb, above != nullptr);
          {
            T rec[RW];
#pragma unroll
            for (int r = 0; r < K; ++r) {
              rec[r] = st.M[r];
              rec[K + r] = st.D[r];
            }
#pragma unroll
            for (int k = 2 * K; k < RW; ++k) rec[k] = 0;  // odd rows: padding to 16 bytes
            rec_store<T, RW>(recS + (size_t)u2 * 32 * RW, lane, rec);
            recI[u2 * 32 + lane] = st.I[0];
          }
        }
        const int EF = st.E;
        // lane 0's boundary row in its own scale (per-base track only)
        const T fS = GQ ? bndS * Num<T>::exp2i(-EF) : (T)0;
        if (__any_sync(FULL, pend))
          adj_rescale<T, L, K, kBias>(as, t, Sseed, ES, pend, H != kNoScale, H - EF,
                                      ain != nullptr, Eo, xo);
        pend = false;
        // reverse over the segment
        // slots kSeg-2 and kSeg-1 are free from reverse step pf_u on (a one-step ramp segment
        // uses slot 0 only)
        const int pf_u = (kPf && q > 0) ? (len - 1 < kSeg - 3 ? len - 1 : kSeg - 3) : -1;
        for (int u2 = len - 1; u2 >= 0; --u2) {
          if (u2 == pf_u) {
            rec_copy_async<T, CKW>(ckS, ckt + (size_t)(q - 1) * 32 * CKW, lane);
            ck_smem = true;
          }
          const int j = b + u2 + 1 - t;  // this lane's column at this step (n < 2^30)
          const int c = code_at(codes, u2);
          // forward values of the lane's rows at column j: M, I, D/zeta (rec[r], [K+r], [2K+r])
          // (the other rows' I follow from the top row's by Eq. 2; a lane holding pad rows
          // takes its top I as zero, which makes I zero down to its first real row, where
          // I is zero anyway)
          T rec[3 * K];
          {
            T sr[RW];
            rec_load<T, RW>(recS + (size_t)u2 * 32 * RW, lane, sr);
#pragma unroll
            for (int r = 0; r < K; ++r) {
              rec[r] = sr[r];
              rec[2 * K + r] = sr[K + r];
            }
            rec[K] = recI[u2 * 32 + lane];
          }
          if constexpr (!GQ) rec[K] = padl ? (T)0 : rec[K];
#pragma unroll
          for (int r = 1; r < K; ++r) rec[K + r] = dl[r] * rec[r - 1] + ei[r] * rec[K + r - 1];
          T e[K];
          load_rows<T, K>(tblE + c * CS, e);
          T rU = __shfl_down_sync(FULL, as.u[0], 1, L);
          T rI = __shfl_down_sync(FULL, as.Itop, 1, L);
          bool adopt_now = false;  // the exponent changed: every lane's factors are renewed
          if (TILED && ain) {  // warp-uniform (one pair per warp)
            // the tile below's lane 0 at this column, converted to this lane's scale
            const T bM = __shfl_sync(FULL, ab.M, u2), bI = __shfl_sync(FULL, ab.I, u2);
            const int bE = (int)__shfl_sync(FULL, ab.E, u2);
            if (t == L - 1) {
              xo = fmax(fabs(bM), bI);
              Eo = bE;
              if (!got_in && xo > (T)0) {
                as.EB = bE - kBias * (K - 1) + Num<T>::ilog2(xo);
                got_in = true;
                adopt_now = true;
              }
              const T cvB = Num<T>::exp2i(bE - as.EB - kBias * (K - 1));
              rU = bM * cvB;
              rI = bI * cvB;
            } else {
              rU *= as.fB;
              rI *= as.fB;
            }
          } else {  // fB is zero in the last lane (no lane below)
            rU *= as.fB;
            rI *= as.fB;
          }
          const T ubK = as.diagU;
          as.diagU = rU;
          // the seed is nonzero in the last lane of the last tile only
          const T sd = (uint32_t)(j - 1) < (uint32_t)n ? as.seed : (T)0;
          // Posterior scale 2^(EF + EB): products of stored forward and adjoint values are
          // accumulated raw, the accumulators re-based when the scale changes.  Lanes whose
          // forward or adjoint values are all zero contribute nothing; h > kHmax with both
          // nonzero means forward and adjoint mass sit in disjoint cells of the lane, beyond
          // the type's range: the pair goes to FP64.
          const int h = EF + as.EB;
          const bool nzB = as.nz || rU != (T)0 || rI != (T)0 || sd != (T)0;
          const bool live = real_lane && nzF && nzB;
          if (live && h > kHmax) hard = true;
          // A step whose posterior scale is negligible (h < kHmin) adds its products at scale
          // kHmin: each is then counted 2^(kHmin - h) times too large, yet stays below
          // 2^(16 + kHmin) of a posterior, far under the rounding of the sums it joins.
          // Every lane runs the same code, with no per-step zeroing.
          const int hq = h < kHmin ? kHmin : h;
          if (live && hq <= kHmax && hq != H) {
            // re-base the sums from 2^-H to 2^-hq (all zero while H is unset); a shift beyond
            // the type's exponent range is applied in two exact halves
            auto rebase = [&](T sc) {
#pragma unroll
              for (int r = 0; r < K; ++r) {
                gA[r] *= sc;
                gD[r] *= sc;
                gZ[r] *= sc;
                gX[r] *= sc;
              }
              gAl *= sc;
              gDl *= sc;
              gEI *= sc;
              gEIe *= sc;
              gED *= sc;
              gMe *= sc;
              if constexpr (GQ) {
#pragma unroll
                for (int r = 0; r < K; ++r) {
                  gSr[r] *= sc;
                  gEIr[r] *= sc;
                  gEDr[r] *= sc;
                }
                gSl *= sc;
                gEIl *= sc;
              }
            };
            if (H != kNoScale) {
              int d = H - hq;
              if (d > kHmax + 20 || d < -(kHmax + 20)) {
                rebase(Num<T>::exp2i(d / 2));
                d -= d / 2;
              }
              rebase(Num<T>::exp2i(d));
            }
            H = hq;
          }
          // Lanes that are not live add zeros (all forward or all adjoint values zero),
          // garbage that is discarded (pad lanes) or garbage of a pair that goes to FP64
          // (h > kHmax): no per-row branch.
          T ub = ubK, Ibl = rI;
          {
#pragma unroll
            for (int r = K - 1; r >= 0; --r) {
              const T apB = r == K - 1 ? apb : ap[r + 1];
              const T dlB = r == K - 1 ? dlb : dl[r + 1];
              const T eiB = r == K - 1 ? eib : ei[r + 1];
              const T uba = fabs(ub);       // u(r+1, j+1); u carries the emission's sign
              const T zD = zt[r] * as.Db[r];
              const T Mv = rec[r], Iv = rec[K + r], Dv = rec[2 * K + r];  // forward, column j
              // M^(r, j); the last row of the last lane adds the seed 1/L (no addition of a
              // zero elsewhere: x + 0 is not free in IEEE arithmetic)
              const T Mb0 = fma(apB, uba, fma(dlB, Ibl, zD));
              const T Mb = r == K - 1 ? Mb0 + sd : Mb0;
              // I^(r, j): one FMA on the row-to-row chain
              const T Ib = fma(eiB, Ibl, r == K - 1 ? uba + sd : uba);
              const T Dn = uba + (GQ ? er[r] : eps) * as.Db[r];            // D^(r, j)
              const T un = e[r] * Mb;                                      // u(r, j)
              {
                if (r == K - 1) {
                  gAl += uba * Mv;
                  gDl += Ibl * Mv;
                  gMe += sd * Mv;
                } else {
                  gA[r + 1] += uba * Mv;
                  gD[r + 1] += Ibl * Mv;
                }
                if constexpr (GQ) {
                  // the I -> I partial counts only where the row below is a real row (pad
                  // rows pass the boundary down with a nonzero coefficient)
                  const T Il = eiB * Ibl;
                  if (r == K - 1) {
                    gSl += uba * (Iv + zt[r] * Dv);
                    gEIl += (r + 1 > first ? Il : (T)0) * Iv;
                  } else {
                    gSr[r + 1] += uba * (Iv + zt[r] * Dv);
                    gEIr[r + 1] += (r + 1 > first ? Il : (T)0) * Iv;
                  }
                  gEDr[r] += zD * Dv;
                } else {
                  // eps x I^(r+1, j) I(r, j) with the row's coefficient eps x bias applied
                  // in phase C; the pad rows' I is zero here (padl), and the coefficient of
                  // a first real row is zero, so only real-to-real transitions count
                  if (r == K - 1) gEIe += Ibl * Iv;
                  else gEI += Ibl * Iv;
                  gED += zD * Dv;
                }
                gZ[r] += as.Db[r] * Mv;
                gX[r] += fmin(un, (T)0) * Mv;
              }
              ub = as.u[r];
              as.u[r] = un;
              as.Db[r] = Dn;
              Ibl = Ib;
            }
            // lane 0's row above: u(0, j+1) times the boundary S = K0 D(0, j)
            if constexpr (GQ) gSr[0] += fabs(ub) * fS;
          }
          as.Itop = Ibl;
          if constexpr (TILED) {
            // this tile's first row adjoints for the tile above (before any renormalisation)
            if (aout && t == 0 && j >= 1 && j <= n) {
              TileCol<T> o;
              o.M = as.u[0];
              o.I = as.Itop;
              o.X = 0;
              o.E = (T)as.EB;
              aout[j - 1] = o;
            }
          }
          const int sf = b + u2 + 1;  // forward step just reversed
          // Inside the adjoint's ramp (the first ramp_b steps from the pair's last column, a
          // window set by the pair alone) a lane without adjoint mass renormalises after every
          // step, to adopt the exponent of the values about to arrive; every lane
          // renormalises at the segment's end (deferred to the next segment's start).
          const bool apply = (sf <= fin && sf > fin - ramp_b && !as.nz) || adopt_now;
          if (u2 == 0) pend = sf <= fin && !apply;
          if (__any_sync(FULL, apply))
            adj_rescale<T, L, K, kBias>(as, t, Sseed, ES, apply, false, 0, ain != nullptr, Eo,
                                        xo);
        }
      }

      // ---- phase C: chain rule to the Phred inputs, per-pair partials of the tile's rows --
      // accumulators to true values; the products of a row's I^ with the row above's M
      // carry one row bias less than the others (x 2^kBias), except across the lane edge
      const T sc = H == kNoScale ? (T)0 : Num<T>::exp2i(H);
      // M occupancy of each row, sum_j M^(r,j) M(r,j): by flow conservation at M(r,j) it
      // is the sum over the cell's out-transitions (to M(r+1,j+1), I(r+1,j), D(r,j+1)) and,
      // at row m, the path's end, each weighted by its coefficient as the reverse step
      // forms M^ (the same scale and row biases)
      T gY[K];
#pragma unroll
      for (int r = 0; r < K; ++r) {
        const T y = r == K - 1 ? fma(apb, gAl, fma(dlb, gDl, gMe))
                               : fma(ap[r + 1], gA[r + 1], dl[r + 1] * gD[r + 1]);
        gY[r] = fma(zt[r], gZ[r], y) * sc;
      }
      gAl *= sc;
      gDl *= sc;
      T dAlpha[K], dDelta[K];
#pragma unroll
      for (int r = 0; r < K; ++r) {
        dAlpha[r] = gA[r] * sc;
        dDelta[r] = gD[r] * (sc * (T)(1 << kBias));
        gZ[r] *= sc;
        gX[r] *= sc;
      }
      {
        const T aup = __shfl_up_sync(FULL, gAl, 1, L);
        const T dup = __shfl_up_sync(FULL, gDl, 1, L);
        dAlpha[0] = t == 0 ? (T)0 : aup;
        dDelta[0] = t == 0 ? (T)0 : dup;
      }
      // eps: the I -> I products carry one row bias less (x 2^kBias) except across the
      // lane edge.  beta (scalar gap continuation): flow conservation at the M states gives
      // the expected number of transitions into M through beta (from I, from D, and the
      // start from D(0, .)) as that of the transitions out of M into I and D plus the
      // path's end in M at row m: sum over the rows of delta_r dDelta_r + zeta_r dZeta_r,
      // plus seed x sum_j M(m,j).  Pad lanes' scalar sums are zero or discarded.
      T gSs = 0, gEs = real_lane ? (gED + (T)(1 << kBias) * gEI + gEIe) * sc : (T)0;
      if constexpr (!GQ) {
        gSs = gMe * sc;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const int pos = tile * LK + t * K + r - npad;
          if (pos >= 0) {
            T dum, del, zet, Q;
            row_params<T>(fa, r0 + pos, dum, del, zet, Q);
            gSs = fma(del, dDelta[r], fma(zet, gZ[r], gSs));
          }
        }
        if (TILED && !last_tile && t == L - 1) {
          // the next tile's first row: its M -> I transitions pair this lane's last row
          const T del = dlb;  // that row's delta (unbiased)
          gSs = fma(del, gDl, gSs);
        }
      }
      T spec = 0;  // the beta term of M(1,1), true value (per-base track; see below)
      if (GQ && t == 0 && tile == 0 && first <= K) {
        // Lane 0 never visits column 0, so when lane 0 holds row 1 or the row above it, the
        // beta term of M(1,1) = lambda beta D(0,0), u(1,1) S(0,0), is added here: the reverse
        // sweep ended at column 1 (as.u holds u(., 1); as.diagU the lower lane's u(row 0, 1)),
        // and S(0,0) is the row above row 1 at column 0 in the initial scale (E = 0): the
        // boundary K0/n, times the pad pass-through bias when row 1 is not the lane's row 0.
        T uf = first == K ? fabs(as.diagU) : (T)0;
#pragma unroll
        for (int r = 0; r < K; ++r)
          if (r == first) uf = fabs(as.u[r]);
        const T S00 = first == 0 ? bnd : bnd * (T)(1ll << (kBias * (first - 1)));
        spec = (uf * S00) * Num<T>::exp2i(as.EB / 2) * Num<T>::exp2i(as.EB - as.EB / 2);
        gSs += spec;
      }
      // With a per-base track: d log10 L / d gcp_r of the lane's rows, from the per-row sums
      // (the lower lane's row 0 receives this lane's gSl / gEIl; row 1 the M(1,1) term) and,
      // for the last lane of a tile above another, the same for the next tile's first row.
      T dgq[GQ ? K : 1];
      T dgq_next = 0;
      if constexpr (GQ) {
        const T upS = __shfl_up_sync(FULL, gSl * sc, 1, L);
        const T upE = __shfl_up_sync(FULL, gEIl * sc, 1, L);
        const T specUp = __shfl_up_sync(FULL, spec, 1, L);
        const int firstUp = __shfl_up_sync(FULL, first, 1, L);
        gSs = 0;
        gEs = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const int pos = tile * LK + t * K + r - npad;
          T Sr = gSr[r] * sc, Er = gEDr[r] * sc + gEIr[r] * sc / er[r];
          if (r == 0 && t > 0) {
            Sr += upS;
            Er += upE / er[0];
            if (t == 1 && tile == 0 && firstUp == K) Sr += specUp;
          }
          if (t == 0 && r == first) Sr += spec;
          dgq[r] = 0;
          if (pos >= 0) {
            T epr, ber;
            row_gap<T>(fa, r0 + pos, epr, ber);
            dgq[r] = -(Er - Sr / ber) * epr * (T)0.1;
            gSs += dgq[r];  // the lane's sum of d log10 L / d gcp_r
          }
        }
        if (TILED && !last_tile && t == L - 1) {
          const int64_t pos = (int64_t)(tile + 1) * LK - npad;
          T epr, ber;
          row_gap<T>(fa, r0 + pos, epr, ber);
          dgq_next = -(gEIl * sc / epr - gSl * sc / ber) * epr * (T)0.1;
          gSs += dgq_next;
        }
      }
      bool finite = true;  // over the real rows (pad rows' sums are never used)
#pragma unroll
      for (int r = 0; r < K; ++r)
        if (r >= first)
          finite = finite && fabs(dAlpha[r]) < (T)1e30 && fabs(dDelta[r]) < (T)1e30 &&
                   fabs(gZ[r]) < (T)1e30 && fabs(gY[r]) < (T)1e30 &&
                   fabs(gX[r]) < (T)1e30;  // false for NaN too
      if (TILED && !last_tile && t == L - 1)
        finite = finite && fabs(gAl) < (T)1e30 && fabs(gDl) < (T)1e30 &&
                 fabs(dgq_next) < (T)1e30;
      if constexpr (GQ) {
#pragma unroll
        for (int r = 0; r < K; ++r)
          if (r >= first) finite = finite && fabs(dgq[r]) < (T)1e30;
      }
      int hs_any = (hard || !finite) ? 1 : 0;
      int wh = hard ? 1 : 0, wf = finite ? 0 : 1;
#pragma unroll
      for (int o = 1; o < L; o <<= 1) {
        gSs += __shfl_xor_sync(FULL, gSs, o, L);
        gEs += __shfl_xor_sync(FULL, gEs, o, L);
        hs_any |= __shfl_xor_sync(FULL, hs_any, o, L);
        wh |= __shfl_xor_sync(FULL, wh, o, L);
        wf |= __shfl_xor_sync(FULL, wf, o, L);
      }
      // d ln L / d eps = gEs - gSs / beta (gSs: the beta count; beta = 1 - eps);
      // d eps / d gcp = -(ln 10 / 10) eps
      // (with a per-base track gSs already holds the sum of the rows' d log10 L / d gcp_r)
      const T dgcp_l = GQ ? gSs : -(gEs - gSs / beta) * eps * (T)0.1;
      if (!(fabs(dgcp_l) < (T)1e30)) hs_any = 1;
      hs_pair |= hs_any;
      why_h |= wh;
      why_f |= wf;
      dgcp_pair += dgcp_l;
      if (valid && !bad && !hs_pair) {
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const int pos = tile * LK + t * K + r - npad;
          if (pos < 0) continue;
          T dum, del, zet, Q, epr = eps, ber = beta;
          if constexpr (GQ) row_gap<T>(fa, r0 + pos, epr, ber);  // the row's beta
          row_params<T>(fa, r0 + pos, dum, del, zet, Q, GQ ? (double)ber : 0.0);
          const T gAlpha = dAlpha[r] / ber;  // d ln L / d alpha_r
          T di, dd;
          if (fa.alpha_mode) {
            const T iq = (T)qual_at(fa.iq, fa.qual_f32, r0 + pos);
            const T dq = (T)qual_at(fa.dq, fa.qual_f32, r0 + pos);
            const T pa = sizeof(T) == 4 ? (T)exp10f((float)(-(iq + dq) * (T)0.1))
                                        : (T)exp10(-(double)(iq + dq) / 10.0);
            di = -(dDelta[r] * del - gAlpha * pa) * (T)0.1;
            dd = -(gZ[r] * zet - gAlpha * pa) * (T)0.1;
          } else {
            di = -(dDelta[r] - gAlpha) * del * (T)0.1;
            dd = -(gZ[r] - gAlpha) * zet * (T)0.1;
          }
          // emission partial: with A1, A2 the match / mismatch parts of sum_j M^ M (the
          // posterior occupancy of M), d ln L / dQ = -A1 / (1 - Q) + A2 / Q, since
          // lambda = 1 - Q on a match and Q / 3 on a mismatch.  gX holds -ex A2 with ex
          // the row's stored (biased) mismatch emission.
          const T bias = r ? (T)(1 << kBias) : (T)1;
          const T ex = bias * (ber * (Q / (T)3));
          const T A2 = -gX[r] / ex;
          const T A1 = gY[r] - A2;
          // d log10 L / d bq = (d ln L / dQ) (-Q / 10)
          const T db = (A1 * (Q / ((T)1 - Q)) - A2) * (T)0.1;
          a.part_bq[po + pos] = (float)(dy * (double)db);
          a.part_iq[po + pos] = (float)(dy * (double)di);
          a.part_dq[po + pos] = (float)(dy * (double)dd);
          if constexpr (GQ) a.part_gq[po + pos] = (float)(dy * (double)dgq[r]);
        }
        if constexpr (TILED) {
          // The tile below's first row: its alpha and delta partials pair its adjoints with
          // this tile's last row (held by the last lane, which formed them); the tile below
          // wrote the rest of that row's partials already.
          if (!last_tile && t == L - 1) {
            const int64_t pos = (int64_t)(tile + 1) * LK - npad;
            T dum, del, zet, Q, epr = eps, ber = beta;
            if constexpr (GQ) row_gap<T>(fa, r0 + pos, epr, ber);
            row_params<T>(fa, r0 + pos, dum, del, zet, Q, GQ ? (double)ber : 0.0);
            const T gAlpha = gAl / ber;
            T di, dd;
            if (fa.alpha_mode) {
              const T iq = (T)qual_at(fa.iq, fa.qual_f32, r0 + pos);
              const T dq = (T)qual_at(fa.dq, fa.qual_f32, r0 + pos);
              const T pa = sizeof(T) == 4 ? (T)exp10f((float)(-(iq + dq) * (T)0.1))
                                          : (T)exp10(-(double)(iq + dq) / 10.0);
              di = -(gDl * del - gAlpha * pa) * (T)0.1;
              dd = (gAlpha * pa) * (T)0.1;
            } else {
              di = -(gDl - gAlpha) * del * (T)0.1;
              dd = gAlpha * zet * (T)0.1;
            }
            a.part_iq[po + pos] = (float)((double)a.part_iq[po + pos] + dy * (double)di);
            a.part_dq[po + pos] = (float)((double)a.part_dq[po + pos] + dy * (double)dd);
            if constexpr (GQ)
              a.part_gq[po + pos] = (float)((double)a.part_gq[po + pos] + dy * (double)dgq_next);
          }
        }
      }
    }  // tiles

    // ---- the pair's results -----------------------------------------------------------------
    __syncwarp();  // partials written by other lanes of the warp, before any NaN fill
    if (valid && bad && a.out && t == 0) {
      a.out[p] = __longlong_as_double(0x7ff8000000000000ll);
      a.oflags[p] = PHMM_FLAG_INVALID;
    }
    if (valid && !bad) {
      const bool to_rescue = hs_pair && !a.rescue;
      if (to_rescue) {
        if (t == 0) {
          const int bin = bin64_of_m(m);
          const int pos = atomicAdd(&a.resc_count[bin], 1);
          a.resc_list[bin][pos] = p;
          if (a.why) {
            if (why_h) atomicAdd(&a.why[0], 1);
            if (why_f) atomicAdd(&a.why[1], 1);
          }
        }
      } else {
        if (a.out && t == 0) {
          // log10 L = log10(S) + (ES - kBias (K-1)) log10 2, as the forward's per-lane-exponent
          // tier writes it
          constexpr double LOG10_2 = 0.301029995663981195213738894724493027;
          a.out[p] = log10((double)S) + (double)(ES - kBias * (K - 1)) * LOG10_2;
          a.oflags[p] = (uint8_t)(sizeof(T) == 4 ? PHMM_FLAG_FP32 : PHMM_FLAG_RESCUED64) |
                        (uint8_t)PHMM_FLAG_EXTENDED;
        }
        if (hs_pair) {  // no finite gradient: every partial of the pair is NaN
          for (int pos = t; pos < m; pos += L) {
            a.part_bq[po + pos] = nanv;
            a.part_iq[po + pos] = nanv;
            a.part_dq[po + pos] = nanv;
            if (GQ) a.part_gq[po + pos] = nanv;
          }
        }
        if (t == 0) a.pair_dgcp[p] = hs_pair ? (double)nanv : dy * (double)dgcp_pair;
      }
    }
  }
}

using BwdKernel = void (*)(const BwdArgs);

// Instantiation tables (nullptr where a group is not built).  FP32: lanes 4..32, rows per
// lane 4/6/8/10/12 (also 14 with 16 lanes, and 16 with 32 lanes for reads up to 512), and
// odd rows where they fit a read-length range more closely: 4 x 9/11, 8 x 7/9/11,
// 16 x 7/9/11/13, 32 x 7/9; FP64 hand-off groups: 32 lanes x rows 4/8/16.
BwdKernel bwd32_lo(int L, int K);   // L in {4, 8}
BwdKernel bwd32_mid(int L, int K);  // L = 16
BwdKernel bwd32_hi(int L, int K);   // L = 32
BwdKernel bwd32_odd_lo(int L, int K);  // odd rows, L in {4, 8}
BwdKernel bwd32_odd_hi(int L, int K);  // odd rows, L in {16, 32}
BwdKernel bwd64_table(int K);       // L = 32
// per-base gap-continuation track: (16,4) (16,8) (32,8) (32,12) (32,16); FP64 32 x 4/8/16
BwdKernel bwd32_gq(int L, int K);
BwdKernel bwd64_gq(int K);

#define PHMM_BWD_ROWS_SWITCH(T, L)             \
  switch (K) {                                 \
    case 4: return wf_backward<T, L, 4>;       \
    case 6: return wf_backward<T, L, 6>;       \
    case 8: return wf_backward<T, L, 8>;       \
    case 10: return wf_backward<T, L, 10>;     \
    case 12: return wf_backward<T, L, 12>;     \
    default: return nullptr;                   \
  }

}  // namespace phmm
