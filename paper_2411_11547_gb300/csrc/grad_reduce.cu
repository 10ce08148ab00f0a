// Batch-wide FP64 gradient accumulation of the adjoint pass, and the device scans it uses.
//
// Every pair writes its per-read-position partial gradients (FP32, relative to its own
// pair) to a buffer at offset poff[p] = sum_{q < p} m_q.  The reads' gradients are the sums
// over the pairs that share each read; they are formed here in FP64 in increasing pair order
// (a deterministic segmented reduction: counting sort of pairs by read, each read's segment
// sorted by pair id), then rounded once to FP32.  d/dgcp is a fixed-shape FP64 tree sum.
#include <cstdint>
#include "phmm_internal.cuh"

namespace phmm {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

// Block-local exclusive scan of kScanTile elements; writes the tile total to sums[block].
__global__ void __launch_bounds__(kScanBlock)
    k_scan_tile(const int64_t *in, int64_t *out, int64_t n, int64_t *sums) {
  __shared__ int64_t part[kScanBlock];
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)t * kScanItems;
  int64_t v[kScanItems], s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    const int64_t x = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  int64_t run = part[t] - s;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (t == kScanBlock - 1) sums[blockIdx.x] = part[t];
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *offs) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t j = i + (int64_t)k * kScanBlock;
    if (j < n) out[j] += offs[blockIdx.x];
  }
}

// Scratch (int64 elements) scan_exclusive needs for n inputs.
int64_t scan_scratch_elems(int64_t n) {
  int64_t tot = 0;
  while (n > 1) {
    n = (n + kScanTile - 1) / kScanTile;
    tot += 2 * n + 1;
  }
  return tot + 2;
}

// out[i] = sum_{k<i} in[k] (in and out may not alias).  Recursive over tiles.
int scan_exclusive(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch,
                   cudaStream_t s) {
  if (n <= 0) return 0;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  int64_t *sums = scratch, *offs = scratch + nb;
  k_scan_tile<<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, n, sums);
  if (nb > 1) {
    int rc = scan_exclusive(sums, offs, nb, scratch + 2 * nb, s);
    if (rc) return rc;
    k_scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(out, n, offs);
  }
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- pair -> read CSR -----

__global__ void k_pair_len(const int32_t *pr, const int64_t *read_off, int64_t P,
                           int64_t *len) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x)
    len[p] = read_off[pr[p] + 1] - read_off[pr[p]];
}

__global__ void k_read_count(const int32_t *pr, int64_t P, int64_t *cnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[pr[p]]), 1ull);
}

__global__ void k_read_scatter(const int32_t *pr, int64_t P, const int64_t *seg_off,
                               int64_t *cursor, int32_t *seg) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = pr[p];
    const unsigned long long k =
        atomicAdd(reinterpret_cast<unsigned long long *>(&cursor[r]), 1ull);
    seg[seg_off[r] + (int64_t)k] = (int32_t)p;
  }
}

// One warp per read: order the read's segment by pair id (rank = number of smaller ids;
// ids are distinct), using `tmp` as the out-of-place target.
__global__ void k_segment_sort(const int64_t *seg_off, int64_t R, const int32_t *seg,
                               int32_t *sorted) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t b = seg_off[r], e = seg_off[r + 1], c = e - b;
    for (int64_t i = lane; i < c; i += 32) {
      const int32_t v = seg[b + i];
      int64_t rank = 0;
      for (int64_t k = 0; k < c; ++k) rank += seg[b + k] < v;
      sorted[b + rank] = v;
    }
  }
}

// One warp per read: FP64 sum of the partials of its pairs, in pair order, each times
// dL[pair] when dL is given (partials of log10 L itself), else as stored (already scaled).
// part_gq / dgq: the per-base gap-continuation partials (null without a track).
__global__ void k_read_reduce(const int64_t *read_off, int64_t R, const int64_t *seg_off,
                              const int32_t *sorted, const int64_t *poff, const float *part_bq,
                              const float *part_iq, const float *part_dq, const float *part_gq,
                              const double *dL, float *dbq, float *diq, float *ddq,
                              float *dgq) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t r0 = read_off[r], m = read_off[r + 1] - r0;
    const int64_t b = seg_off[r], e = seg_off[r + 1];
    for (int64_t i = lane; i < m; i += 32) {
      double sb = 0.0, si = 0.0, sd = 0.0, sg = 0.0;
      for (int64_t k = b; k < e; ++k) {
        const int32_t pr = sorted[k];
        const int64_t o = poff[pr] + i;
        const double w = dL ? dL[pr] : 1.0;
        sb += w * (double)part_bq[o];
        si += w * (double)part_iq[o];
        sd += w * (double)part_dq[o];
        if (part_gq) sg += w * (double)part_gq[o];
      }
      dbq[r0 + i] = (float)sb;
      diq[r0 + i] = (float)si;
      ddq[r0 + i] = (float)sd;
      if (dgq) dgq[r0 + i] = (float)sg;
    }
  }
}

// Fixed-shape FP64 sum of P values: kSumBlocks block partials, then one block.
constexpr int kSumBlocks = 256;
__global__ void __launch_bounds__(256) k_sum_stage1(const double *x, const double *w, int64_t P,
                                                    double *part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x; i < P; i += (int64_t)kSumBlocks * 256)
    s += w ? w[i] * x[i] : x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void __launch_bounds__(256) k_sum_stage2(const double *part, double *out) {
  __shared__ double sh[256];
  sh[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

static int grid_for(int64_t n, int block, int cap = 152 * 16) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Layout (bytes) of the reduction scratch for P pairs and R reads.
size_t reduce_scratch_bytes(int64_t P, int64_t R) {
  const int64_t n = P > R + 1 ? P : R + 1;
  return 8 * (size_t)(P + 1)                       // pair lengths
         + 8 * (size_t)(P + 1)                     // poff
         + 8 * (size_t)(R + 1) * 3                 // counts, seg_off, cursor
         + 4 * (size_t)(P + 1) * 2                 // seg, sorted
         + 8 * (size_t)scan_scratch_elems(n)       // scans
         + 8 * (size_t)kSumBlocks + 1024;
}

struct ReduceScratch {
  int64_t *len, *poff, *cnt, *seg_off, *cursor, *scan;
  int32_t *seg, *sorted;
  double *sum_part;
};

static ReduceScratch carve(char *base, int64_t P, int64_t R) {
  ReduceScratch s;
  char *p = base;
  auto take = [&](size_t bytes) {
    char *at = p;
    p += (bytes + 255) & ~(size_t)255;
    return at;
  };
  s.len = (int64_t *)take(8 * (size_t)(P + 1));
  s.poff = (int64_t *)take(8 * (size_t)(P + 1));
  s.cnt = (int64_t *)take(8 * (size_t)(R + 1));
  s.seg_off = (int64_t *)take(8 * (size_t)(R + 1));
  s.cursor = (int64_t *)take(8 * (size_t)(R + 1));
  s.seg = (int32_t *)take(4 * (size_t)(P + 1));
  s.sorted = (int32_t *)take(4 * (size_t)(P + 1));
  const int64_t n = P > R + 1 ? P : R + 1;
  s.scan = (int64_t *)take(8 * (size_t)scan_scratch_elems(n));
  s.sum_part = (double *)take(8 * (size_t)kSumBlocks);
  return s;
}

size_t reduce_scratch_bytes_aligned(int64_t P, int64_t R) {
  return reduce_scratch_bytes(P, R) + 12 * 256;
}

// poff[p] = sum_{q<p} m_q (partial-gradient offsets); returns the int64 array in scratch.
int pair_offsets(const phmm_batch &b, char *scratch, int64_t **poff, cudaStream_t s) {
  ReduceScratch rs = carve(scratch, b.n_pairs, b.n_reads);
  if (b.n_pairs > 0) {
    k_pair_len<<<grid_for(b.n_pairs, 256), 256, 0, s>>>(b.pair_read, b.read_off, b.n_pairs, rs.len);
    int rc = scan_exclusive(rs.len, rs.poff, b.n_pairs, rs.scan, s);
    if (rc) return rc;
  }
  *poff = rs.poff;
  return (int)cudaGetLastError();
}

// Per-read FP64 reduction of the pair partials and the FP64 sum of per-pair d/dgcp; with
// dL non-null the per-pair values are partials of log10 L, weighted by dL[p] in FP64.
int reduce_gradients(const phmm_batch &b, char *scratch, const float *part_bq,
                     const float *part_iq, const float *part_dq, const float *part_gq,
                     const double *pair_dgcp, const double *dL, float *dbq, float *diq,
                     float *ddq, float *dgq, double *dgcp, cudaStream_t s, int *launches) {
  ReduceScratch rs = carve(scratch, b.n_pairs, b.n_reads);
  const int64_t P = b.n_pairs, R = b.n_reads;
  cudaMemsetAsync(rs.cnt, 0, 8 * (size_t)(R + 1), s);
  cudaMemsetAsync(rs.cursor, 0, 8 * (size_t)(R + 1), s);
  if (P > 0) k_read_count<<<grid_for(P, 256), 256, 0, s>>>(b.pair_read, P, rs.cnt);
  int rc = scan_exclusive(rs.cnt, rs.seg_off, R + 1, rs.scan, s);
  if (rc) return rc;
  if (P > 0) {
    k_read_scatter<<<grid_for(P, 256), 256, 0, s>>>(b.pair_read, P, rs.seg_off, rs.cursor,
                                                    rs.seg);
    k_segment_sort<<<grid_for(R * 32, 256), 256, 0, s>>>(rs.seg_off, R, rs.seg, rs.sorted);
  }
  k_read_reduce<<<grid_for(R * 32, 256), 256, 0, s>>>(b.read_off, R, rs.seg_off, rs.sorted,
                                                      rs.poff, part_bq, part_iq, part_dq,
                                                      part_gq, dL, dbq, diq, ddq, dgq);
  k_sum_stage1<<<kSumBlocks, 256, 0, s>>>(pair_dgcp, dL, P, rs.sum_part);
  k_sum_stage2<<<1, 256, 0, s>>>(rs.sum_part, dgcp);
  *launches += 8;
  return (int)cudaGetLastError();
}

}  // namespace phmm
