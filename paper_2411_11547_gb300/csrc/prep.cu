// Preparation and length binning kernels of the forward pass.
//
//   validate : input checks at plan time (bases, Phred ranges, pair ids), cell count (Eq. 5)
//   prep_reads : per read position -> base code and FP32 transition/emission parameters
//   prep_haps  : haplotype bases -> codes in a 16-byte-aligned, NULLC-padded buffer so the
//                wavefront's lane 0 reads 16 columns per 128-bit load (Sec. III-B reads char4)
//   pair_keys / scan / scatter : the length partitioning of Sec. III-C, on the GPU: every
//                pair gets the smallest wavefront group that holds its read (key = group,
//                haplotype-length bucket longest first); a counting sort lays the pairs of
//                each group out contiguously so a warp packs pairs of similar length.
#include <cstdint>
#include "phmm_internal.cuh"
#include "wavefront.cuh"

namespace phmm {

__device__ __forceinline__ int base_code(uint8_t b) {
  switch (b) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    case 'N': case 'n': return 4;
    default: return -1;
  }
}

// Error bits of the validation word.
constexpr unsigned kErrBase = 1u, kErrQual = 2u, kErrPair = 4u, kErrAlpha = 8u, kErrGcp = 16u;

__global__ void k_validate_reads(const uint8_t *bases, const void *bq, const void *iq,
                                 const void *dq, const void *gq, int qual_f32, int alpha_mode,
                                 int64_t total, unsigned *err) {
  unsigned e = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (base_code(bases[g]) < 0) e |= kErrBase;
    // a per-base gap-continuation value must leave eps < 1 (beta > 0)
    if (gq && !(qual_at(gq, qual_f32, g) > 0.0)) e |= kErrGcp;
    // uint8 and float32 Phred values are exact in float
    const float b = (float)qual_at(bq, qual_f32, g), i = (float)qual_at(iq, qual_f32, g),
                d = (float)qual_at(dq, qual_f32, g);
    if (!(b >= 0.f) || !(i >= 0.f) || !(d >= 0.f)) e |= kErrQual;  // NaN or negative
    // delta + zeta <= 1 holds whenever both gap quals are >= 10 log10(2) ~ 3.0103 (each term
    // <= 1/2); only below that is the exact FP64 test needed (FP64 is slow on this part)
    if (alpha_mode == 0 && fminf(i, d) < 3.0103f &&
        pow(10.0, -(double)i / 10.0) + pow(10.0, -(double)d / 10.0) > 1.0)
      e |= kErrAlpha;
  }
  if (e) atomicOr(err, e);
}

__global__ void k_validate_haps(const uint8_t *bases, int64_t total, unsigned *err) {
  unsigned e = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x)
    if (base_code(bases[g]) < 0) e |= kErrBase;
  if (e) atomicOr(err, e);
}

__global__ void k_validate_pairs(const int32_t *pr, const int32_t *ph, int64_t P,
                                 const int64_t *read_off, const int64_t *hap_off, int64_t R,
                                 int64_t H, unsigned *err, unsigned long long *cells) {
  unsigned e = 0;
  unsigned long long c = 0, rows = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = pr[p], h = ph[p];
    if (r < 0 || r >= R || h < 0 || h >= H) {
      e |= kErrPair;
      continue;
    }
    c += (unsigned long long)(read_off[r + 1] - read_off[r]) *
         (unsigned long long)(hap_off[h + 1] - hap_off[h]);
    rows += (unsigned long long)(read_off[r + 1] - read_off[r]);
  }
  if (e) atomicOr(err, e);
  // warp-aggregate the cell count (Eq. 5) and the sum over pairs of read lengths
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, o);
    rows += __shfl_down_sync(0xffffffffu, rows, o);
  }
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cells, c);
  if ((threadIdx.x & 31) == 0 && rows) atomicAdd(cells + 1, rows);
}

// Per read position: code + (alpha/beta, delta, zeta, Q) in FP32; with a per-base
// gap-continuation track also (eps_i, beta_i), each rounded from FP64 as the scalar eps and
// beta are (so a uniform track gives the scalar path's parameters exactly).
__global__ void k_prep_reads(const uint8_t *bases, const void *bq, const void *iq,
                             const void *dq, const void *gq, int qual_f32, int alpha_mode,
                             int64_t total, float beta, RowParams *rp, uint8_t *rcode,
                             float2 *rgap) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int c = base_code(bases[g]);
    rcode[g] = (uint8_t)(c < 0 ? kN : c);
    const float b = (float)qual_at(bq, qual_f32, g), i = (float)qual_at(iq, qual_f32, g),
                d = (float)qual_at(dq, qual_f32, g);
    const float Q = exp10f(-b * 0.1f), dl = exp10f(-i * 0.1f), zt = exp10f(-d * 0.1f);
    const float al = alpha_mode ? 1.f - exp10f(-(i + d) * 0.1f) : 1.f - (dl + zt);
    float be = beta;
    if (gq) {
      const double e64 = pow(10.0, -qual_at(gq, qual_f32, g) / 10.0);
      be = (float)(1.0 - e64);
      rgap[g] = make_float2((float)e64, be);
    }
    rp[g] = make_float4(al / be, dl, zt, Q);
  }
}

// One warp per haplotype: codes into hcode[hap_start(h) ...], NULLC up to the 16-byte end,
// and kHapGuard bytes of NULLC before and after (guards of neighbouring haplotypes may
// overlap; both write NULLC there).
__global__ void k_prep_haps(const uint8_t *bases, const int64_t *hap_off, int64_t H,
                            uint8_t *hcode) {
  const int lane = threadIdx.x & 31;
  constexpr int kG = kHapGuard / 16;
  for (int64_t h = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; h < H;
       h += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t o = hap_off[h], n = hap_off[h + 1] - o;
    const int64_t hs = hap_start(o, h);
    const int64_t chunks = (n + 15) >> 4;
    for (int64_t k = lane - kG; k < chunks + kG; k += 32) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int64_t j = k * 16 + q * 4 + b;
          int c = kNull;
          if (j >= 0 && j < n) {
            c = base_code(bases[o + j]);
            if (c < 0) c = kN;
          }
          v |= (uint32_t)c << (8 * b);
        }
        w[q] = v;
      }
      *reinterpret_cast<uint4 *>(hcode + hs + k * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// key = group * kNBuckets + haplotype-length bucket (longest first); histogram per key.
__global__ void k_pair_keys(const int32_t *pr, const int32_t *ph, int64_t P,
                            const int64_t *read_off, const int64_t *hap_off, int64_t R,
                            int64_t H, const CfgTable tab, int32_t *key,
                            int32_t *counts) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = pr[p], h = ph[p];
    int cfg = 0, nb = 0;
    if (r >= 0 && r < R && h >= 0 && h < H) {
      int64_t m = read_off[r + 1] - read_off[r];
      if (m < 0) m = 0;
      if (m > PHMM_MAX_READ_LEN) m = PHMM_MAX_READ_LEN;  // kernel flags it invalid
      cfg = tab.cfg[m];
      nb = nbucket_desc(hap_off[h + 1] - hap_off[h]);
    }
    const int k = cfg * kNBuckets + nb;
    key[p] = k;
    atomicAdd(&counts[k], 1);
  }
}

// Exclusive scan of nkeys counts (one block of 1024 threads); writes offsets and a cursor
// copy, and per-group begin/count.
__global__ void __launch_bounds__(1024) k_scan_keys(const int32_t *counts, int nkeys,
                                                    int32_t *offsets, int32_t *cursor,
                                                    int32_t *grp_begin, int32_t *grp_count) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x;
  const int per = (nkeys + 1023) / 1024;
  int32_t s = 0;
  for (int i = 0; i < per; ++i) {
    const int k = t * per + i;
    if (k < nkeys) s += counts[k];
  }
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int32_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - s;
  for (int i = 0; i < per; ++i) {
    const int k = t * per + i;
    if (k < nkeys) {
      offsets[k] = run;
      cursor[k] = run;
      run += counts[k];
    }
  }
  __syncthreads();
  const int ngrp = nkeys / kNBuckets;
  for (int g = t; g < ngrp; g += 1024) {
    const int32_t b = offsets[g * kNBuckets];
    const int32_t e = (g + 1 < ngrp) ? offsets[(g + 1) * kNBuckets] : part[1023];
    grp_begin[g] = b;
    grp_count[g] = e - b;
  }
}

__global__ void k_scatter(const int32_t *key, int64_t P, int32_t *cursor, int32_t *order) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int pos = atomicAdd(&cursor[key[p]], 1);
    order[pos] = (int32_t)p;
  }
}

// ---------------------------------------------------------------- host launchers ------

static int grid_for(int64_t n, int block, int cap = 152 * 16) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

int launch_validate(const phmm_batch &b, int64_t sum_m, int64_t sum_n, unsigned *err,
                    unsigned long long *cells, cudaStream_t s) {
  if (sum_m > 0)
    k_validate_reads<<<grid_for(sum_m, 256), 256, 0, s>>>(
        b.read_bases, b.base_q, b.ins_q, b.del_q, b.gcp_q, b.qual_dtype == PHMM_QUAL_F32,
        b.alpha_mode, sum_m, err);
  if (sum_n > 0) k_validate_haps<<<grid_for(sum_n, 256), 256, 0, s>>>(b.hap_bases, sum_n, err);
  if (b.n_pairs > 0)
    k_validate_pairs<<<grid_for(b.n_pairs, 256), 256, 0, s>>>(
        b.pair_read, b.pair_hap, b.n_pairs, b.read_off, b.hap_off, b.n_reads, b.n_haps, err,
        cells);
  return (int)cudaGetLastError();
}

int launch_prep(const phmm_batch &b, int64_t sum_m, float beta32, RowParams *rp,
                uint8_t *rcode, uint8_t *hcode, float2 *rgap, cudaStream_t s, int *launches) {
  if (sum_m > 0) {
    k_prep_reads<<<grid_for(sum_m, 256), 256, 0, s>>>(
        b.read_bases, b.base_q, b.ins_q, b.del_q, b.gcp_q, b.qual_dtype == PHMM_QUAL_F32,
        b.alpha_mode, sum_m, beta32, rp, rcode, rgap);
    ++*launches;
  }
  k_prep_haps<<<grid_for(b.n_haps * 32, 256), 256, 0, s>>>(b.hap_bases, b.hap_off, b.n_haps,
                                                           hcode);
  ++*launches;
  return (int)cudaGetLastError();
}

int launch_binning(const phmm_batch &b, const CfgTable &tab, int32_t *key, int32_t *counts,
                   int32_t *offsets, int32_t *cursor, int32_t *grp_begin, int32_t *grp_count,
                   int32_t *order, cudaStream_t s, int *launches) {
  const int nkeys = kNumCfg32 * kNBuckets;
  if (b.n_pairs > 0)
    k_pair_keys<<<grid_for(b.n_pairs, 256), 256, 0, s>>>(b.pair_read, b.pair_hap, b.n_pairs,
                                                         b.read_off, b.hap_off, b.n_reads,
                                                         b.n_haps, tab, key, counts);
  k_scan_keys<<<1, 1024, 0, s>>>(counts, nkeys, offsets, cursor, grp_begin, grp_count);
  if (b.n_pairs > 0)
    k_scatter<<<grid_for(b.n_pairs, 256), 256, 0, s>>>(key, b.n_pairs, cursor, order);
  *launches += b.n_pairs > 0 ? 3 : 1;
  return (int)cudaGetLastError();
}

}  // namespace phmm
