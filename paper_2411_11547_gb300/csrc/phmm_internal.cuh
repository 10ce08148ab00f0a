// Internal definitions shared by the CUDA translation units of libphmm.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "phmm.h"

namespace phmm {

// Base codes.  A C G T N as 0..4; NULLC marks a column outside 1..n of a haplotype (columns
// before the wavefront reaches a lane and after the haplotype ends): its emission is 0, so
// M and I stay exactly 0 there and the last-row sum needs no guard.
constexpr int kA = 0, kN = 4, kNull = 5, kCodes = 6;

// Initial constants (powers of two, so scaling is exact): the row-0 boundary is K0/n.
constexpr float kK32 = 1.329227995784916e36f;              // 2^120
constexpr double kK64 = 1.1235582092889474e307;            // 2^1020
constexpr float kMinAccepted32 = 1e-28f;                   // scaled FP32 sum below: rescue
constexpr double kMinAccepted64 = 1e-290;                  // scaled FP64 sum below: extended

// Fixed-function FP32 wavefront groups: lanes per pair x rows per lane.
// cfg = li * 17 + (rows - 4) with lanes 4 << li (4, 8, 16, 32) and rows 4 .. 20.  The forward
// kernels are built for even rows; the adjoint also for some odd ones (a closer fit of the
// read length).  Group tables of the options hold these indices.
constexpr int kRowsPerLanes = 17;
constexpr int kNumCfg32 = 4 * kRowsPerLanes;
__host__ __device__ constexpr int cfg_lanes(int cfg) { return 4 << (cfg / kRowsPerLanes); }
__host__ __device__ constexpr int cfg_rows(int cfg) { return 4 + cfg % kRowsPerLanes; }
__host__ __device__ constexpr int cfg_index(int L, int K) {
  return (L == 4 ? 0 : L == 8 ? 1 : L == 16 ? 2 : 3) * kRowsPerLanes + (K - 4);
}

// FP64 rescue groups: 32 lanes x {4, 8, 16} rows (reads up to 128 / 256 / 512).
constexpr int kNumCfg64 = 3;
__host__ __device__ constexpr int rows64(int c) { return c == 0 ? 4 : (c == 1 ? 8 : 16); }
__host__ __device__ inline int bin64_of_m(int m) { return m <= 128 ? 0 : (m <= 256 ? 1 : 2); }

// n-bucket keys for sorting pairs inside a bin by haplotype length, longest first.
constexpr int kNBuckets = 256;
__host__ __device__ inline int nbucket_desc(int64_t n) {
  int64_t b = n < 512 ? n / 8 : 64 + (n - 512) / 16;
  if (b > kNBuckets - 1) b = kNBuckets - 1;
  return kNBuckets - 1 - (int)b;
}

// Read length -> FP32 wavefront group, passed to the binning kernel by value.
struct CfgTable {
  int8_t cfg[PHMM_MAX_READ_LEN + 1];
};

// Per-read-position FP32 parameters written by the prep kernel.
//   x = alpha/beta, y = delta, z = zeta, w = Q
using RowParams = float4;

struct FwdArgs {
  const int32_t *pair_read, *pair_hap;
  const int64_t *read_off, *hap_off;
  const RowParams *rp;      // FP32 path parameters per read position
  const uint8_t *rcode;     // read base codes per read position
  const uint8_t *hcode;     // haplotype codes, each haplotype 16-byte aligned, NULLC padded
  const void *bq, *iq, *dq; // raw Phred inputs (FP64 path derives its own parameters)
  const void *gq;           // raw per-base gap-continuation Phred values, or null
  const float2 *rgap;       // FP32 (eps_i, beta_i) per read position (plans with a track)
  int32_t qual_f32, alpha_mode;
  int64_t n_reads, n_haps;
  const int32_t *list;      // pair ids to process (nullptr: identity 0..count-1)
  const int32_t *count_dev; // device-side item count (nullptr: use count)
  int64_t count;
  int64_t list_offset;      // start of this bin inside `list` (device count case: from dev)
  const int32_t *offset_dev;
  int32_t *counter;         // persistent work counter (zeroed before the launch)
  int32_t persistent;
  double *out;
  uint8_t *flags;
  int32_t *rescue_list[kNumCfg64];  // append targets for the next precision tier
  int32_t *rescue_count;            // [kNumCfg64]
  float eps32, beta32;
  double eps64, beta64;
  int32_t mode;             // 0 plain32, 1 ext32, 2 plain64, 3 ext64
  int32_t rescue;           // 1: append failures to rescue lists, 0: write whatever results
  void *tilebuf;            // row tiles: 2 x tile_cols TileCol<T> per resident warp (or null)
  int64_t tile_cols;        // columns per tile buffer (the longest haplotype)
  // debug builds (PHMM_DEBUG): the sizes the kernels check their indexes against, and the
  // word they report a failed check in (null: no checks)
  unsigned *dbg_err;
  int64_t dbg_sum_m, dbg_hcode_bytes, dbg_nslots;
};

// Bits of the debug word (PHMM_DEBUG builds).
constexpr unsigned kDbgGuard = 1u, kDbgPairIndex = 4u, kDbgSlot = 8u, kDbgCheckpoints = 16u;

// Host-side NVTX range over a library call (profilers show the calls on their timelines;
// the markers cost nothing without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char *name);
  ~NvtxRange();
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Launchers (one per precision); return cudaError_t of the launch.
int launch_fwd32(int cfg, bool ext, int grid, int block, cudaStream_t s, const FwdArgs &a);
int launch_fwd64(int cfg64, bool ext, int grid, int block, cudaStream_t s, const FwdArgs &a);
size_t fwd32_smem(int cfg, int block);
size_t fwd64_smem(int cfg64, int block);
int fwd32_blocks_per_sm(int cfg, bool ext, int block, bool gq = false);
int fwd64_blocks_per_sm(int cfg64, bool ext, int block, bool gq = false);

// Read length -> group of a plan with a per-base gap-continuation track (the kernels with
// per-row gap continuation are built for these groups only).
__host__ __device__ constexpr int gq_cfg_of_m(int m) {
  return m <= 64 ? cfg_index(16, 4)
                 : (m <= 128 ? cfg_index(16, 8)
                             : (m <= 256 ? cfg_index(32, 8)
                                         : (m <= 384 ? cfg_index(32, 12) : cfg_index(32, 16))));
}

}  // namespace phmm
