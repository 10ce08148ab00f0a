// Forward scoring without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another component owns every
// device allocation (a framework's caching pool, an inference server that forbids
// allocation on its request path), callers that may not take the implicit device-wide
// synchronisation cudaMalloc/cudaFree can cause, and plugins that are handed only input
// and output buffers.  phmm_forward_noalloc serves them: it runs the same preparation and
// FP32 wavefront kernels as phmm_forward, with their scratch (row parameters, base codes,
// padded haplotype codes) in one statically sized device array instead of a workspace.
#include <cuda_runtime.h>
#include <cstring>
#include <mutex>
#include "phmm_internal.cuh"
#include "wavefront.cuh"

namespace phmm {
int launch_prep(const phmm_batch &b, int64_t sum_m, float beta32, RowParams *rp,
                uint8_t *rcode, uint8_t *hcode, float2 *rgap, cudaStream_t s, int *launches);
int launch_fwd32(int cfg, bool ext, int grid, int block, cudaStream_t s, const FwdArgs &a);
}  // namespace phmm

using namespace phmm;

// The scratch every call shares (one copy per device that loads the library, held until the
// process exits).
static __device__ __align__(256) unsigned char g_noalloc_scratch[PHMM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

// Header at the start of the scratch: the longest read and an error word, written by
// k_check_offsets.
struct Header {
  int32_t max_m;
  uint32_t err;  // nonzero: the offsets are not non-decreasing from 0 with non-empty entries
  int32_t pad[62];
};

// Offset checks (the planned entry points make them on the host after copying the offsets;
// here the offsets stay on the device): read_off[0] == hap_off[0] == 0, every read and
// haplotype non-empty, haplotypes at most INT32_MAX / 2 long; and the longest read.  Bad
// offsets would otherwise let the preparation kernels write past the scratch they were
// sized for.
__global__ void k_check_offsets(const int64_t *read_off, int64_t R, const int64_t *hap_off,
                                int64_t H, Header *h) {
  int32_t mx = 0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid == 0) bad = read_off[0] != 0 || hap_off[0] != 0;
  for (int64_t r = tid; r < R; r += stride) {
    const int64_t m = read_off[r + 1] - read_off[r];
    if (m <= 0) bad = true;
    const int32_t v = m < 0 ? 0 : (m > 1 << 30 ? 1 << 30 : (int32_t)m);
    mx = v > mx ? v : mx;
  }
  for (int64_t k = tid; k < H; k += stride) {
    const int64_t n = hap_off[k + 1] - hap_off[k];
    if (n <= 0 || n > INT32_MAX / 2) bad = true;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const int32_t y = __shfl_down_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&h->max_m, mx);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&h->err, 1u);
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int phmm_forward_noalloc(const phmm_batch *batch, double *out_log10,
                                    uint8_t *out_flags, void *stream) {
  if (!batch) return PHMM_EINVAL;
  const phmm_batch &b = *batch;
  if (b.n_reads < 1 || b.n_haps < 1 || b.n_pairs < 0) return PHMM_EINVAL;
  if (b.n_reads > INT32_MAX || b.n_haps > INT32_MAX || b.n_pairs > INT32_MAX) return PHMM_EINVAL;
  if (!b.read_bases || !b.base_q || !b.ins_q || !b.del_q || !b.read_off || !b.hap_bases ||
      !b.hap_off)
    return PHMM_EINVAL;
  if (b.n_pairs > 0 && (!b.pair_read || !b.pair_hap || !out_log10 || !out_flags))
    return PHMM_EINVAL;
  if (b.qual_dtype != PHMM_QUAL_U8 && b.qual_dtype != PHMM_QUAL_F32) return PHMM_EINVAL;
  if (b.alpha_mode != 0 && b.alpha_mode != 1) return PHMM_EINVAL;
  if (!(b.gcp > 0.0) || !(b.gcp < 1e300)) return PHMM_EINVAL;
  if (b.gcp_q) return PHMM_EINVAL;  // scalar gap continuation only
  cudaStream_t s = (cudaStream_t)stream;

  // set-up, once per device: the device address of the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PHMM_ECUDA;
  unsigned char *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PHMM_ECUDA;
      g_addr[dev] = (unsigned char *)p;
    }
    scratch = g_addr[dev];
  }

  // sizes: total read and haplotype bases, the longest read and the offset checks (one wait
  // on `stream`)
  Header *hdr = (Header *)scratch;
  int64_t sum_m = 0, sum_n = 0;
  int32_t hh[2] = {0, 0};  // max_m, err
  if (cudaMemsetAsync(hdr, 0, sizeof(Header), s) != cudaSuccess) return PHMM_ECUDA;
  k_check_offsets<<<64, 256, 0, s>>>(b.read_off, b.n_reads, b.hap_off, b.n_haps, hdr);
  if (cudaGetLastError() != cudaSuccess) return PHMM_ECUDA;
  if (cudaMemcpyAsync(&sum_m, b.read_off + b.n_reads, 8, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(&sum_n, b.hap_off + b.n_haps, 8, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(hh, hdr, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PHMM_ECUDA;
  const int32_t max_m = hh[0];
  if (hh[1] != 0) return PHMM_EINVAL;
  if (sum_m <= 0 || sum_n <= 0 || max_m <= 0) return PHMM_EINVAL;
  if (max_m > PHMM_MAX_READ_LEN) return PHMM_ETOOLONG;

  // carve the scratch; reject batches that do not fit
  const size_t o_rp = up256(sizeof(Header));
  const size_t o_rcode = up256(o_rp + sizeof(RowParams) * (size_t)sum_m);
  const size_t o_hcode = up256(o_rcode + (size_t)sum_m);
  const size_t end = o_hcode + (size_t)hap_code_bytes(sum_n, b.n_haps);
  if (end > (size_t)PHMM_NOALLOC_SCRATCH_BYTES) return PHMM_ENOMEM;
  RowParams *rp = (RowParams *)(scratch + o_rp);
  uint8_t *rcode = scratch + o_rcode, *hcode = scratch + o_hcode;

  const double eps64 = pow(10.0, -b.gcp / 10.0);
  int launches = 0;
  if (launch_prep(b, sum_m, (float)(1.0 - eps64), rp, rcode, hcode, nullptr, s, &launches) != 0)
    return PHMM_ECUDA;
  if (b.n_pairs == 0) return PHMM_OK;

  // one lanes x rows group for the whole batch: the fewest lanes holding the longest read
  int li = 0;
  while ((4 << li) * 20 < max_m) ++li;
  const int L = 4 << li;
  int K = (max_m + L - 1) / L;
  K = K < 4 ? 4 : (K + 1) / 2 * 2;
  const int cfg = cfg_index(L, K);

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
  a.qual_f32 = b.qual_dtype == PHMM_QUAL_F32;
  a.alpha_mode = b.alpha_mode;
  a.n_reads = b.n_reads;
  a.n_haps = b.n_haps;
  a.count = b.n_pairs;
  a.out = out_log10;
  a.flags = out_flags;
  a.eps32 = (float)eps64;
  a.beta32 = (float)(1.0 - eps64);
  a.eps64 = eps64;
  a.beta64 = 1.0 - eps64;
  a.mode = 1;
  a.rescue = 0;
  a.persistent = 0;
  const int G = 32 / L, wpb = 4;
  const int64_t items = (b.n_pairs + G - 1) / G;
  const int grid = (int)((items + wpb - 1) / wpb);
  if (launch_fwd32(cfg, true, grid, 32 * wpb, s, a) != 0) return PHMM_ECUDA;
  return PHMM_OK;
}
