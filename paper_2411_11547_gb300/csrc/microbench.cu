// Arithmetic-pipe peak probes: the roofline denominators for the Pair-HMM kernels.
//
// The Pair-HMM recurrences (Eq. 1-3) are plain FP32 multiply/add work, so the bound that
// matters is the FP32 pipe, not HBM and not the tensor cores.  These probes measure, on the
// GPU at hand, how many FP32 (scalar FFMA and packed fma.rn.f32x2) and FP64 (DFMA) lane
// operations per second one kernel can sustain.  Each thread runs NCHAIN independent
// dependency chains so that issue, not latency, is the limit.
//
// One lane operation = one multiply-add on one value (an f32x2 instruction counts as two).

#include <cuda_runtime.h>
#include <cstdint>
#include "phmm_internal.cuh"

namespace {

constexpr int NCHAIN = 8;

__global__ void __launch_bounds__(256) probe_ffma(float* out, int iters) {
  float a[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) a[c] = 1e-3f * (threadIdx.x + c);
  const float b = 0.9999f, d = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < NCHAIN; ++c) a[c] = fmaf(a[c], b, d);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) probe_ffma2(float* out, int iters) {
  unsigned long long a[NCHAIN], b, d;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) {
    float x = 1e-3f * (threadIdx.x + c);
    asm volatile("mov.b64 %0, {%1,%2};" : "=l"(a[c]) : "f"(x), "f"(x + 0.5f));
  }
  asm volatile("mov.b64 %0, {%1,%2};" : "=l"(b) : "f"(0.9999f), "f"(0.9998f));
  asm volatile("mov.b64 %0, {%1,%2};" : "=l"(d) : "f"(1e-7f), "f"(2e-7f));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < NCHAIN; ++c)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[c]) : "l"(b), "l"(d));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) {
    float lo, hi;
    asm volatile("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[c]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) probe_dfma(float* out, int iters) {
  double a[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) a[c] = 1e-3 * (threadIdx.x + c);
  const double b = 0.9999, d = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < NCHAIN; ++c) a[c] = fma(a[c], b, d);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

}  // namespace

// kind: 0 = scalar FFMA, 1 = packed FFMA2 (fma.rn.f32x2), 2 = DFMA.
extern "C" int phmm_probe_pipe(int kind, int iters, double* lane_ops_per_s, double* ms_out) {
  if (!lane_ops_per_s || iters <= 0 || kind < 0 || kind > 2) return PHMM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PHMM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PHMM_ECUDA;
  const int threads = 256, blocks = sms * 8;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * threads * blocks) != cudaSuccess) return PHMM_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int it) {
    if (kind == 0) probe_ffma<<<blocks, threads>>>(out, it);
    else if (kind == 1) probe_ffma2<<<blocks, threads>>>(out, it);
    else probe_dfma<<<blocks, threads>>>(out, it);
  };
  launch(iters / 10 + 1);  // warm-up: clocks ramp, module loads
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return PHMM_ECUDA;
  const double per_thread = (double)iters * 16 * NCHAIN * (kind == 1 ? 2 : 1);
  *lane_ops_per_s = per_thread * threads * blocks / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return PHMM_OK;
}
