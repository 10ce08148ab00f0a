// Adjoint kernels for batches with a per-base gap-continuation track (the groups of the
// track's fixed read-length table, and the FP64 hand-off groups).
#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd32_gq(int L, int K) {
  if (L == 16 && K == 4) return wf_backward<float, 16, 4, true>;
  if (L == 16 && K == 8) return wf_backward<float, 16, 8, true>;
  if (L == 32 && K == 8) return wf_backward<float, 32, 8, true>;
  if (L == 32 && K == 12) return wf_backward<float, 32, 12, true>;
  if (L == 32 && K == 16) return wf_backward<float, 32, 16, true>;
  return nullptr;
}
BwdKernel bwd64_gq(int K) {
  switch (K) {
    case 4: return wf_backward<double, 32, 4, true>;
    case 8: return wf_backward<double, 32, 8, true>;
    case 16: return wf_backward<double, 32, 16, true>;
    default: return nullptr;
  }
}
}  // namespace phmm
