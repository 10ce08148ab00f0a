// Forward kernels for batches with a per-base gap-continuation track: the extended-range FP32
// tier in the groups of the track's fixed read-length table, and the FP64 rescue tiers.
#include "fwd_inst.cuh"
namespace phmm {
FwdKernel fwd32_gq(int L, int K) {
  if (L == 16 && K == 4) return wf_forward<float, 16, 4, true, true>;
  if (L == 16 && K == 8) return wf_forward<float, 16, 8, true, true>;
  if (L == 32 && K == 8) return wf_forward<float, 32, 8, true, true>;
  if (L == 32 && K == 12) return wf_forward<float, 32, 12, true, true>;
  if (L == 32 && K == 16) return wf_forward<float, 32, 16, true, true>;
  return nullptr;
}
FwdKernel fwd64_gq(int K, bool ext) {
  switch (K) {
    case 4: return ext ? wf_forward<double, 32, 4, true, true> : wf_forward<double, 32, 4, false, true>;
    case 8: return ext ? wf_forward<double, 32, 8, true, true> : wf_forward<double, 32, 8, false, true>;
    case 16:
      return ext ? wf_forward<double, 32, 16, true, true> : wf_forward<double, 32, 16, false, true>;
    default: return nullptr;
  }
}
}  // namespace phmm
