#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd32_odd_lo(int L, int K) {
  if (L == 4 && K == 9) return wf_backward<float, 4, 9>;
  if (L == 4 && K == 11) return wf_backward<float, 4, 11>;
  if (L == 8 && K == 7) return wf_backward<float, 8, 7>;
  if (L == 8 && K == 9) return wf_backward<float, 8, 9>;
  if (L == 8 && K == 11) return wf_backward<float, 8, 11>;
  return nullptr;
}
}  // namespace phmm
