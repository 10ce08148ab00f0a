#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd32_odd_hi(int L, int K) {
  if (L == 16 && K == 7) return wf_backward<float, 16, 7>;
  if (L == 16 && K == 9) return wf_backward<float, 16, 9>;
  if (L == 16 && K == 11) return wf_backward<float, 16, 11>;
  if (L == 16 && K == 13) return wf_backward<float, 16, 13>;
  if (L == 32 && K == 7) return wf_backward<float, 32, 7>;
  if (L == 32 && K == 9) return wf_backward<float, 32, 9>;
  return nullptr;
}
}  // namespace phmm
