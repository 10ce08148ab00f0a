#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd32_hi(int L, int K) {
  if (L == 32) {
    if (K == 16) return wf_backward<float, 32, 16>;
    PHMM_BWD_ROWS_SWITCH(float, 32)
  }
  return nullptr;
}
}  // namespace phmm
