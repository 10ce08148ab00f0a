#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd32_mid(int L, int K) {
  if (L == 16) {
    if (K == 14) return wf_backward<float, 16, 14>;  // reads up to 224 (autotuner candidate)
    PHMM_BWD_ROWS_SWITCH(float, 16)
  }
  return nullptr;
}
}  // namespace phmm
