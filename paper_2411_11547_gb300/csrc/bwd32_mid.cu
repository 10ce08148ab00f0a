#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd32_mid(int L, int K) {
  if (L == 16) { PHMM_BWD_ROWS_SWITCH(float, 16) }
  return nullptr;
}
}  // namespace phmm
