#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd32_lo(int L, int K) {
  if (L == 4) { PHMM_BWD_ROWS_SWITCH(float, 4) }
  if (L == 8) { PHMM_BWD_ROWS_SWITCH(float, 8) }
  return nullptr;
}
}  // namespace phmm
