#include "fwd_inst.cuh"
namespace phmm {
FwdKernel fwd32_plain_hi(int L, int K) {
  if (L == 16) { PHMM_FWD_ROWS_SWITCH(float, 16, false) }
  if (L == 32) { PHMM_FWD_ROWS_SWITCH(float, 32, false) }
  return nullptr;
}
}  // namespace phmm
