#include "fwd_inst.cuh"
namespace phmm {
FwdKernel fwd32_ext_hi(int L, int K) {
  if (L == 16) { PHMM_FWD_ROWS_SWITCH(float, 16, true) }
  if (L == 32) { PHMM_FWD_ROWS_SWITCH(float, 32, true) }
  return nullptr;
}
}  // namespace phmm
