#include "fwd_inst.cuh"
namespace phmm {
FwdKernel fwd32_ext_lo(int L, int K) {
  if (L == 4) { PHMM_FWD_ROWS_SWITCH(float, 4, true) }
  if (L == 8) { PHMM_FWD_ROWS_SWITCH(float, 8, true) }
  return nullptr;
}
}  // namespace phmm
