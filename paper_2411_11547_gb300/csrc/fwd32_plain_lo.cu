#include "fwd_inst.cuh"
namespace phmm {
FwdKernel fwd32_plain_lo(int L, int K) {
  if (L == 4) { PHMM_FWD_ROWS_SWITCH(float, 4, false) }
  if (L == 8) { PHMM_FWD_ROWS_SWITCH(float, 8, false) }
  return nullptr;
}
}  // namespace phmm
