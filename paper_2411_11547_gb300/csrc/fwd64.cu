#include "fwd_inst.cuh"
namespace phmm {
FwdKernel fwd64_table(int K, bool ext) {
  switch (K) {
    case 4: return ext ? wf_forward<double, 32, 4, true> : wf_forward<double, 32, 4, false>;
    case 8: return ext ? wf_forward<double, 32, 8, true> : wf_forward<double, 32, 8, false>;
    case 16: return ext ? wf_forward<double, 32, 16, true> : wf_forward<double, 32, 16, false>;
    default: return nullptr;
  }
}
}  // namespace phmm
