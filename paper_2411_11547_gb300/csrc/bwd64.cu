#include "bwd_kernel.cuh"
namespace phmm {
BwdKernel bwd64_table(int K) {
  switch (K) {
    case 4: return wf_backward<double, 32, 4>;
    case 8: return wf_backward<double, 32, 8>;
    case 16: return wf_backward<double, 32, 16>;
    default: return nullptr;
  }
}
}  // namespace phmm
