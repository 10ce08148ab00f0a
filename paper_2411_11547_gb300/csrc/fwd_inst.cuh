// Explicit instantiation tables of the forward wavefront, split over translation units so
// the build compiles them in parallel.
#pragma once
#include "wavefront.cuh"

namespace phmm {

using FwdKernel = void (*)(const FwdArgs);

// Table entry for rows-per-lane K (0 if not instantiated).
#define PHMM_FWD_ROWS_SWITCH(T, L, EXT)          \
  switch (K) {                                   \
    case 4: return wf_forward<T, L, 4, EXT>;     \
    case 6: return wf_forward<T, L, 6, EXT>;     \
    case 8: return wf_forward<T, L, 8, EXT>;     \
    case 10: return wf_forward<T, L, 10, EXT>;   \
    case 12: return wf_forward<T, L, 12, EXT>;   \
    case 14: return wf_forward<T, L, 14, EXT>;   \
    case 16: return wf_forward<T, L, 16, EXT>;   \
    case 18: return wf_forward<T, L, 18, EXT>;   \
    case 20: return wf_forward<T, L, 20, EXT>;   \
    default: return nullptr;                     \
  }

FwdKernel fwd32_plain_lo(int L, int K);  // L in {4, 8}
FwdKernel fwd32_plain_hi(int L, int K);  // L in {16, 32}
FwdKernel fwd32_ext_lo(int L, int K);
FwdKernel fwd32_ext_hi(int L, int K);
FwdKernel fwd64_table(int K, bool ext);  // L = 32, K in {4, 8, 16}
// per-base gap-continuation track: extended FP32 groups of the track's table, FP64 tiers
FwdKernel fwd32_gq(int L, int K);
FwdKernel fwd64_gq(int K, bool ext);

}  // namespace phmm
