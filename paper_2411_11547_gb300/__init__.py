"""GB300 (sm_103a) batched Pair-HMM forward/adjoint (gpuPairHMM, arXiv 2411.11547).

The compute path is libphmm.so (CUDA kernels behind the C ABI of include/phmm.h); `phmm`
is its thin ctypes binding and `autograd` the torch.autograd.Function on top of it.
`synth` draws seeded synthetic workloads.
"""
from . import synth  # noqa: F401
