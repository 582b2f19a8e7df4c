"""fsgpu: fixed-sector fermionic state vectors on one GB300 GPU.

The computation runs in libfsgpu.so (hand-written CUDA for sm_103a, C ABI in
include/fsgpu.h); `fsgpu` is its Python binding and `autograd` wraps the
LUCJ forward/VJP pair as a torch.autograd.Function.  `inputs` holds the
seeded synthetic workloads.  Importing this package loads nothing; the
library is loaded on first use.
"""
