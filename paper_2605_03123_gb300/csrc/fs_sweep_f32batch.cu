// Complex64 batched sweep kernels (work queue over circuits and slabs),
// compiled apart from fs_sweep.cu so the sweep kernels build in parallel.
#include "fs_sweep_kern.cuh"

namespace fs {
template void launch_batch_t<float, 1, false, 6, 256, false>(const SweepJob*, int, int, int*,
                                                            size_t, int, cudaStream_t);
template void launch_batch_t<float, 1, false, 6, 512, false>(const SweepJob*, int, int, int*,
                                                            size_t, int, cudaStream_t);
template void launch_batch_t<float, 1, false, 6, 256, false, true>(const SweepJob*, int, int, int*,
                                                                  size_t, int, cudaStream_t);
template void launch_batch_t<float, 1, false, 6, 512, false, true>(const SweepJob*, int, int, int*,
                                                                  size_t, int, cudaStream_t);
template void launch_batch_t<float, 2, true, 6, 512, false, true>(const SweepJob*, int, int, int*,
                                                          size_t, int, cudaStream_t);
}  // namespace fs
