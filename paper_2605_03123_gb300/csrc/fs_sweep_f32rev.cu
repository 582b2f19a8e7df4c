// Complex64 reverse window sweeps (two states per thread: packed, W = 6 in
// one CTA; W = 5 in clusters), compiled apart from fs_sweep.cu so the sweep
// kernels build in parallel.
#include "fs_sweep_kern.cuh"

namespace fs {
template void launch_sweep_t<float, 1, 2, true, 6, 512, false, WProg<float>, false, true>(
    const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
template void dispatch_cs<float, 2, true, 5, 512, WProg<float>, false>(
    int, const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
}  // namespace fs
