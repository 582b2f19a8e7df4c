// Complex64 forward window sweeps (one state, W = 6, 256 and 512 threads;
// one vector, or packed vector pairs),
// compiled apart from fs_sweep.cu so the sweep kernels build in parallel.
#include "fs_sweep_kern.cuh"

namespace fs {
template void dispatch_cs<float, 1, false, 6, 256, WProg<float>, false>(
    int, const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
template void dispatch_cs<float, 1, false, 6, 512, WProg<float>, false>(
    int, const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
template void launch_sweep_t<float, 1, 1, false, 6, 256, false, WProg<float>, false, true>(
    const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
template void launch_sweep_t<float, 1, 1, false, 6, 512, false, WProg<float>, false, true>(
    const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
}  // namespace fs
