// Throughput probe of the FP32 fused multiply-add pipe: the denominator of
// the arithmetic roofline of the Givens sweeps, measured on the device the
// library runs on instead of taken from a data sheet.
#include <cuda_runtime.h>

#include "fs_internal.h"

namespace fs {

constexpr int kFmaChains = 8;
constexpr int kFmaIters = 4096;
constexpr int kFmaThreads = 256;

// kFmaChains independent FMA chains per thread, so the pipe, not the
// dependency latency, sets the rate.  The sums are stored so the compiler
// keeps the work.
__global__ void __launch_bounds__(kFmaThreads) k_fma_chains(float* out, float b, float c) {
  float a[kFmaChains];
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) a[i] = threadIdx.x * 1e-7f + i;
  for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace fs

using namespace fs;

extern "C" int fs_measure_fp32_fma(void* stream, double* tflops, double* ms_out) {
  return guarded([&] {
    FS_REQUIRE(tflops != nullptr, FS_ERR_ARG, "null result pointer");
    int dev = 0, sms = 0;
    FS_CUDA(cudaGetDevice(&dev));
    FS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = sms * 8;  // 64 resident warps per SM
    float* out = nullptr;
    FS_CUDA(cudaMallocAsync(&out, (size_t)blocks * kFmaThreads * sizeof(float), st));
    cudaEvent_t e0, e1;
    FS_CUDA(cudaEventCreate(&e0));
    FS_CUDA(cudaEventCreate(&e1));
    for (int w = 0; w < 2; ++w) k_fma_chains<<<blocks, kFmaThreads, 0, st>>>(out, 0.999f, 1e-3f);
    FS_CUDA(cudaGetLastError());
    const int reps = 5;
    FS_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) k_fma_chains<<<blocks, kFmaThreads, 0, st>>>(out, 0.999f, 1e-3f);
    FS_CUDA(cudaEventRecord(e1, st));
    FS_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    FS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    FS_CUDA(cudaEventDestroy(e0));
    FS_CUDA(cudaEventDestroy(e1));
    FS_CUDA(cudaFreeAsync(out, st));
    FS_CUDA(cudaStreamSynchronize(st));
    const double fma = (double)reps * blocks * kFmaThreads * kFmaChains * kFmaIters;
    *tflops = 2.0 * fma / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms / reps;
  });
}
