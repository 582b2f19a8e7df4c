// FP32-accurate GEMM on the tcgen05 tensor cores, for the dense contractions
// of the library (the minor-matrix rotation, §2.3; the two-body contraction
// of the operator action).
//
//   C[m][n] = sum_k A[m][k] B[n][k],   m < M, n < N, k < K,
//
// with A and B given exactly as three BF16 pieces each (x = x1 + x2 + x3,
// see tc::split_bf16x3), K contiguous (K-major), rows 16-byte aligned.  The
// six products A_i B_j with i + j <= 4 over the pieces are accumulated in
// TMEM (FP32); the dropped products are below 2^-24 of the result.
//
// The kernel is persistent (one CTA per SM, tiles of 128 x 256 of C dealt
// round-robin, consecutive CTAs on the same column panel so the B panel is
// shared in L2) and warp-specialized:
//   * warp 0 (one thread) streams K in chunks of 32 through a three-stage
//     shared-memory ring: per chunk six 2-D TMA loads (A1..A3: 128 x 32,
//     B1..B3: 256 x 32 BF16, 64-byte swizzle, out-of-range rows and k read as
//     zeros) completing on the stage's "full" mbarrier;
//   * warp 1 (one thread) issues the chunk's twelve MMAs (six products x two
//     K steps of 16, 128 x 256 each) into one of two TMEM accumulators
//     (2 x 256 columns) and commits them to the stage's "empty" mbarrier, and
//     after a tile's last chunk to the accumulator's "full" mbarrier;
//   * warps 2..5 (TMEM lanes 32 (w mod 4) ..) drain an accumulator with
//     tcgen05.ld, write it in one of the output forms below, and release it,
//     so the epilogue of one tile overlaps the products of the next.
// Every wait is bounded (status word FS_ERR_TIMEOUT on give-up); the TMEM is
// always freed.
#include <cuda_bf16.h>

#include <algorithm>

#include "fs_common.cuh"
#include "fs_internal.h"
#include "fs_tc.cuh"

namespace fs {
namespace gtc {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 3;
constexpr int THREADS = 192;                 // TMA warp, MMA warp, 4 epilogue warps
constexpr int A_BYTES = BM * BK * 2;         // one BF16 piece of A: 8 KB
constexpr int B_BYTES = BN * BK * 2;         // one BF16 piece of B: 16 KB
constexpr int STAGE_BYTES = 3 * A_BYTES + 3 * B_BYTES;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
// 64-byte swizzle, K-major: rows of BK = 32 BF16 (64 bytes), 8-row atoms of
// 512 bytes; the K step of 16 inside a row advances the start by 32 bytes
constexpr uint32_t SBO = 8 * BK * 2;
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)(SBO >> 4) << 32) |
         (1ull << 46) | (4ull << 61);
}

}  // namespace gtc

struct GemmMaps {
  CUtensorMap a[3], b[3];
};

__global__ void __launch_bounds__(gtc::THREADS, 1)
    k_gemm_tc(const __grid_constant__ GemmMaps maps, const __grid_constant__ GemmTc g,
              int tiles_m, int tiles) {
  using namespace gtc;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) uint64_t s_full[STAGES], s_empty[STAGES], s_accf[2], s_acce[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = (tc::smem_u32(smraw) + 1023u) & ~1023u;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(tc::smem_u32(&s_full[s]), 1);
      tc::mbar_init(tc::smem_u32(&s_empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(tc::smem_u32(&s_accf[a]), 1);
      tc::mbar_init(tc::smem_u32(&s_acce[a]), 4);
    }
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(tc::smem_u32(&s_tmem), 2 * BN);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = s_tmem;
  const int nk = (g.K + BK - 1) / BK;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      int i = 0;  // chunk counter over all tiles of this CTA
      for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int m0 = (t % tiles_m) * BM, n0 = (t / tiles_m) * BN;
        for (int kc = 0; kc < nk; ++kc, ++i) {
          const int s = i % STAGES, u = i / STAGES;
          if (u >= 1 && !tc::mbar_wait(tc::smem_u32(&s_empty[s]), (uint32_t)(u - 1) & 1u))
            ok = false;
          const uint32_t st = sbase + (uint32_t)(s * STAGE_BYTES);
          const uint32_t fb = tc::smem_u32(&s_full[s]);
          tc::mbar_expect_tx(fb, STAGE_BYTES);
#pragma unroll
          for (int p = 0; p < 3; ++p) tc::tma_load_2d(st + p * A_BYTES, &maps.a[p], kc * BK, m0, fb);
#pragma unroll
          for (int p = 0; p < 3; ++p)
            tc::tma_load_2d(st + 3 * A_BYTES + p * B_BYTES, &maps.b[p], kc * BK, n0, fb);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0, j = 0;
      for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
        const int a = j & 1, v = j >> 1;
        if (v >= 1 && !tc::mbar_wait(tc::smem_u32(&s_acce[a]), (uint32_t)(v - 1) & 1u)) ok = false;
        tc::fence_after();
        const uint32_t d = tm + (uint32_t)(a * BN);
        for (int kc = 0; kc < nk; ++kc, ++i) {
          const int s = i % STAGES, u = i / STAGES;
          if (!tc::mbar_wait(tc::smem_u32(&s_full[s]), (uint32_t)u & 1u)) ok = false;
          tc::fence_after();
          const uint32_t st = sbase + (uint32_t)(s * STAGE_BYTES);
          constexpr int kA[6] = {2, 1, 0, 1, 0, 0};
          constexpr int kB[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
          for (int pr = 0; pr < 6; ++pr)
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
              const uint64_t ad = sdesc_sw64(st + kA[pr] * A_BYTES + ks * 32);
              const uint64_t bd = sdesc_sw64(st + 3 * A_BYTES + kB[pr] * B_BYTES + ks * 32);
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                  "l"(ad), "l"(bd), "r"(IDESC), "r"((kc > 0 || pr > 0 || ks > 0) ? 1u : 0u)
                  : "memory");
            }
          tc::mma_commit(tc::smem_u32(&s_empty[s]));
        }
        tc::mma_commit(tc::smem_u32(&s_accf[a]));
      }
    }
  } else {
    // epilogue: this warp's TMEM lane quadrant, all 256 columns of a tile
    const int q = warp & 3;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    int j = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
      const int a = j & 1, v = j >> 1;
      if (!tc::mbar_wait(tc::smem_u32(&s_accf[a]), (uint32_t)v & 1u)) ok = false;
      tc::fence_after();
      const int m0 = (t % tiles_m) * BM, n0 = (t / tiles_m) * BN;
      const int m = m0 + 32 * q + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t vv[2][8];
        tc::tmem_ld8(tm + lanes + (uint32_t)(a * BN + c0), vv[0]);
        tc::tmem_ld8(tm + lanes + (uint32_t)(a * BN + c0 + 8), vv[1]);
        tc::wait_ld();
        if (m >= g.M) continue;
#pragma unroll
        for (int jj = 0; jj < 16; jj += 2) {
          const int n = n0 + c0 + jj;
          const float x0 = __uint_as_float(vv[jj >> 3][jj & 7]);
          const float x1 = __uint_as_float(vv[(jj + 1) >> 3][(jj + 1) & 7]);
          switch (g.mode) {
            case GEMM_REAL:
              if (n < g.N) reinterpret_cast<float*>(g.out)[(int64_t)m * g.ldo + n] = x0;
              if (n + 1 < g.N) reinterpret_cast<float*>(g.out)[(int64_t)m * g.ldo + n + 1] = x1;
              break;
            case GEMM_REAL_T:
              if (n < g.N) reinterpret_cast<float*>(g.out)[(int64_t)n * g.ldo + m] = x0;
              if (n + 1 < g.N)
                reinterpret_cast<float*>(g.out)[(int64_t)(n + 1) * g.ldo + m] = x1;
              break;
            case GEMM_CPLX_T:
              if (n + 1 < g.N)
                reinterpret_cast<float2*>(g.out)[(int64_t)(n >> 1) * g.ldo + m] =
                    make_float2(x0, x1);
              break;
            case GEMM_CPLX_T_PLANES:
              if (n + 1 < g.N) {
                uint32_t p1, p2, p3;
                tc::split_bf16x3(x0, x1, p1, p2, p3);
                const int64_t w = ((int64_t)(n >> 1) * g.ldp + 2 * m) >> 1;
                reinterpret_cast<uint32_t*>(g.outp[0])[w] = p1;
                reinterpret_cast<uint32_t*>(g.outp[1])[w] = p2;
                reinterpret_cast<uint32_t*>(g.outp[2])[w] = p3;
              }
              break;
            default: break;
          }
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tc::smem_u32(&s_acce[a]));
    }
  }
  if (!ok && g.status) atomicCAS(g.status, 0, (int)FS_ERR_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(tm, 2 * BN);
  }
}

// Three BF16 planes of a complex matrix X (rows x cols, leading dimension
// ldx complex elements): plane p, row r, columns 2c, 2c+1 = piece p of
// (Re, Im) X[r][c]; columns 2 cols .. ldk - 1 are zeroed.
__global__ void k_split_planes(const float2* X, int64_t rows, int cols, int64_t ldx,
                               __nv_bfloat16* p1, __nv_bfloat16* p2, __nv_bfloat16* p3,
                               int64_t ldk) {
  const int64_t wpr = ldk / 2;  // 32-bit words per plane row
  const int64_t total = rows * wpr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / wpr, c = i - r * wpr;
    uint32_t a = 0, b = 0, d = 0;
    if (c < cols) {
      const float2 x = X[r * ldx + c];
      tc::split_bf16x3(x.x, x.y, a, b, d);
    }
    reinterpret_cast<uint32_t*>(p1)[i] = a;
    reinterpret_cast<uint32_t*>(p2)[i] = b;
    reinterpret_cast<uint32_t*>(p3)[i] = d;
  }
}

void gemm_tc(const GemmTc& g, cudaStream_t st) {
  FS_REQUIRE(g.M > 0 && g.N > 0 && g.K > 0, FS_ERR_ARG, "empty GEMM");
  FS_REQUIRE(g.lda % 8 == 0 && g.ldb % 8 == 0, FS_ERR_ARG,
             "GEMM operand rows must be 16-byte aligned");
  for (int p = 0; p < 3; ++p)
    FS_REQUIRE(((uintptr_t)g.A[p] & 15) == 0 && ((uintptr_t)g.B[p] & 15) == 0, FS_ERR_ARG,
               "GEMM operand planes must be 16-byte aligned");
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    FS_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 gtc::SMEM));
    int dev = 0;
    FS_CUDA(cudaGetDevice(&dev));
    FS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    attr = true;
  }
  GemmMaps maps;
  for (int p = 0; p < 3; ++p) {
    CUresult r = tc::encode_map_2d(&maps.a[p], CU_TENSOR_MAP_DATA_TYPE_UINT16, (void*)g.A[p],
                                   (uint64_t)g.K, (uint64_t)g.M, (uint64_t)g.lda * 2, gtc::BK,
                                   gtc::BM, CU_TENSOR_MAP_SWIZZLE_64B);
    FS_REQUIRE(r == CUDA_SUCCESS, FS_ERR_CUDA, "cuTensorMapEncodeTiled failed for a GEMM operand");
    r = tc::encode_map_2d(&maps.b[p], CU_TENSOR_MAP_DATA_TYPE_UINT16, (void*)g.B[p],
                          (uint64_t)g.K, (uint64_t)g.N, (uint64_t)g.ldb * 2, gtc::BK, gtc::BN,
                          CU_TENSOR_MAP_SWIZZLE_64B);
    FS_REQUIRE(r == CUDA_SUCCESS, FS_ERR_CUDA, "cuTensorMapEncodeTiled failed for a GEMM operand");
  }
  const int tiles_m = (g.M + gtc::BM - 1) / gtc::BM;
  const int64_t tiles = (int64_t)tiles_m * ((g.N + gtc::BN - 1) / gtc::BN);
  FS_REQUIRE(tiles <= 0x7FFFFFFF, FS_ERR_UNSUPPORTED, "GEMM too large");
  const int grid = (int)std::min<int64_t>(tiles, sms);
  k_gemm_tc<<<grid, gtc::THREADS, gtc::SMEM, st>>>(maps, g, tiles_m, (int)tiles);
  FS_CUDA(cudaGetLastError());
}

void split_planes(const void* X, int64_t rows, int cols, int64_t ldx, void* const planes[3],
                  int64_t ldk, cudaStream_t st) {
  FS_REQUIRE(ldk % 8 == 0 && ldk >= 2 * (int64_t)cols, FS_ERR_ARG, "bad plane stride");
  const int64_t total = rows * (ldk / 2);
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_split_planes<<<grid, 256, 0, st>>>((const float2*)X, rows, cols, ldx,
                                       (__nv_bfloat16*)planes[0], (__nv_bfloat16*)planes[1],
                                       (__nv_bfloat16*)planes[2], ldk);
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
