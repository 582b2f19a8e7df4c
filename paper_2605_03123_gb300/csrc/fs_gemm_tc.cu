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
// A CTA computes a 128 x 256 tile of C: K is walked in chunks of 32, each
// chunk's six piece-tiles (A1..A3: 8 KB each, B1..B3: 16 KB each) copied by
// cp.async into a three-stage shared-memory ring in the K-major no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix, LBO = 128 B along
// K, SBO = 512 B between 8-row groups); one thread issues the 12 MMAs of a
// chunk (128 x 256 x 16 each) and commits them to the stage's mbarrier,
// which frees the stage for the chunk two ahead.  The epilogue reads the
// tile from TMEM (warp w: lanes 32 (w mod 4), columns 128 (w / 4) ..) and
// writes it in one of the output forms below.  Waits are bounded (status
// word FS_ERR_TIMEOUT on give-up); the TMEM is always freed.
#include <cuda_bf16.h>

#include <algorithm>

#include "fs_common.cuh"
#include "fs_internal.h"
#include "fs_tc.cuh"

namespace fs {
namespace gtc {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 3, THREADS = 256;
constexpr int A_BYTES = BM * BK * 2;         // one BF16 piece of A: 8 KB
constexpr int B_BYTES = BN * BK * 2;         // one BF16 piece of B: 16 KB
constexpr int STAGE_BYTES = 3 * A_BYTES + 3 * B_BYTES;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
constexpr uint32_t SBO = (BK / 8) * 128;
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr int A_CHUNKS = BM * BK / 8, B_CHUNKS = BN * BK / 8;  // 16-byte copies per piece

}  // namespace gtc

__global__ void __launch_bounds__(gtc::THREADS, 1) k_gemm_tc(const __grid_constant__ GemmTc g) {
  using namespace gtc;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) uint64_t s_mbar[STAGES];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const uint32_t sraw = tc::smem_u32(smraw);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) tc::mbar_init(tc::smem_u32(&s_mbar[s]), 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&s_tmem), BN);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = s_tmem;
  const int nk = (g.K + BK - 1) / BK;

  // chunk kc of all six pieces into stage s (rows past M / N and k past K
  // read as zeros)
  auto load = [&](int kc, int s) {
    const uint32_t st = sbase + (uint32_t)(s * STAGE_BYTES);
    const int k0 = kc * BK;
    for (int c = tid; c < 3 * (A_CHUNKS + B_CHUNKS); c += THREADS) {
      const bool isA = c < 3 * A_CHUNKS;
      const int cb = isA ? c : c - 3 * A_CHUNKS;
      const int piece = isA ? cb / A_CHUNKS : cb / B_CHUNKS;
      const int cc = isA ? cb - piece * A_CHUNKS : cb - piece * B_CHUNKS;
      const int r = ((cc >> 5) << 3) | (cc & 7), kq = (cc >> 3) & 3;
      const int row = (isA ? m0 : n0) + r;
      const uint16_t* src = isA ? g.A[piece] : g.B[piece];
      const int64_t ld = isA ? g.lda : g.ldb;
      const int kk = k0 + kq * 8;
      int bytes = 0;
      if (row < (isA ? g.M : g.N) && kk < g.K) bytes = min(8, g.K - kk) * 2;
      const uint16_t* gp = bytes ? src + (int64_t)row * ld + kk : src;
      const uint32_t base = isA ? (uint32_t)(piece * A_BYTES)
                                : (uint32_t)(3 * A_BYTES + piece * B_BYTES);
      const uint32_t dst = st + base + (uint32_t)((r >> 3) * SBO) +
                           (uint32_t)(kq * 128 + (r & 7) * 16);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(gp),
                   "r"(bytes)
                   : "memory");
    }
  };
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nk) load(s, s);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc % STAGES;
    asm volatile("cp.async.wait_group %0;" ::"n"(STAGES - 2) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t st = sbase + (uint32_t)(s * STAGE_BYTES);
      constexpr int kA[6] = {2, 1, 0, 1, 0, 0};
      constexpr int kB[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
      for (int pr = 0; pr < 6; ++pr)
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint64_t ad = tc::sdesc(st + kA[pr] * A_BYTES + ks * 256, 128, SBO);
          const uint64_t bd = tc::sdesc(st + 3 * A_BYTES + kB[pr] * B_BYTES + ks * 256, 128, SBO);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tm),
              "l"(ad), "l"(bd), "r"(IDESC), "r"((kc > 0 || pr > 0 || ks > 0) ? 1u : 0u)
              : "memory");
        }
      tc::mma_commit(tc::smem_u32(&s_mbar[s]));
    }
    // chunk kc + STAGES - 1 refills the stage of chunk kc - 1 once its
    // products are done
    const int kn = kc + STAGES - 1;
    if (kn < nk) {
      const int sn = kn % STAGES;
      if (kc >= 1 &&
          !tc::mbar_wait(tc::smem_u32(&s_mbar[sn]), (uint32_t)((kc - 1) / STAGES) & 1u) &&
          g.status)
        atomicCAS(g.status, 0, (int)FS_ERR_TIMEOUT);
      load(kn, sn);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (nk > 0 && !tc::mbar_wait(tc::smem_u32(&s_mbar[(nk - 1) % STAGES]),
                               (uint32_t)((nk - 1) / STAGES) & 1u) &&
      g.status)
    atomicCAS(g.status, 0, (int)FS_ERR_TIMEOUT);
  tc::fence_after();

  // epilogue: warp w reads lanes 32 (w mod 4) .. and columns 128 (w / 4) ..
  const int q = warp & 3, h = warp >> 2;
  const int m = m0 + 32 * q + lane;
  const uint32_t lanes = (uint32_t)(32 * q) << 16;
#pragma unroll 1
  for (int c0 = 0; c0 < BN / 2; c0 += 16) {
    uint32_t v[2][8];
    tc::tmem_ld8(tm + lanes + (uint32_t)(BN / 2 * h + c0), v[0]);
    tc::tmem_ld8(tm + lanes + (uint32_t)(BN / 2 * h + c0 + 8), v[1]);
    tc::wait_ld();
    if (m >= g.M || nk == 0) continue;
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
      const int n = n0 + BN / 2 * h + c0 + j;
      const float x0 = __uint_as_float(v[j >> 3][j & 7]);
      const float x1 = __uint_as_float(v[(j + 1) >> 3][(j + 1) & 7]);
      switch (g.mode) {
        case GEMM_REAL:
          if (n < g.N) reinterpret_cast<float*>(g.out)[(int64_t)m * g.ldo + n] = x0;
          if (n + 1 < g.N) reinterpret_cast<float*>(g.out)[(int64_t)m * g.ldo + n + 1] = x1;
          break;
        case GEMM_REAL_T:
          if (n < g.N) reinterpret_cast<float*>(g.out)[(int64_t)n * g.ldo + m] = x0;
          if (n + 1 < g.N) reinterpret_cast<float*>(g.out)[(int64_t)(n + 1) * g.ldo + m] = x1;
          break;
        case GEMM_CPLX_T:
          if (n + 1 < g.N)
            reinterpret_cast<float2*>(g.out)[(int64_t)(n >> 1) * g.ldo + m] = make_float2(x0, x1);
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
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tm, BN);
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
  static bool attr = false;
  if (!attr) {
    FS_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 gtc::SMEM));
    attr = true;
  }
  dim3 grid((unsigned)((g.N + gtc::BN - 1) / gtc::BN), (unsigned)((g.M + gtc::BM - 1) / gtc::BM));
  k_gemm_tc<<<grid, gtc::THREADS, gtc::SMEM, st>>>(g);
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
