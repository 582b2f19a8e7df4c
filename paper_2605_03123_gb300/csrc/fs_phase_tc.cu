// Diagonal-Coulomb phase with the alpha-beta cross term on the tensor cores
// (complex64 states).
//
// theta(i, j) = A_i + B_j + sum_{p in I_a(i), q in I_b(j)} X[p][q]  (§3.2.2,
// X = -t J_ab).  With Y[p][j] = sum_{q in I_b(j)} X[p][q] (formed in FP64 and
// reduced mod 2 pi), the cross term is the contraction Z = Occ_a Y over the
// orbitals: a (dim_a x N) 0/1 matrix times an (N x dim_b) matrix.  Y is split
// into three bf16 pieces (24 significand bits); occupations are exact in
// bf16, so each tensor-core product is exact and only the FP32 accumulation
// of at most 3N terms rounds.  A_i and B_j arrive as per-string factors.
#include <cuda_bf16.h>

#include <algorithm>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

constexpr int kTcRows = 128, kTcCols = 128;

// Y pieces: ypc[(piece * ncolpad + j) * nk + p], bf16, zero beyond norb and
// beyond dim_b.
__global__ void k_dc_y(__nv_bfloat16* ypc, const uint32_t* mb, int64_t db, int64_t ncolpad,
                       int norb, int nk, const __grid_constant__ Mat X) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= ncolpad) return;
  const uint32_t m = j < db ? mb[j] : 0u;
  for (int p = 0; p < nk; ++p) {
    double y = 0;
    if (p < norb && j < db)
      for (uint32_t b = m; b; b &= b - 1) y += X.v[p * norb + (__ffs(b) - 1)];
    y -= 6.283185307179586 * rint(y * 0.15915494309189535);
    const float yf = (float)y;
    const __nv_bfloat16 hi = __float2bfloat16_rn(yf);
    const float r1 = yf - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    ypc[(0 * ncolpad + j) * nk + p] = hi;
    ypc[(1 * ncolpad + j) * nk + p] = mid;
    ypc[(2 * ncolpad + j) * nk + p] = lo;
  }
}

__device__ __forceinline__ uint32_t occ_pair(uint32_t m, int k) {
  // bf16 1.0 = 0x3F80; two consecutive orbitals k, k+1 of the mask
  return (((m >> k) & 1u) ? 0x3F80u : 0u) | (((m >> (k + 1)) & 1u) ? 0x3F800000u : 0u);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One CTA: a 128 x 128 tile of the state; warp w owns rows 16w .. 16w+15
// and all 16 column groups of 8.
__global__ void __launch_bounds__(256)
    k_phase_tc(float2* vec, int64_t da, int64_t db, const uint32_t* ma, const float2* ea_a,
               const float2* ea_b, const uint32_t* ypc, int64_t ncolpad, int nk) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t i0 = blockIdx.y * (int64_t)kTcRows + 16 * w;
  const int64_t j0 = blockIdx.x * (int64_t)kTcCols;
  const int64_t r0 = i0 + g, r1 = i0 + g + 8;
  const uint32_t m0 = r0 < da ? ma[r0] : 0u, m1 = r1 < da ? ma[r1] : 0u;
  const float2 f0 = r0 < da ? ea_a[r0] : make_float2(0, 0);
  const float2 f1 = r1 < da ? ea_a[r1] : make_float2(0, 0);
  const int nkw = nk >> 1;  // 32-bit words of bf16 pairs per column
#pragma unroll 1
  for (int nt = 0; nt < kTcCols / 8; ++nt) {
    // lane holds rows (g, g+8), columns 2t, 2t+1 of the n-tile; the two
    // columns move as one 16-byte access when the row allows it.  The state
    // and the beta factors are loaded before the contraction so that their
    // latency overlaps it.
    const int64_t jj = j0 + 8 * nt + 2 * t;
    float2 v[2][2], fb[2];
    bool pair[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) fb[c] = jj + c < db ? ea_b[jj + c] : make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = h ? r1 : r0;
      const float2* p = vec + (r < da ? r : 0) * db + jj;
      pair[h] = r < da && jj + 1 < db && ((reinterpret_cast<uintptr_t>(p) & 15u) == 0);
      if (pair[h]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[h][0] = make_float2(q.x, q.y);
        v[h][1] = make_float2(q.z, q.w);
      } else {
#pragma unroll
        for (int c = 0; c < 2; ++c)
          v[h][c] = (r < da && jj + c < db) ? p[c] : make_float2(0.f, 0.f);
      }
    }
    const int64_t jc = j0 + 8 * nt + g;  // column of this lane's B fragment
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kb = 0; kb < nk; kb += 16) {
      const uint32_t a0 = occ_pair(m0, kb + 2 * t), a1 = occ_pair(m1, kb + 2 * t);
      const uint32_t a2 = occ_pair(m0, kb + 2 * t + 8), a3 = occ_pair(m1, kb + 2 * t + 8);
#pragma unroll
      for (int pc = 0; pc < 3; ++pc) {
        const uint32_t* yb = ypc + (pc * ncolpad + jc) * nkw + (kb >> 1);
        mma_bf16(z, a0, a1, a2, a3, __ldg(yb + t), __ldg(yb + t + 4));
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = h ? r1 : r0;
      if (r >= da) continue;
      const float2 fa = h ? f1 : f0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        // z is a sum of at most 3N terms reduced to [-pi, pi]: bring it back
        // to [-pi, pi] (2 pi in two parts) and take the hardware sincos,
        // whose absolute error there is below 1e-6
        const float zz = z[2 * h + c];
        const float kq = rintf(zz * 0.15915494f);
        const float rr = fmaf(kq, 1.7484555e-07f, fmaf(-kq, 6.28318548f, zz));  // 2 pi = hi - 1.75e-7
        float s, co;
        __sincosf(rr, &s, &co);
        const float2 fab = make_float2(fa.x * fb[c].x - fa.y * fb[c].y,
                                       fa.x * fb[c].y + fa.y * fb[c].x);
        const float2 f = make_float2(fab.x * co - fab.y * s, fab.x * s + fab.y * co);
        v[h][c] = make_float2(f.x * v[h][c].x - f.y * v[h][c].y,
                              f.x * v[h][c].y + f.y * v[h][c].x);
      }
      float2* p = vec + r * db + jj;
      if (pair[h]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[h][0].x, v[h][0].y, v[h][1].x, v[h][1].y);
      } else {
#pragma unroll
        for (int c = 0; c < 2; ++c)
          if (jj + c < db) p[c] = v[h][c];
      }
    }
  }
}

bool phase_tc_supported(int dtype, const Space* sa) {
  return dtype == FS_C64 && sa->norb <= 32;
}

void launch_phase_tc(Ctx* ctx, const Space* sa, const Space* sb, void* vec, const PhaseDev& ph,
                     cudaStream_t st) {
  const int nk = sa->norb <= 16 ? 16 : 32;
  const int64_t ncolpad = (sb->dim + kTcCols - 1) / kTcCols * kTcCols;
  __nv_bfloat16* ypc =
      (__nv_bfloat16*)scratch(ctx, "dc_tc_y", 3 * ncolpad * nk * sizeof(__nv_bfloat16));
  ProfScope ps("phase_tc_f32", st, 2);
  k_dc_y<<<(unsigned)((ncolpad + 127) / 128), 128, 0, st>>>(ypc, sb->masks, sb->dim, ncolpad,
                                                            sa->norb, nk, ph.X);
  FS_CUDA(cudaGetLastError());
  dim3 grid((unsigned)(ncolpad / kTcCols), (unsigned)((sa->dim + kTcRows - 1) / kTcRows));
  k_phase_tc<<<grid, 256, 0, st>>>((float2*)vec, sa->dim, sb->dim, sa->masks,
                                   (const float2*)ph.ea_a, (const float2*)ph.ea_b,
                                   (const uint32_t*)ypc, ncolpad, nk);
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
