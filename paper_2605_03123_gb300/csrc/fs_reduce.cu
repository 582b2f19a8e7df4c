// Gradient of a diagonal-Coulomb gate with respect to its coupling matrices.
//
// For D = exp(i theta) with theta = -1/2 [occ_a^T J_aa occ_a + occ_b^T J_aa
// occ_b + 2 occ_a^T J_ab occ_b] (§3.2.2, spin-balanced, t = 1) and a loss
// L = Re <g, D psi>, dL/dtheta_ij = -W_ij with W = Im(conj(g) D psi), so
//   dL/dJ_ab = Occ_a^T W Occ_b,
//   dL/dJ_aa = 1/2 (Occ_a^T diag(W 1) Occ_a + Occ_b^T diag(W^T 1) Occ_b).
// W is written by the reverse-mode sweep; these kernels reduce it.
#include <algorithm>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

constexpr int kRThreads = 256;

// Rows: V_i[q] = sum_j W_ij occ_b(j)_q and r_i = sum_j W_ij; then
// dJ_ab[p][q] += occ_a(i)_p V_i[q] and dJ_aa[p][q] += 1/2 r_i occ_a(i)_p occ_a(i)_q,
// accumulated per CTA in shared memory and flushed once.
// Per-thread partial sums and the warp sums run in the precision of W (FP32
// for complex64 states, where FP64 arithmetic would be 1/64-rate); the block
// reduction and the accumulators are FP64.
template <typename R, int NQ>
__global__ void __launch_bounds__(kRThreads)
    k_dc_rows(const R* W, int64_t da, int64_t db, const uint32_t* ma, const uint32_t* mb,
              int norb, double* dJaa, double* dJab) {
  __shared__ double sab[kMaxOrb * kMaxOrb], saa[kMaxOrb * kMaxOrb];
  __shared__ double red[kRThreads / 32][NQ + 1];
  for (int k = threadIdx.x; k < norb * norb; k += kRThreads) sab[k] = saa[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t i = blockIdx.x; i < da; i += gridDim.x) {
    R pacc[NQ];
    R pr = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) pacc[q] = 0;
    const R* row = W + i * db;
    // eight independent loads in flight per thread before the sums
    constexpr int U = 8;
    for (int64_t j0 = threadIdx.x; j0 < db; j0 += U * kRThreads) {
      R w[U];
      uint32_t m[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = j0 + (int64_t)u * kRThreads;
        w[u] = j < db ? row[j] : (R)0;
        m[u] = j < db ? __ldg(mb + j) : 0u;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        pr += w[u];
#pragma unroll
        for (int q = 0; q < NQ; ++q) pacc[q] += ((m[u] >> q) & 1u) ? w[u] : (R)0;
      }
    }
    // warp sums in the precision of W (the FP64 shuffles of 17 values per
    // row would cost more than reading the row on GB300), FP64 from here on
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      pr += __shfl_xor_sync(0xFFFFFFFFu, pr, off);
#pragma unroll
      for (int q = 0; q < NQ; ++q) pacc[q] += __shfl_xor_sync(0xFFFFFFFFu, pacc[q], off);
    }
    if (lane == 0) {
      red[wid][NQ] = (double)pr;
#pragma unroll
      for (int q = 0; q < NQ; ++q) red[wid][q] = (double)pacc[q];
    }
    __syncthreads();
    if (threadIdx.x < norb + 1) {
      double s = 0;
      const int q = threadIdx.x < norb ? threadIdx.x : NQ;
      for (int k = 0; k < kRThreads / 32; ++k) s += red[k][q];
      red[0][q] = s;  // safe: each q column is owned by one thread
    }
    __syncthreads();
    uint32_t mi = ma[i];
    const double ri = red[0][NQ];
    for (int k = threadIdx.x; k < norb * norb; k += kRThreads) {
      int p = k / norb, q = k - p * norb;
      if ((mi >> p) & 1u) {
        sab[k] += red[0][q];
        if ((mi >> q) & 1u) saa[k] += 0.5 * ri;
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < norb * norb; k += kRThreads) {
    if (sab[k] != 0) atomicAdd(dJab + k, sab[k]);
    if (saa[k] != 0) atomicAdd(dJaa + k, saa[k]);
  }
}

// Columns: c_j = sum_i W_ij over a chunk of rows, accumulated atomically.
template <typename R>
__global__ void k_dc_cols(const R* W, int64_t da, int64_t db, int rows_per, double* c) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= db) return;
  int64_t i0 = (int64_t)blockIdx.y * rows_per, i1 = min(da, i0 + rows_per);
  R s = 0;
#pragma unroll 8
  for (int64_t i = i0; i < i1; ++i) s += W[i * db + j];
  atomicAdd(c + j, (double)s);
}

// dJ_aa[p][q] += 1/2 sum_j c_j occ_b(j)_p occ_b(j)_q; one block per (p, q).
__global__ void __launch_bounds__(kRThreads)
    k_dc_beta_aa(const double* c, int64_t db, const uint32_t* mb, int norb, double* dJaa) {
  __shared__ double red[kRThreads / 32];
  const int p = blockIdx.x / norb, q = blockIdx.x % norb;
  const uint32_t want = (1u << p) | (1u << q);
  double s = 0;
  for (int64_t j = threadIdx.x; j < db; j += kRThreads)
    if ((__ldg(mb + j) & want) == want) s += c[j];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kRThreads / 32; ++k) t += red[k];
    dJaa[blockIdx.x] += 0.5 * t;
  }
}

void launch_dc_grad(Ctx* ctx, const Space* sa, const Space* sb, const void* W, int dtype,
                    double* dJ_aa, double* dJ_ab, cudaStream_t st) {
  ProfScope ps("dc_grad", st, 3);
  const int norb = sa->norb;
  const int sms = ctx->prop.multiProcessorCount;
  unsigned grid = (unsigned)std::min<int64_t>(sa->dim, 4 * sms);
  if (dtype == FS_C64) {
    if (norb <= 16)
      k_dc_rows<float, 16><<<grid, kRThreads, 0, st>>>((const float*)W, sa->dim, sb->dim,
                                                       sa->masks, sb->masks, norb, dJ_aa, dJ_ab);
    else
      k_dc_rows<float, 32><<<grid, kRThreads, 0, st>>>((const float*)W, sa->dim, sb->dim,
                                                       sa->masks, sb->masks, norb, dJ_aa, dJ_ab);
  } else {
    if (norb <= 16)
      k_dc_rows<double, 16><<<grid, kRThreads, 0, st>>>((const double*)W, sa->dim, sb->dim,
                                                        sa->masks, sb->masks, norb, dJ_aa, dJ_ab);
    else
      k_dc_rows<double, 32><<<grid, kRThreads, 0, st>>>((const double*)W, sa->dim, sb->dim,
                                                        sa->masks, sb->masks, norb, dJ_aa, dJ_ab);
  }
  FS_CUDA(cudaGetLastError());
  double* c = (double*)scratch(ctx, "dc_colsum", sb->dim * sizeof(double));
  FS_CUDA(cudaMemsetAsync(c, 0, sb->dim * sizeof(double), st));
  const int rows_per = 64;
  dim3 g2((unsigned)((sb->dim + 255) / 256), (unsigned)((sa->dim + rows_per - 1) / rows_per));
  if (dtype == FS_C64)
    k_dc_cols<float><<<g2, 256, 0, st>>>((const float*)W, sa->dim, sb->dim, rows_per, c);
  else
    k_dc_cols<double><<<g2, 256, 0, st>>>((const double*)W, sa->dim, sb->dim, rows_per, c);
  FS_CUDA(cudaGetLastError());
  k_dc_beta_aa<<<norb * norb, kRThreads, 0, st>>>(c, sb->dim, sb->masks, norb, dJ_aa);
  FS_CUDA(cudaGetLastError());
}

// out[c][r] = in[r][c] for a rows x cols matrix of complex elements: TR x TC
// tiles (TR input rows, TC input columns) through shared memory, so reads
// and writes are both row-contiguous.  256 threads read the tile as rows of
// TC lanes and write it as rows of TR lanes; every thread keeps
// TR * TC / 256 independent loads in flight.
template <typename T, int TR, int TC>
__global__ void __launch_bounds__(256)
    k_transpose(const T* __restrict__ in, T* __restrict__ out, int64_t rows, int64_t cols) {
  static_assert(256 % TC == 0 && 256 % TR == 0, "tile sides divide the block");
  __shared__ T tile[TR][TC + 1];
  const int64_t c0 = (int64_t)blockIdx.x * TC, r0 = (int64_t)blockIdx.y * TR;
  {
    const int tx = threadIdx.x % TC, ty = threadIdx.x / TC;
#pragma unroll
    for (int k = ty; k < TR; k += 256 / TC) {
      const int64_t r = r0 + k, c = c0 + tx;
      if (r < rows && c < cols) tile[k][tx] = in[r * cols + c];
    }
  }
  __syncthreads();
  {
    const int tx = threadIdx.x % TR, ty = threadIdx.x / TR;
#pragma unroll
    for (int k = ty; k < TC; k += 256 / TR) {
      const int64_t c = c0 + k, r = r0 + tx;
      if (c < cols && r < rows) out[c * rows + r] = tile[tx][k];
    }
  }
}

__global__ void k_gather_f64(const double* __restrict__ a, int64_t na,
                             const double* __restrict__ b, int64_t nb,
                             const double* __restrict__ c, int64_t nc, double* out) {
  const int64_t n = na + nb + nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i < na ? a[i] : i < na + nb ? b[i - na] : c[i - na - nb];
}

void launch_gather_f64(const double* a, int64_t na, const double* b, int64_t nb,
                       const double* c, int64_t nc, double* out, cudaStream_t st) {
  const int64_t n = na + nb + nc;
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  k_gather_f64<<<blocks, 256, 0, st>>>(a, na, b, nb, c, nc, out);
  FS_CUDA(cudaGetLastError());
}

void launch_transpose(const void* in, void* out, int64_t rows, int64_t cols, int dtype,
                      cudaStream_t st) {
  ProfScope ps("transpose", st);
  if (dtype == FS_C64) {  // 32 x 64 tiles (17 KB of shared memory)
    FS_REQUIRE((rows + 31) / 32 <= 65535, FS_ERR_UNSUPPORTED, "transpose: too many rows");
    dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((rows + 31) / 32));
    k_transpose<float2, 32, 64><<<grid, 256, 0, st>>>((const float2*)in, (float2*)out, rows, cols);
  } else {  // 32 x 32 tiles of 16-byte elements (17 KB)
    FS_REQUIRE((rows + 31) / 32 <= 65535, FS_ERR_UNSUPPORTED, "transpose: too many rows");
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    k_transpose<double2, 32, 32><<<grid, 256, 0, st>>>((const double2*)in, (double2*)out, rows,
                                                       cols);
  }
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
