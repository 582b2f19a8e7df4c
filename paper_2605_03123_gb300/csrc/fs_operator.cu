// Action of a molecular Hamiltonian with real tensors on a state
// (operator-action section; the molecular Hamiltonian equation).
//
// Within one spin, a^dag_p a^dag_r a_s a_q = E_pq E_rs - delta_qr E_ps, and
// the two spin orders of the mixed term are the same product of commuting
// one-spin operators, so
//   H = c + sum_pq k_pq (E^a_pq + E^b_pq)
//         + sum_pq E^a_pq [sum_rs V_pqrs E^a_rs + W_pqrs E^b_rs]
//         + sum_pq E^b_pq [sum_rs V_pqrs E^b_rs],
//   k_pq = h_pq - 1/2 sum_r h_prrq,  V = h / 2,  W_pqrs = (h_pqrs + h_rspq) / 2.
// Each bracket is a contraction over rs: with D_rs = E_rs psi it is the
// GEMM G = V D (a real matrix times the complex vectors viewed as pairs of
// reals): complex64 on the tcgen05 tensor cores (gemm_tc: D transposed and
// split into exact BF16 triples, V split on the host; FP32 accuracy),
// complex128 as a tiled FP64 GEMM on the CUDA cores; and the outer E_pq is a
// gather through the single-excitation table.  The beta part runs on
// blocks of rows (a beta excitation stays in its row), the alpha and mixed
// parts on blocks of columns (an alpha excitation stays in its column);
// the block size bounds the N^2 x block intermediates.
#include <cuda_bf16.h>

#include <algorithm>

#include "fs_common.cuh"
#include "fs_internal.h"
#include "fs_tc.cuh"

namespace fs {

// D[rs][t][c] = (E_rs X)[t][col0 + c] for all rs, the rows t of X being
// strings of the excited spin: sign * X[E_sr t][col0 + c] or 0.  One CTA per
// target row.
template <typename R>
__global__ void __launch_bounds__(256)
    k_excite_rows(cx_t<R>* D, const cx_t<R>* X, int64_t ldx, int64_t col0, int ncol,
                  int64_t nrows, const uint16_t* gpq, const uint32_t* gsrc, int ne, int NN,
                  int64_t dstride) {
  extern __shared__ int ent[];  // NN: entry index of rs in row t's table, or -1
  for (int64_t t = blockIdx.x; t < nrows; t += gridDim.x) {
    for (int k = threadIdx.x; k < NN; k += blockDim.x) ent[k] = -1;
    __syncthreads();
    for (int k = threadIdx.x; k < ne; k += blockDim.x) ent[gpq[t * ne + k]] = k;
    __syncthreads();
    for (int rs = 0; rs < NN; ++rs) {
      const int k = ent[rs];
      cx_t<R>* d = D + rs * dstride + t * ncol;
      if (k < 0) {
        for (int c = threadIdx.x; c < ncol; c += blockDim.x) d[c] = mk<R>(0, 0);
      } else {
        const uint32_t v = gsrc[t * ne + k];
        const R sg = (v >> 31) ? R(-1) : R(1);
        const cx_t<R>* x = X + (int64_t)(v & 0x7FFFFFFFu) * ldx + col0;
        for (int c = threadIdx.x; c < ncol; c += blockDim.x)
          d[c] = mk<R>(sg * x[c].x, sg * x[c].y);
      }
    }
    __syncthreads();
  }
}

// D[rs][ii][c] = (E_rs X)[row0 + ii][col0 + c] with the columns of X
// strings of the excited spin: sign * X[row0 + ii][E_sr (col0 + c)] or 0.
// One thread per output element; its column's table is walked in rs order.
template <typename R>
__global__ void __launch_bounds__(256)
    k_excite_cols(cx_t<R>* D, const cx_t<R>* X, int64_t ldx, int64_t row0, int64_t nrow,
                  int64_t col0, int64_t ncol, const uint16_t* gpq, const uint32_t* gsrc, int ne,
                  int NN, int64_t dstride) {
  const int64_t total = nrow * ncol;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ii = idx / ncol, col = col0 + (idx - ii * ncol);
    const cx_t<R>* x = X + (row0 + ii) * ldx;
    const uint16_t* tp = gpq + col * ne;
    const uint32_t* ts = gsrc + col * ne;
    int k = 0;
    int next = ne > 0 ? tp[0] : NN;
    for (int rs = 0; rs < NN; ++rs) {
      cx_t<R> v = mk<R>(0, 0);
      if (rs == next) {
        const uint32_t s = ts[k];
        const cx_t<R> a = x[s & 0x7FFFFFFFu];
        v = (s >> 31) ? mk<R>(-a.x, -a.y) : a;
        ++k;
        next = k < ne ? tp[k] : NN;
      }
      D[rs * dstride + idx] = v;
    }
  }
}

// out[t][col0 + c] (+)= sum over row t's table entries (pq, src, sign) of
// sign * (G[pq][src][c] + k_pq X[src][col0 + c]): the outer E_pq along rows.
template <typename R>
__global__ void __launch_bounds__(256)
    k_gather_rows(cx_t<R>* out, int64_t ldo, int64_t col0, int ncol, int64_t nrows,
                  const cx_t<R>* G, int64_t gstride, const cx_t<R>* X, int64_t ldx,
                  const uint16_t* gpq, const uint32_t* gsrc, int ne,
                  const __grid_constant__ Mat kmat) {
  for (int64_t t = blockIdx.x; t < nrows; t += gridDim.x) {
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      cx_t<R> acc = out[t * ldo + col0 + c];
      for (int k = 0; k < ne; ++k) {
        const uint32_t v = gsrc[t * ne + k];
        const int pq = gpq[t * ne + k];
        const int64_t src = v & 0x7FFFFFFFu;
        const R sg = (v >> 31) ? R(-1) : R(1), kk = (R)kmat.v[pq];
        const cx_t<R> g = G[pq * gstride + src * ncol + c];
        const cx_t<R> x = X[src * ldx + col0 + c];
        acc.x += sg * (g.x + kk * x.x);
        acc.y += sg * (g.y + kk * x.y);
      }
      out[t * ldo + col0 + c] = acc;
    }
  }
}

// out[row0 + ii][j] = c X[row0 + ii][j] + sum over column j's entries of
// sign * (G[pq][ii][src] + k_pq X[row0 + ii][src]): the outer E_pq along
// columns, which also initialises the output.
template <typename R>
__global__ void __launch_bounds__(256)
    k_gather_cols(cx_t<R>* out, int64_t ldo, int64_t row0, int64_t nrow, int64_t ncol,
                  const cx_t<R>* G, int64_t gstride, const cx_t<R>* X, int64_t ldx,
                  const uint16_t* gpq, const uint32_t* gsrc, int ne,
                  const __grid_constant__ Mat kmat, double constant) {
  const int64_t total = nrow * ncol;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ii = idx / ncol, j = idx - ii * ncol;
    const cx_t<R>* x = X + (row0 + ii) * ldx;
    const R cst = (R)constant;
    cx_t<R> acc = mk<R>(cst * x[j].x, cst * x[j].y);
    for (int k = 0; k < ne; ++k) {
      const uint32_t v = gsrc[j * ne + k];
      const int pq = gpq[j * ne + k];
      const int64_t src = v & 0x7FFFFFFFu;
      const R sg = (v >> 31) ? R(-1) : R(1), kk = (R)kmat.v[pq];
      const cx_t<R> g = G[pq * gstride + ii * ncol + src];
      acc.x += sg * (g.x + kk * x[src].x);
      acc.y += sg * (g.y + kk * x[src].y);
    }
    out[(row0 + ii) * ldo + j] = acc;
  }
}

// The left operand of the tensor-core contraction: A_q[(2 p + c) * lda + k]
// = piece q of component c (0 = Re, 1 = Im) of D[k][p], for k < K rows of D
// (K x X complex, row stride X) and positions p < X; columns K .. lda - 1
// are zeroed.  32 x 32 tiles through shared memory, so both the reads of D
// and the writes of the planes run along contiguous memory.
__global__ void __launch_bounds__(256)
    k_transpose_split(const float2* D, int K, int64_t X, __nv_bfloat16* A0, __nv_bfloat16* A1,
                      __nv_bfloat16* A2, int64_t lda) {
  __shared__ float2 tile[32][33];
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r;
    const int64_t p = p0 + tx;
    tile[r][tx] = (k < K && p < X) ? D[(int64_t)k * X + p] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  __nv_bfloat16* planes[3] = {A0, A1, A2};
  for (int r = ty; r < 32; r += 8) {  // r: position within the tile; tx: k
    const int64_t p = p0 + r;
    const int k = k0 + tx;
    if (p >= X || k >= (int)lda) continue;
    const float2 v = tile[tx][r];
    uint32_t w[3];
    tc::split_bf16x3(v.x, v.y, w[0], w[1], w[2]);  // low half Re, high half Im
    for (int q = 0; q < 3; ++q) {
      planes[q][(2 * p) * lda + k] = __ushort_as_bfloat16((unsigned short)(w[q] & 0xFFFFu));
      planes[q][(2 * p + 1) * lda + k] = __ushort_as_bfloat16((unsigned short)(w[q] >> 16));
    }
  }
}

// G[m][n] = sum_k V[m][k] D[k][n], real FP64 (row-major, leading dimensions
// ldv, ldd, ldg): 64 x 64 tiles, 256 threads, 4 x 4 outputs per thread.
constexpr int kRT = 64, kRK = 16;
__global__ void __launch_bounds__(256)
    k_rgemm_f64(const double* V, int64_t ldv, const double* D, int64_t ldd, double* G,
                int64_t ldg, int M, int64_t N, int K) {
  __shared__ double sa[kRK][kRT + 1];
  __shared__ double sb[kRK][kRT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kRT;
  const int64_t n0 = (int64_t)blockIdx.x * kRT;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kRK) {
    for (int e = threadIdx.x; e < kRK * kRT; e += 256) {
      const int kk = e / kRT, mm = e - kk * kRT;
      const int gk = k0 + kk;
      sa[kk][mm] = (m0 + mm < M && gk < K) ? V[(int64_t)(m0 + mm) * ldv + gk] : 0.0;
      sb[kk][mm] = (n0 + mm < N && gk < K) ? D[(int64_t)gk * ldd + n0 + mm] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kRK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sa[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sb[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty * 4 + i;
      const int64_t n = n0 + tx * 4 + j;
      if (m < M && n < N) G[(int64_t)m * ldg + n] = acc[i][j];
    }
}

// G (row-major [n][2X] reals) = V (row-major [n][k] reals, leading dimension
// ldv; for complex64 its three BF16 planes Vp with the same layout) x
// D (k rows of X complex).  Ap: scratch for the transposed planes of D.
template <typename R>
static void contract(Ctx* ctx, int64_t X, int n, int k, const void* D, const R* Vd,
                     const uint16_t* Vp, int ldv, int ldvp, void* G, uint16_t* Ap,
                     cudaStream_t st) {
  FS_REQUIRE(2 * X <= 0x7FFFFFFF, FS_ERR_UNSUPPORTED, "operator block too large for one GEMM");
  if constexpr (sizeof(R) == 4) {
    const int64_t lda = (k + 7) / 8 * 8;
    const size_t plane = (size_t)2 * X * lda;
    dim3 grid((unsigned)((X + 31) / 32), (unsigned)((lda + 31) / 32));
    k_transpose_split<<<grid, 256, 0, st>>>((const float2*)D, k, X, (__nv_bfloat16*)Ap,
                                            (__nv_bfloat16*)(Ap + plane),
                                            (__nv_bfloat16*)(Ap + 2 * plane), lda);
    FS_CUDA(cudaGetLastError());
    GemmTc g{};
    for (int q = 0; q < 3; ++q) {
      g.A[q] = Ap + q * plane;
      g.B[q] = Vp + (size_t)q * n * ldvp;
    }
    g.M = (int)(2 * X);
    g.N = n;
    g.K = k;
    g.lda = lda;
    g.ldb = ldvp;
    g.out = G;
    g.mode = GEMM_REAL_T;
    g.ldo = 2 * X;
    g.status = ctx->d_status;
    gemm_tc(g, st);
  } else {
    dim3 grid((unsigned)((2 * X + kRT - 1) / kRT), (unsigned)((n + kRT - 1) / kRT));
    k_rgemm_f64<<<grid, 256, 0, st>>>(Vd, ldv, (const double*)D, 2 * X, (double*)G, 2 * X, n,
                                      2 * X, k);
    FS_CUDA(cudaGetLastError());
  }
}

template <typename R>
static void molecular_hamiltonian_t(Ctx* ctx, Space* sa, Space* sb, const void* vec_, void* out_,
                                    const double* h1, const double* h2, double constant,
                                    int64_t ws, cudaStream_t st) {
  using C = cx_t<R>;
  const int N = sa->norb, NN = N * N;
  const C* vec = (const C*)vec_;
  C* out = (C*)out_;
  const int64_t da = sa->dim, db = sb->dim;
  build_gather_table(sa, st);
  build_gather_table(sb, st);
  // host: k, and V = [h/2 | W] as the row-major NN x 2NN real matrix
  Mat kmat{};
  std::vector<R> V((size_t)NN * 2 * NN);
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) {
      double s = h1[p * N + q];
      for (int r = 0; r < N; ++r) s -= 0.5 * h2[((size_t)(p * N + r) * N + r) * N + q];
      kmat.v[p * N + q] = s;
    }
  for (int pq = 0; pq < NN; ++pq)
    for (int rs = 0; rs < NN; ++rs) {
      const double a = h2[(size_t)pq * NN + rs], b = h2[(size_t)rs * NN + pq];
      V[(size_t)pq * 2 * NN + rs] = (R)(0.5 * a);
      V[(size_t)pq * 2 * NN + NN + rs] = (R)(0.5 * (a + b));
    }
  R* Vd = (R*)scratch(ctx, "op_V", V.size() * sizeof(R));
  FS_CUDA(cudaMemcpyAsync(Vd, V.data(), V.size() * sizeof(R), cudaMemcpyHostToDevice, st));
  uint16_t* Vp = nullptr;
  std::vector<uint16_t> Vh;
  const int ldvp = (2 * NN + 7) / 8 * 8;
  if (sizeof(R) == 4) {
    // three BF16 planes of V from FP64 (each the nearest BF16 of the
    // remainder), rows padded to a multiple of 8 entries (16 bytes)
    const size_t nv = (size_t)NN * ldvp;
    Vh.assign(3 * nv, 0);
    for (int pq = 0; pq < NN; ++pq)
      for (int rs = 0; rs < 2 * NN; ++rs) {
        const double a = h2[(size_t)pq * NN + rs % NN], b = h2[(size_t)(rs % NN) * NN + pq];
        double r = rs < NN ? 0.5 * a : 0.5 * (a + b);
        for (int q = 0; q < 3; ++q) {
          const __nv_bfloat16 v = __float2bfloat16_rn((float)r);
          Vh[q * nv + (size_t)pq * ldvp + rs] = __bfloat16_as_ushort(v);
          r -= (double)__bfloat162float(v);
        }
      }
    Vp = (uint16_t*)scratch(ctx, "op_Vp", Vh.size() * sizeof(uint16_t));
    FS_CUDA(cudaMemcpyAsync(Vp, Vh.data(), Vh.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                            st));
  }
  // block sizes from the workspace budget (D and G together)
  const size_t csz = sizeof(C);
  size_t budget = (size_t)ws;
  if (ws <= 0) {
    size_t fr = 0, tot = 0;
    FS_CUDA(cudaMemGetInfo(&fr, &tot));
    budget = std::min<size_t>((size_t)8 << 30, fr / 4);
  }
  // per position: D (2 N^2 complex), G (N^2 complex) and, for complex64, the
  // transposed BF16 planes of D (3 x 2 x 2 N^2 x 2 bytes)
  const size_t per = (size_t)3 * NN * csz + (sizeof(R) == 4 ? (size_t)24 * NN : 0);
  const int64_t nr = std::max<int64_t>(1, std::min<int64_t>(da, budget / (per * db)));
  const int64_t nc = std::max<int64_t>(1, std::min<int64_t>(db, budget / (per * da)));
  const int64_t xmax = std::max(nr * db, nc * da);
  C* D = (C*)scratch(ctx, "op_D", (size_t)2 * NN * xmax * csz);
  C* G = (C*)scratch(ctx, "op_G", (size_t)NN * xmax * csz);
  uint16_t* Ap = sizeof(R) == 4
                     ? (uint16_t*)scratch(ctx, "op_Dp", (size_t)3 * 2 * xmax * (2 * NN + 8) * 2)
                     : nullptr;
  const int sms = ctx->prop.multiProcessorCount;
  // beta part on row blocks; also writes c psi and the beta one-body term
  for (int64_t i0 = 0; i0 < da; i0 += nr) {
    const int64_t nrow = std::min(nr, da - i0), X = nrow * db;
    {
      ProfScope ps("op_excite", st);
      const unsigned grid = (unsigned)std::min<int64_t>((X + 255) / 256, 32 * sms);
      k_excite_cols<R><<<grid, 256, 0, st>>>(D, vec, db, i0, nrow, 0, db, sb->gpq, sb->gsrc,
                                             sb->ne, NN, X);
      FS_CUDA(cudaGetLastError());
    }
    {
      ProfScope ps("op_gemm", st, sizeof(R) == 4 ? 2 : 1);
      contract<R>(ctx, X, NN, NN, D, Vd, Vp, 2 * NN, ldvp, G, Ap, st);
    }
    {
      ProfScope ps("op_gather", st);
      const unsigned grid = (unsigned)std::min<int64_t>((X + 255) / 256, 32 * sms);
      k_gather_cols<R><<<grid, 256, 0, st>>>(out, db, i0, nrow, db, G, X, vec, db, sb->gpq,
                                             sb->gsrc, sb->ne, kmat, constant);
      FS_CUDA(cudaGetLastError());
    }
  }
  // alpha and mixed parts on column blocks, added to the output
  for (int64_t j0 = 0; j0 < db; j0 += nc) {
    const int64_t ncol = std::min(nc, db - j0), X = da * ncol;
    {
      ProfScope ps("op_excite", st, 2);
      const unsigned g1 = (unsigned)std::min<int64_t>(da, 32 * sms);
      k_excite_rows<R><<<g1, 256, NN * sizeof(int), st>>>(D, vec, db, j0, (int)ncol, da, sa->gpq,
                                                          sa->gsrc, sa->ne, NN, X);
      FS_CUDA(cudaGetLastError());
      const unsigned g2 = (unsigned)std::min<int64_t>((X + 255) / 256, 32 * sms);
      k_excite_cols<R><<<g2, 256, 0, st>>>(D + (int64_t)NN * X, vec, db, 0, da, j0, ncol, sb->gpq,
                                           sb->gsrc, sb->ne, NN, X);
      FS_CUDA(cudaGetLastError());
    }
    {
      ProfScope ps("op_gemm", st, sizeof(R) == 4 ? 2 : 1);
      contract<R>(ctx, X, NN, 2 * NN, D, Vd, Vp, 2 * NN, ldvp, G, Ap, st);
    }
    {
      ProfScope ps("op_gather", st);
      const unsigned grid = (unsigned)std::min<int64_t>(da, 32 * sms);
      k_gather_rows<R><<<grid, 256, 0, st>>>(out, db, j0, (int)ncol, da, G, X, vec, db, sa->gpq,
                                             sa->gsrc, sa->ne, kmat);
      FS_CUDA(cudaGetLastError());
    }
  }
}

void molecular_hamiltonian(Ctx* ctx, Space* sa, Space* sb, const void* vec, void* out, int dtype,
                           const double* h1, const double* h2, double constant,
                           int64_t workspace_bytes, cudaStream_t st) {
  FS_REQUIRE(sa->norb * sa->norb <= 1024 && sa->norb * sa->norb < 65536, FS_ERR_UNSUPPORTED,
             "operator action supports norb <= 32");
  if (dtype == FS_C64)
    molecular_hamiltonian_t<float>(ctx, sa, sb, vec, out, h1, h2, constant, workspace_bytes, st);
  else
    molecular_hamiltonian_t<double>(ctx, sa, sb, vec, out, h1, h2, constant, workspace_bytes, st);
}

}  // namespace fs
