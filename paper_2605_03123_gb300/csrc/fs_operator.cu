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
// plain GEMM G = V D (cuBLAS; complex64 with FP32 emulated on the bf16
// tensor cores, complex128 in FP64; real matrix times the complex vectors
// viewed as pairs of reals), and the outer E_pq is a
// gather through the single-excitation table.  The beta part runs on
// blocks of rows (a beta excitation stays in its row), the alpha and mixed
// parts on blocks of columns (an alpha excitation stays in its column);
// the block size bounds the N^2 x block intermediates.
#include <cublas_v2.h>

#include <algorithm>

#include "fs_common.cuh"
#include "fs_internal.h"

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

static cublasHandle_t blas_handle(Ctx* ctx) {
  if (!ctx->blas) {
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) {
      set_error("cublasCreate failed");
      throw Fail{FS_ERR_CUDA};
    }
    ctx->blas = h;
  }
  return (cublasHandle_t)ctx->blas;
}

void release_blas(Ctx* ctx) {
  if (ctx->blas) cublasDestroy((cublasHandle_t)ctx->blas);
  ctx->blas = nullptr;
}

// G (row-major [n][m]) = V (row-major [n][k], leading dimension ldv) x
// D (row-major [k][m]), real; m counts reals (two per complex element).
static void gemm(Ctx* ctx, int dtype, int64_t m, int n, int k, const void* D, const void* V,
                 int ldv, void* G, cudaStream_t st) {
  FS_REQUIRE(m <= 0x7FFFFFFF, FS_ERR_UNSUPPORTED, "operator block too large for one GEMM");
  cublasHandle_t h = blas_handle(ctx);
  cublasSetStream(h, st);
  cublasStatus_t s;
  if (dtype == FS_C64) {
    // FP32 products emulated on the bf16 tensor cores (three-way bf16
    // splits; FP32-level accuracy): measured 1.25x faster than FP32 FFMA
    cublasSetMathMode(h, CUBLAS_FP32_EMULATED_BF16X9_MATH);
    const float one = 1, zero = 0;
    s = cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)m, n, k, &one, (const float*)D, (int)m,
                    (const float*)V, ldv, &zero, (float*)G, (int)m);
  } else {
    cublasSetMathMode(h, CUBLAS_DEFAULT_MATH);
    const double one = 1, zero = 0;
    s = cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)m, n, k, &one, (const double*)D, (int)m,
                    (const double*)V, ldv, &zero, (double*)G, (int)m);
  }
  if (s != CUBLAS_STATUS_SUCCESS) {
    set_error("cuBLAS GEMM failed with status " + std::to_string((int)s));
    throw Fail{FS_ERR_CUDA};
  }
}

template <typename R>
static void molecular_hamiltonian_t(Ctx* ctx, Space* sa, Space* sb, const void* vec_, void* out_,
                                    const double* h1, const double* h2, double constant,
                                    int64_t ws, cudaStream_t st) {
  using C = cx_t<R>;
  const int N = sa->norb, NN = N * N;
  const int dtype = sizeof(R) == 4 ? FS_C64 : FS_C128;
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
  // block sizes from the workspace budget (D and G together)
  const size_t csz = sizeof(C);
  size_t budget = (size_t)ws;
  if (ws <= 0) {
    size_t fr = 0, tot = 0;
    FS_CUDA(cudaMemGetInfo(&fr, &tot));
    budget = std::min<size_t>((size_t)8 << 30, fr / 4);
  }
  const int64_t nr = std::max<int64_t>(1, std::min<int64_t>(da, budget / (2 * NN * csz * db)));
  const int64_t nc = std::max<int64_t>(1, std::min<int64_t>(db, budget / (3 * NN * csz * da)));
  const int64_t xmax = std::max(nr * db, nc * da);
  C* D = (C*)scratch(ctx, "op_D", (size_t)2 * NN * xmax * csz);
  C* G = (C*)scratch(ctx, "op_G", (size_t)NN * xmax * csz);
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
      ProfScope ps("op_gemm", st, 0);
      gemm(ctx, dtype, 2 * X, NN, NN, D, Vd, 2 * NN, G, st);
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
      ProfScope ps("op_gemm", st, 0);
      gemm(ctx, dtype, 2 * X, NN, 2 * NN, D, Vd, 2 * NN, G, st);
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
