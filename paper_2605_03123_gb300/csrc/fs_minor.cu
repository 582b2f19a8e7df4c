// Orbital rotation by dense minor matrices, for small string dimensions.
//
// From U a^dag_p U^dag = sum_q U_qp a^dag_q (§2.3) applied to every creation
// operator of |I> = cre(I)|vac>, the rotated string is
//   U|I> = sum_J det(U[J, I]) |J>   (rows J, columns I, both ascending),
// so one spin is rotated by the matrix M[J][I] = det(U[J, I]) and the state
// by psi' = M_a psi M_b^T.  The minors are computed in FP64 on the device.
// complex64: the two products run on the tcgen05 tensor cores (gemm_tc,
// operands as exact BF16 triples, FP32 accuracy), the complex matrices in
// real form; complex128: tiled complex GEMMs on the FP64 CUDA cores.
#include <cuda_bf16.h>

#include <algorithm>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

constexpr int kMinorMaxN = 16;  // electrons per spin on this path

// M[J][I] = det(U[rows of J, columns of I]), FP64 Gaussian elimination with
// partial pivoting; one thread per entry.
template <typename R>
__global__ void k_minor_matrix(cx_t<R>* M, const uint32_t* masks, int64_t d, int norb, int n,
                               const __grid_constant__ CMat U) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= d * d) return;
  const int64_t J = t / d, I = t - J * d;
  double2 a[kMinorMaxN * kMinorMaxN];
  const uint32_t mj = masks[J], mi = masks[I];
  int r = 0;
  for (int p = 0; p < norb; ++p) {
    if (!((mj >> p) & 1u)) continue;
    int c = 0;
    for (int q = 0; q < norb; ++q) {
      if (!((mi >> q) & 1u)) continue;
      a[r * n + c] = make_double2(U.v[2 * (p * norb + q)], U.v[2 * (p * norb + q) + 1]);
      ++c;
    }
    ++r;
  }
  double dr = 1, di = 0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = hypot(a[k * n + k].x, a[k * n + k].y);
    for (int i = k + 1; i < n; ++i) {
      double h = hypot(a[i * n + k].x, a[i * n + k].y);
      if (h > best) {
        best = h;
        piv = i;
      }
    }
    if (best == 0) {
      dr = di = 0;
      break;
    }
    if (piv != k) {
      for (int c = 0; c < n; ++c) {
        double2 tmp = a[k * n + c];
        a[k * n + c] = a[piv * n + c];
        a[piv * n + c] = tmp;
      }
      dr = -dr;
      di = -di;
    }
    const double2 pk = a[k * n + k];
    const double nr = dr * pk.x - di * pk.y;
    di = dr * pk.y + di * pk.x;
    dr = nr;
    const double inv = 1.0 / (pk.x * pk.x + pk.y * pk.y);
    for (int i = k + 1; i < n; ++i) {
      const double2 x = a[i * n + k];
      const double fr = (x.x * pk.x + x.y * pk.y) * inv, fi = (x.y * pk.x - x.x * pk.y) * inv;
      for (int c = k + 1; c < n; ++c) {
        const double2 y = a[k * n + c];
        a[i * n + c].x -= fr * y.x - fi * y.y;
        a[i * n + c].y -= fr * y.y + fi * y.x;
      }
    }
  }
  M[t] = mk<R>((R)dr, (R)di);
}

// C[m][n] = sum_k A[m][k] * B'[k][n] with B' = B (TB = false) or B^T
// (TB = true, B stored [n][k]); complex, 64 x 64 tiles, 256 threads, each
// thread 4 x 4 outputs.
constexpr int kTile = 64, kTk = 16;
template <typename R, bool TB>
__global__ void __launch_bounds__(256)
    k_cgemm(const cx_t<R>* A, const cx_t<R>* B, cx_t<R>* Cm, int M, int N, int K) {
  using Cx = cx_t<R>;
  __shared__ Cx sa[kTk][kTile + 1];
  __shared__ Cx sb[kTk][kTile + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  Cx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<R>(0, 0);
  for (int k0 = 0; k0 < K; k0 += kTk) {
    for (int e = threadIdx.x; e < kTk * kTile; e += 256) {
      const int kk = e / kTile, mm = e - kk * kTile;
      const int gm = m0 + mm, gk = k0 + kk;
      sa[kk][mm] = (gm < M && gk < K) ? A[(int64_t)gm * K + gk] : mk<R>(0, 0);
      const int gn = n0 + mm;
      Cx bv = mk<R>(0, 0);
      if (gn < N && gk < K) bv = TB ? B[(int64_t)gn * K + gk] : B[(int64_t)gk * N + gn];
      sb[kk][mm] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTk; ++kk) {
      Cx av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sa[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = sb[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(av[i].x, bv[j].x, fma(-av[i].y, bv[j].y, acc[i][j].x));
          acc[i][j].y = fma(av[i].x, bv[j].y, fma(av[i].y, bv[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) Cm[(int64_t)gm * N + gn] = acc[i][j];
    }
}

// det(U[rows of mj, columns of mi]) for NE electrons, FP64 Gaussian
// elimination with partial pivoting (on the squared modulus) in registers.
template <int NE>
__device__ __forceinline__ double2 minor_det(uint32_t mj, uint32_t mi, int norb, const double* Uv) {
  if constexpr (NE == 0) {
    return make_double2(1, 0);
  } else {
  int rows[NE], cols[NE];
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    rows[k] = __ffs(mj) - 1;
    mj &= mj - 1;
    cols[k] = __ffs(mi) - 1;
    mi &= mi - 1;
  }
  double2 a[NE][NE];
#pragma unroll
  for (int r = 0; r < NE; ++r)
#pragma unroll
    for (int c = 0; c < NE; ++c) {
      const int o = 2 * (rows[r] * norb + cols[c]);
      a[r][c] = make_double2(Uv[o], Uv[o + 1]);
    }
  double dr = 1, di = 0;
  bool singular = false;
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    int piv = k;
    double best = a[k][k].x * a[k][k].x + a[k][k].y * a[k][k].y;
#pragma unroll
    for (int i = k + 1; i < NE; ++i) {
      const double h = a[i][k].x * a[i][k].x + a[i][k].y * a[i][k].y;
      if (h > best) {
        best = h;
        piv = i;
      }
    }
    singular = singular || best == 0;
    // row swap k <-> piv by selects, so that every index stays compile-time
#pragma unroll
    for (int i = k + 1; i < NE; ++i) {
      const bool sw = i == piv;
#pragma unroll
      for (int c = k; c < NE; ++c) {
        const double2 tk = a[k][c], ti = a[i][c];
        a[k][c] = sw ? ti : tk;
        a[i][c] = sw ? tk : ti;
      }
    }
    if (piv != k) {
      dr = -dr;
      di = -di;
    }
    const double2 pk = a[k][k];
    const double nr = dr * pk.x - di * pk.y;
    di = dr * pk.y + di * pk.x;
    dr = nr;
    const double inv = best > 0 ? 1.0 / best : 0.0;
#pragma unroll
    for (int i = k + 1; i < NE; ++i) {
      const double2 x = a[i][k];
      const double fr = (x.x * pk.x + x.y * pk.y) * inv, fi = (x.y * pk.x - x.x * pk.y) * inv;
#pragma unroll
      for (int c = k + 1; c < NE; ++c) {
        const double2 y = a[k][c];
        a[i][c].x -= fr * y.x - fi * y.y;
        a[i][c].y -= fr * y.y + fi * y.x;
      }
    }
  }
  return singular ? make_double2(0, 0) : make_double2(dr, di);
  }
}

// The minor matrix M[J][I] = det(U[J, I]) in the real form of a complex
// right operand, as three BF16 planes (row stride ld): row 2J + x, column
// 2I + y holds [[Re, -Im], [Im, Re]][x][y] of M[J][I], split from FP64 into
// the nearest BF16 of each remainder.  One thread per (J, I).
template <int NE>
__global__ void k_minor_planes(const uint32_t* masks, int64_t d, int norb,
                               const __grid_constant__ CMat U, __nv_bfloat16* p0,
                               __nv_bfloat16* p1, __nv_bfloat16* p2, int64_t ld) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= d * d) return;
  const int64_t J = t / d, I = t - J * d;
  const double2 v = minor_det<NE>(masks[J], masks[I], norb, U.v);
  const double ent[4] = {v.x, -v.y, v.y, v.x};
  __nv_bfloat16* planes[3] = {p0, p1, p2};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t off = (2 * J + (e >> 1)) * ld + 2 * I + (e & 1);
    double rem = ent[e];
#pragma unroll
    for (int pc = 0; pc < 3; ++pc) {
      const __nv_bfloat16 b = __float2bfloat16_rn((float)rem);
      planes[pc][off] = b;
      rem -= (double)__bfloat162float(b);
    }
  }
}

template <int NE>
static void minor_planes_n(const Space* sp, const CMat& U, uint16_t* B, size_t plane, int64_t ld,
                           cudaStream_t st) {
  const int64_t d = sp->dim;
  k_minor_planes<NE><<<(unsigned)((d * d + 127) / 128), 128, 0, st>>>(
      sp->masks, d, sp->norb, U, (__nv_bfloat16*)B, (__nv_bfloat16*)(B + plane),
      (__nv_bfloat16*)(B + 2 * plane), ld);
  FS_CUDA(cudaGetLastError());
}

static void minor_planes(const Space* sp, const CMat& U, uint16_t* B, size_t plane, int64_t ld,
                         cudaStream_t st) {
  switch (sp->nocc) {
    case 0: minor_planes_n<0>(sp, U, B, plane, ld, st); break;
    case 1: minor_planes_n<1>(sp, U, B, plane, ld, st); break;
    case 2: minor_planes_n<2>(sp, U, B, plane, ld, st); break;
    case 3: minor_planes_n<3>(sp, U, B, plane, ld, st); break;
    case 4: minor_planes_n<4>(sp, U, B, plane, ld, st); break;
    case 5: minor_planes_n<5>(sp, U, B, plane, ld, st); break;
    case 6: minor_planes_n<6>(sp, U, B, plane, ld, st); break;
    case 7: minor_planes_n<7>(sp, U, B, plane, ld, st); break;
    case 8: minor_planes_n<8>(sp, U, B, plane, ld, st); break;
    case 9: minor_planes_n<9>(sp, U, B, plane, ld, st); break;
    case 10: minor_planes_n<10>(sp, U, B, plane, ld, st); break;
    case 11: minor_planes_n<11>(sp, U, B, plane, ld, st); break;
    case 12: minor_planes_n<12>(sp, U, B, plane, ld, st); break;
    case 13: minor_planes_n<13>(sp, U, B, plane, ld, st); break;
    case 14: minor_planes_n<14>(sp, U, B, plane, ld, st); break;
    case 15: minor_planes_n<15>(sp, U, B, plane, ld, st); break;
    case 16: minor_planes_n<16>(sp, U, B, plane, ld, st); break;
    default: FS_REQUIRE(false, FS_ERR_UNSUPPORTED, "at most 16 electrons per spin");
  }
}

// complex64 on the tensor cores: tmp^T = (psi M_b^T)^T, then
// psi' = (tmp^T M_a^T)^T, each a real-form GEMM whose right operand is an
// expanded minor matrix.
static void minor_rotation_tc(Ctx* ctx, const Space* sa, const Space* sb, void* vec,
                              const CMat& Ua, const CMat& Ub, cudaStream_t st) {
  const int64_t da = sa->dim, db = sb->dim;
  const int64_t lka = (2 * da + 7) / 8 * 8, lkb = (2 * db + 7) / 8 * 8;
  const size_t pa = (size_t)2 * da * lka, pb = (size_t)2 * db * lkb;  // elements per plane
  const size_t ppsi = (size_t)da * lkb, ptmp = (size_t)db * lka;
  uint16_t* Ba = (uint16_t*)scratch(ctx, "minor_tc_a", 3 * pa * 2);
  uint16_t* Bb = (uint16_t*)scratch(ctx, "minor_tc_b", 3 * pb * 2);
  uint16_t* Ap = (uint16_t*)scratch(ctx, "minor_tc_psi", 3 * ppsi * 2);
  uint16_t* Tp = (uint16_t*)scratch(ctx, "minor_tc_tmp", 3 * ptmp * 2);
  {
    // (padding columns past K are never read: the GEMM loads stop at K)
    ProfScope ps("minor_matrices", st, 2);
    minor_planes(sa, Ua, Ba, pa, lka, st);
    minor_planes(sb, Ub, Bb, pb, lkb, st);
  }
  ProfScope ps("minor_gemm_tc", st, 3);
  void* psi_planes[3] = {Ap, Ap + ppsi, Ap + 2 * ppsi};
  split_planes(vec, da, (int)db, db, psi_planes, lkb, st);
  GemmTc g{};
  for (int p = 0; p < 3; ++p) {
    g.A[p] = Ap + p * ppsi;
    g.B[p] = Bb + p * pb;
    g.outp[p] = Tp + p * ptmp;
  }
  g.M = (int)da;
  g.N = (int)(2 * db);
  g.K = (int)(2 * db);
  g.lda = lkb;
  g.ldb = lkb;
  g.mode = GEMM_CPLX_T_PLANES;
  g.ldp = lka;
  g.status = ctx->d_status;
  gemm_tc(g, st);
  GemmTc h{};
  for (int p = 0; p < 3; ++p) {
    h.A[p] = Tp + p * ptmp;
    h.B[p] = Ba + p * pa;
  }
  h.M = (int)db;
  h.N = (int)(2 * da);
  h.K = (int)(2 * da);
  h.lda = lka;
  h.ldb = lka;
  h.out = vec;
  h.mode = GEMM_CPLX_T;
  h.ldo = db;
  h.status = ctx->d_status;
  gemm_tc(h, st);
}

template <typename R>
static void minor_rotation_t(Ctx* ctx, const Space* sa, const Space* sb, void* vec,
                             const CMat& Ua, const CMat& Ub, cudaStream_t st) {
  using Cx = cx_t<R>;
  const int64_t da = sa->dim, db = sb->dim;
  Cx* Ma = (Cx*)scratch(ctx, "minor_a", da * da * sizeof(Cx));
  Cx* Mb = (Cx*)scratch(ctx, "minor_b", db * db * sizeof(Cx));
  Cx* tmp = (Cx*)scratch(ctx, "minor_tmp", da * db * sizeof(Cx));
  {
    ProfScope ps("minor_matrices", st, 2);
    k_minor_matrix<R><<<(unsigned)((da * da + 127) / 128), 128, 0, st>>>(Ma, sa->masks, da,
                                                                          sa->norb, sa->nocc, Ua);
    FS_CUDA(cudaGetLastError());
    k_minor_matrix<R><<<(unsigned)((db * db + 127) / 128), 128, 0, st>>>(Mb, sb->masks, db,
                                                                          sb->norb, sb->nocc, Ub);
    FS_CUDA(cudaGetLastError());
  }
  ProfScope ps(sizeof(R) == 4 ? "minor_gemm_f32" : "minor_gemm_f64", st, 2);
  // tmp = psi M_b^T, then psi = M_a tmp
  dim3 g1((unsigned)((db + kTile - 1) / kTile), (unsigned)((da + kTile - 1) / kTile));
  k_cgemm<R, true><<<g1, 256, 0, st>>>((const Cx*)vec, Mb, tmp, (int)da, (int)db, (int)db);
  FS_CUDA(cudaGetLastError());
  k_cgemm<R, false><<<g1, 256, 0, st>>>(Ma, tmp, (Cx*)vec, (int)da, (int)db, (int)da);
  FS_CUDA(cudaGetLastError());
}

bool minor_path_supported(const Space* sa, const Space* sb) {
  return sa->dim <= kMaxMinorDim && sb->dim <= kMaxMinorDim && sa->nocc <= kMinorMaxN &&
         sb->nocc <= kMinorMaxN;
}

void launch_minor_rotation(Ctx* ctx, const Space* sa, const Space* sb, void* vec, int dtype,
                           const CMat& Ua, const CMat& Ub, cudaStream_t st) {
  FS_REQUIRE(minor_path_supported(sa, sb), FS_ERR_UNSUPPORTED,
             "the minor-matrix rotation supports string dimensions up to 4096 and at most "
             "16 electrons per spin");
  if (dtype == FS_C64)
    minor_rotation_tc(ctx, sa, sb, vec, Ua, Ub, st);
  else
    minor_rotation_t<double>(ctx, sa, sb, vec, Ua, Ub, st);
}

}  // namespace fs
