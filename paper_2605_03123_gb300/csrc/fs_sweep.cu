// Givens-rotation sweeps and per-configuration phases.
//
// An orbital rotation of one spin acts on every "vector" of the state that
// holds all strings of that spin: the columns for alpha (dir 0), the rows
// for beta (dir 1).  A slab of KV such vectors is staged in shared memory
// (split over a thread-block cluster when one vector exceeds one SM's shared
// memory), every Givens rotation of the program is applied to it in order
// (§3.2.3: each rotation updates the amplitude pairs (I, I^{p->p+1})), and
// the slab is written back once, multiplied by the configuration phases
// (the diagonal layer of the decomposition, and optionally a fused
// diagonal-Coulomb / number-operator evolution, §3.2.1-§3.2.2).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include <cuda_bf16.h>

#include "fs_common.cuh"
#include "fs_internal.h"
#include "fs_tc.cuh"

namespace cg = cooperative_groups;

namespace fs {

constexpr int kMaxKV = 64;

template <typename R>
struct GProg {
  int m;
  int8_t p[kMaxGivens];
  R c[kMaxGivens];
  R sr[kMaxGivens];
  R si[kMaxGivens];
};

// Subsets of a W-orbital window holding M electrons, in ascending-mask
// order, and for every local adjacent pair (u, u+1) the index pairs
// (S, S') with u in S, u+1 not in S and S' = S - {u} + {u+1}.
__host__ __device__ constexpr int cbinom(int n, int k) {
  if (k < 0 || k > n) return 0;
  int r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
__host__ __device__ constexpr int cpopc(int x) {
  int c = 0;
  while (x) {
    c += x & 1;
    x >>= 1;
  }
  return c;
}
// k-th W-bit mask with M bits set, in ascending order.
__host__ __device__ constexpr int win_mask(int W, int M, int k) {
  for (int x = 0; x < (1 << W); ++x)
    if (cpopc(x) == M && k-- == 0) return x;
  return -1;
}
__host__ __device__ constexpr int win_index(int W, int M, int mask) {
  int k = 0;
  for (int x = 0; x < mask; ++x) k += cpopc(x) == M;
  return k;
}
// The j-th pair (S, S') of local rotation u: S has u and not u+1.
__host__ __device__ constexpr int win_src_mask(int W, int M, int u, int j) {
  for (int x = 0; x < (1 << W); ++x)
    if (cpopc(x) == M && ((x >> u) & 1) && !((x >> (u + 1)) & 1) && j-- == 0) return x;
  return -1;
}
__host__ __device__ constexpr int win_npairs(int W, int M, int u) {
  int n = 0;
  for (int x = 0; x < (1 << W); ++x) n += cpopc(x) == M && ((x >> u) & 1) && !((x >> (u + 1)) & 1);
  return n;
}

template <int W, int M, int U, int J, typename R, int NV, int NS>
__device__ __forceinline__ void win_pair(cx_t<R> (&v)[NV][NS], R c, R sr, R si) {
  constexpr int sm = win_src_mask(W, M, U, J);
  constexpr int a = win_index(W, M, sm);
  constexpr int b = win_index(W, M, sm ^ (1 << U) ^ (1 << (U + 1)));
#pragma unroll
  for (int x = 0; x < NV; ++x) givens2<R>(v[x][a], v[x][b], c, sr, si);
}
template <int W, int M, int U, typename R, int NV, int NS, int... J>
__device__ __forceinline__ void win_pairs_seq(cx_t<R> (&v)[NV][NS], R c, R sr, R si,
                                              std::integer_sequence<int, J...>) {
  (win_pair<W, M, U, J, R, NV, NS>(v, c, sr, si), ...);
}
template <int W, int M, int U, typename R, int NV, int NS>
__device__ __forceinline__ void win_pairs(cx_t<R> (&v)[NV][NS], R c, R sr, R si) {
  if constexpr (U + 1 < W)
    win_pairs_seq<W, M, U, R, NV, NS>(v, c, sr, si,
                                      std::make_integer_sequence<int, win_npairs(W, M, U)>{});
}

template <int W, int M, int K>
__device__ __forceinline__ int win_offset(const uint16_t* Fc) {
  constexpr int mk = win_mask(W, M, K);
  return __ldg(Fc + mk);
}
template <int W, int M, int... K>
__device__ __forceinline__ void win_offsets(const uint16_t* Fc, int (&e)[sizeof...(K)],
                                            std::integer_sequence<int, K...>) {
  ((e[K] = win_offset<W, M, K>(Fc)), ...);
}

// ------------------------------------------- tensor-core window steps
// Per-CTA state of the tensor-core steps (see fs_tc.cuh).
struct TcCtx {
  uint32_t tbase;      // TMEM base of the CTA (lane 0, column 0)
  uint32_t bsm[2];     // shared-memory addresses of the two step-image buffers
  uint32_t mbar_b[2];  // their bulk-copy mbarriers
  uint32_t mbar_mma;   // this warpgroup's MMA-completion mbarrier
  uint32_t ph_mma;     // its next phase parity
  int wg, wq, lane;    // warpgroup, warp within it, lane
  int* status;
};

__device__ __forceinline__ void tc_timeout(int* status) {
  if (status) atomicCAS(status, 0, (int)FS_ERR_TIMEOUT);
}

// Gather-index row length of class M (C(6, M) addresses padded to 8).
template <int M>
constexpr int tc_pad() {
  return (cbinom(tc::kW, M) + 7) / 8 * 8;
}

// One tile of class M: rows [row0, row0 + 128) of the class's rows
// [.., row_end); row = (state s, vector kv, orbit o) with o fastest, and
// orbit o's string addresses are row o of the class's gather indices `ix`
// (shared memory).  Every thread of the warpgroup runs this (the tcgen05
// loads and stores are warp-collective); rows past row_end load zeros and
// store nothing.
template <int M, int CS>
__device__ __forceinline__ void tc_tile(TcCtx& t, int row0, int row_end, int count, int kv_eff,
                                        int KV, size_t st_stride, const uint16_t* ix,
                                        cx_t<float>* const* base, const int (&cbr)[CS + 1],
                                        int buf, uint32_t ph_b, bool& b_ready) {
  using C = cx_t<float>;
  constexpr int NS = cbinom(tc::kW, M);
  constexpr int KP = tc::kp(M);
  constexpr int PAD = tc_pad<M>();
  const uint32_t col0 = t.tbase + (uint32_t)(t.wg * tc::kWgCols);
  const uint32_t lanes = (uint32_t)(t.wq * 32) << 16;
  const int row = row0 + t.wq * 32 + t.lane;
  const bool valid = row < row_end;
  int ad[NS];
  int own[CS > 1 ? NS : 1];
  if (valid) {
    const int per = kv_eff * count;
    const int s = row / per;
    const int rem = row - s * per;
    const int kv = rem / count;
    const int o = rem - kv * count;
    uint32_t w[PAD / 2];
    const uint4* src = reinterpret_cast<const uint4*>(ix + o * PAD);
#pragma unroll
    for (int q = 0; q < PAD / 8; ++q) {
      const uint4 u = src[q];
      w[4 * q] = u.x;
      w[4 * q + 1] = u.y;
      w[4 * q + 2] = u.z;
      w[4 * q + 3] = u.w;
    }
    const int sbase = (int)(s * st_stride) + kv;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int e = (int)((w[k >> 1] >> (16 * (k & 1))) & 0xFFFFu);
      int b0 = 0;
      if constexpr (CS > 1) {
        int r0 = 0;
#pragma unroll
        for (int r = 1; r < CS; ++r)
          if (e >= cbr[r]) {
            r0 = r;
            b0 = cbr[r];
          }
        own[k] = r0;
      }
      ad[k] = sbase + (e - b0) * KV;
    }
  }
  // gather, split, A = [x1 | x2 | x3] into this thread's TMEM lane, 4
  // amplitudes (8 BF16 of K, 4 columns per piece) at a time; padding
  // columns get zeros
  constexpr int AC = tc::a_cols(M);
#pragma unroll
  for (int c = 0; c < AC / 4; ++c) {
    uint32_t p1[4], p2[4], p3[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * c + j;
      C x = mk<float>(0.f, 0.f);
      if (k < NS && valid) x = base[CS > 1 ? own[k < NS ? k : 0] : 0][ad[k < NS ? k : 0]];
      tc::split_bf16x3(x.x, x.y, p1[j], p2[j], p3[j]);
    }
    tc::tmem_st4(col0 + lanes + 4 * c, p1);
    tc::tmem_st4(col0 + lanes + AC + 4 * c, p2);
    tc::tmem_st4(col0 + lanes + 2 * AC + 4 * c, p3);
  }
  tc::wait_st();
  tc::fence_before();
  tc::wg_bar(1 + t.wg);
  if (t.wq == 0 && t.lane == 0) {
    tc::fence_after();
    if (!b_ready) {
      if (!tc::mbar_wait(t.mbar_b[buf], ph_b)) tc_timeout(t.status);
      b_ready = true;
    }
    const uint32_t b0 = t.bsm[buf] + tc::class_offset(M);
    constexpr uint32_t SBO = (KP / 8) * 128;
    constexpr uint32_t ID = tc::idesc(M);
    const uint32_t d = col0 + tc::kPieces * AC;
    // the six products A_i B_j (i + j <= 4 over pieces 1..3), smallest first
    constexpr int kA[6] = {2, 1, 0, 1, 0, 0};
    constexpr int kB[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
    for (int pr = 0; pr < 6; ++pr)
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks) {
        const uint64_t bd = tc::sdesc(b0 + kB[pr] * tc::piece_bytes(M) + ks * 256, 128, SBO);
        tc::mma_bf16(d, col0 + kA[pr] * AC + 8 * ks, bd, ID, (pr > 0 || ks > 0) ? 1u : 0u);
      }
    tc::mma_commit(t.mbar_mma);
  }
  __syncwarp();
  if (!tc::mbar_wait(t.mbar_mma, t.ph_mma)) tc_timeout(t.status);
  t.ph_mma ^= 1u;
  tc::fence_after();
  // D row back to the slab: all loads of the row, one wait, then the stores
  // (which the wait's memory clobber keeps after it)
  constexpr int NC = (2 * NS + 7) / 8;
  uint32_t v[NC][8];
#pragma unroll
  for (int c = 0; c < NC; ++c) tc::tmem_ld8(col0 + lanes + tc::kPieces * AC + 8 * c, v[c]);
  tc::wait_ld();
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * c + j;
      if (k < NS && valid)
        base[CS > 1 ? own[k < NS ? k : 0] : 0][ad[k < NS ? k : 0]] =
            mk<float>(__uint_as_float(v[c][2 * j]), __uint_as_float(v[c][2 * j + 1]));
    }
}

// The tiles of class M (the i-th class of the step) that fall to this
// warpgroup: tiles are numbered across the classes of the step from
// `tile_base` and dealt round-robin over the warpgroups.
template <int M, int CS, int NST>
__device__ __forceinline__ void tc_class(TcCtx& t, const TcSeg& sg, int i, int& ioff,
                                         int& tile_base, bool split_rows, int rank, int kv_eff,
                                         int KV, size_t st_stride, const uint16_t* six,
                                         cx_t<float>* const* base, const int (&cbr)[CS + 1],
                                         int buf, uint32_t ph_b, bool& b_ready) {
  const int count = sg.cnt[i];
  const int rows = NST * kv_eff * count;
  int lo = 0, hi = rows;
  if (CS > 1 && split_rows) {  // rows shared out over the cluster
    lo = (int)((int64_t)rows * rank / CS);
    hi = (int)((int64_t)rows * (rank + 1) / CS);
  }
  const int nt = (hi - lo + tc::kRows - 1) / tc::kRows;
  const uint16_t* ix = six + ioff;
  for (int tl = ((t.wg - tile_base) % tc::kWg + tc::kWg) % tc::kWg; tl < nt; tl += tc::kWg)
    tc_tile<M, CS>(t, lo + tl * tc::kRows, hi, count, kv_eff, KV, st_stride, ix, base, cbr, buf,
                   ph_b, b_ready);
  tile_base += nt;
  ioff += count * tc_pad<M>();
}

// All window steps of a program on the tensor cores, for the CTA's part of
// the slab(s).  `bsm` (128-byte aligned shared memory) holds two step images
// and then two gather-index buffers of g.tc_idx_cap bytes; step st + 1's
// image and indices are copied in while step st runs.  Ends with every
// bulk copy complete and the TMEM freed.
template <int CS, int NST>
__device__ void tc_window_steps(const SweepGeom& g, const WProg<float>& prog,
                                cx_t<float>* const* base, const int (&cbr)[CS + 1], int KV,
                                int kv_eff, size_t st_stride, int rank, unsigned char* bsm) {
  __shared__ __align__(8) uint64_t s_mbar[2 + tc::kWg];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  TcCtx t;
  t.wg = warp >> 2;
  t.wq = warp & 3;
  t.lane = tid & 31;
  t.status = g.status;
  uint16_t* sidx[2] = {reinterpret_cast<uint16_t*>(bsm + 2 * tc::kStepBytes),
                       reinterpret_cast<uint16_t*>(bsm + 2 * tc::kStepBytes + g.tc_idx_cap)};
  if (tid == 0) {
    for (int i = 0; i < 2 + tc::kWg; ++i) tc::mbar_init(tc::smem_u32(&s_mbar[i]), 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&s_tmem), tc::kTmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  t.tbase = s_tmem;
  t.bsm[0] = tc::smem_u32(bsm);
  t.bsm[1] = t.bsm[0] + tc::kStepBytes;
  t.mbar_b[0] = tc::smem_u32(&s_mbar[0]);
  t.mbar_b[1] = tc::smem_u32(&s_mbar[1]);
  t.mbar_mma = tc::smem_u32(&s_mbar[2 + t.wg]);
  t.ph_mma = 0;
  const int nsteps = prog.nsteps;
  // the segment of step st: this rank's orbits when the window is clear of
  // the top orbitals of a blocked cluster, else the whole list
  auto segment = [&](int st, const uint16_t*& idx) -> const TcSeg* {
    const int a = prog.a[st];
    if (CS > 1 && g.blocked && a + tc::kW <= g.norb - g.lgcs) {
      idx = g.tc_idx_grp;
      return g.tc_seg_grp + a * CS + rank;
    }
    idx = g.tc_idx_full;
    return g.tc_seg_full + a;
  };
  auto stage = [&](int st, int b) {  // thread 0: step st's image and indices into buffer b
    const uint16_t* idx;
    const TcSeg* sp = segment(st, idx);
    const int start = __ldg(&sp->start), len = __ldg(&sp->len);
    tc::mbar_expect_tx(t.mbar_b[b], tc::kStepBytes + 2u * (uint32_t)len);
    tc::bulk_g2s(t.bsm[b], g.tc_b + (size_t)st * tc::kStepBytes, tc::kStepBytes, t.mbar_b[b]);
    if (len > 0)
      tc::bulk_g2s(tc::smem_u32(sidx[b]), idx + start, 2u * (uint32_t)len, t.mbar_b[b]);
  };
  if (tid == 0 && nsteps > 0) stage(0, 0);
  for (int st = 0; st < nsteps; ++st) {
    const int buf = st & 1;
    const uint32_t ph_b = (uint32_t)(st >> 1) & 1u;
    if (tid == 0 && st + 1 < nsteps) {  // the other buffer's last readers are done
      // its previous copy (step st - 1) has landed before it is reused
      if (st >= 1 && !tc::mbar_wait(t.mbar_b[buf ^ 1], (uint32_t)((st - 1) >> 1) & 1u))
        tc_timeout(t.status);
      stage(st + 1, buf ^ 1);
    }
    // every thread reads this step's gather indices: wait for them
    if (!tc::mbar_wait(t.mbar_b[buf], ph_b)) tc_timeout(t.status);
    bool b_ready = true;
    const uint16_t* idx_unused;
    const TcSeg sg = *segment(st, idx_unused);
    const bool split_rows = !(CS > 1 && g.blocked && prog.a[st] + tc::kW <= g.norb - g.lgcs);
    int ioff = 0, tile_base = 0;
    tc_class<3, CS, NST>(t, sg, 0, ioff, tile_base, split_rows, rank, kv_eff, KV, st_stride, sidx[buf], base, cbr, buf, ph_b, b_ready);
    tc_class<2, CS, NST>(t, sg, 1, ioff, tile_base, split_rows, rank, kv_eff, KV, st_stride, sidx[buf], base, cbr, buf, ph_b, b_ready);
    tc_class<4, CS, NST>(t, sg, 2, ioff, tile_base, split_rows, rank, kv_eff, KV, st_stride, sidx[buf], base, cbr, buf, ph_b, b_ready);
    tc_class<1, CS, NST>(t, sg, 3, ioff, tile_base, split_rows, rank, kv_eff, KV, st_stride, sidx[buf], base, cbr, buf, ph_b, b_ready);
    tc_class<5, CS, NST>(t, sg, 4, ioff, tile_base, split_rows, rank, kv_eff, KV, st_stride, sidx[buf], base, cbr, buf, ph_b, b_ready);
    if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();
  }
  // every bulk copy has landed (the buffers become the epilogue's tables),
  // then the TMEM is freed
  if (tid == 0 && nsteps > 0) {
    for (int b = 0; b < 2 && b < nsteps; ++b) {
      const int lst = ((nsteps - 1) & 1) == b ? nsteps - 1 : nsteps - 2;  // last step using b
      if (!tc::mbar_wait(t.mbar_b[b], (uint32_t)(lst >> 1) & 1u)) tc_timeout(t.status);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(t.tbase, tc::kTmemCols);
  }
}

// The B images of the tensor-core steps of one program, FP64 on the device:
// per step, V = G_k ... G_1 (the step's Givens rotations in the window's
// local orbitals, applied first to last), then for each class m the
// compound matrix C_m(V)[S', S] = det V[S', S] in its real form
// [[Re, -Im], [Im, Re]] (rows n = output reals, columns k = input reals,
// re/im interleaved), split into three BF16 pieces (each the nearest BF16
// of the remainder so far), K-major core matrices (see tc::b_offset).  One
// block per step.
__global__ void __launch_bounds__(256)
    k_tc_bmats(const __grid_constant__ WProg<double> p, unsigned char* out) {
  __shared__ double2 V[tc::kW * tc::kW];
  const int st = blockIdx.x;
  unsigned char* img = out + (size_t)st * tc::kStepBytes;
  for (int i = threadIdx.x; i < tc::kStepBytes / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(img)[i] = 0u;
  if (threadIdx.x == 0) {
    for (int i = 0; i < tc::kW; ++i)
      for (int j = 0; j < tc::kW; ++j) V[i * tc::kW + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    for (int q = p.g0[st]; q < p.g0[st + 1]; ++q) {
      const int u = p.u[q];
      const double c = p.c[q], sr = p.sr[q], si = p.si[q];
      for (int j = 0; j < tc::kW; ++j) {
        const double2 x = V[u * tc::kW + j], y = V[(u + 1) * tc::kW + j];
        // row u <- c x + s y, row u+1 <- -conj(s) x + c y
        V[u * tc::kW + j] = make_double2(c * x.x + sr * y.x - si * y.y, c * x.y + sr * y.y + si * y.x);
        V[(u + 1) * tc::kW + j] =
            make_double2(-(sr * x.x + si * x.y) + c * y.x, -(sr * x.y - si * x.x) + c * y.y);
      }
    }
  }
  __syncthreads();
  for (int m = 1; m < tc::kW; ++m) {
    const int ns = tc::binom6(m), kpad = tc::kp(m);
    for (int idx = threadIdx.x; idx < ns * ns; idx += blockDim.x) {
      const int ip = idx / ns, iq = idx - ip * ns;
      const int rm = win_mask(tc::kW, m, ip), cm = win_mask(tc::kW, m, iq);
      double2 a[5 * 5];
      int r = 0;
      for (int i = 0; i < tc::kW; ++i) {
        if (!((rm >> i) & 1)) continue;
        int cc = 0;
        for (int j = 0; j < tc::kW; ++j)
          if ((cm >> j) & 1) a[r * m + (cc++)] = V[i * tc::kW + j];
        ++r;
      }
      // det by Gaussian elimination with partial pivoting
      double dr = 1, di = 0;
      for (int k = 0; k < m; ++k) {
        int piv = k;
        double best = hypot(a[k * m + k].x, a[k * m + k].y);
        for (int i = k + 1; i < m; ++i) {
          const double h = hypot(a[i * m + k].x, a[i * m + k].y);
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
          for (int j = 0; j < m; ++j) {
            const double2 tmp = a[k * m + j];
            a[k * m + j] = a[piv * m + j];
            a[piv * m + j] = tmp;
          }
          dr = -dr;
          di = -di;
        }
        const double2 pk = a[k * m + k];
        const double nr = dr * pk.x - di * pk.y;
        di = dr * pk.y + di * pk.x;
        dr = nr;
        const double inv = 1.0 / (pk.x * pk.x + pk.y * pk.y);
        for (int i = k + 1; i < m; ++i) {
          const double2 x = a[i * m + k];
          const double fr = (x.x * pk.x + x.y * pk.y) * inv, fi = (x.y * pk.x - x.x * pk.y) * inv;
          for (int j = k + 1; j < m; ++j) {
            const double2 y = a[k * m + j];
            a[i * m + j].x -= fr * y.x - fi * y.y;
            a[i * m + j].y -= fr * y.y + fi * y.x;
          }
        }
      }
      const double ent[4] = {dr, -di, di, dr};  // (2ip, 2iq), (2ip, 2iq+1), (2ip+1, 2iq), (2ip+1, 2iq+1)
      for (int e = 0; e < 4; ++e) {
        const int n = 2 * ip + (e >> 1), k = 2 * iq + (e & 1);
        const int off = tc::b_offset(n, k, kpad);
        double r = ent[e];
        for (int pc = 0; pc < tc::kPieces; ++pc) {  // nearest BF16 of the remainder
          const __nv_bfloat16 b = __float2bfloat16_rn((float)r);
          *reinterpret_cast<__nv_bfloat16*>(img + tc::class_offset(m) + pc * tc::piece_bytes(m) + off) = b;
          r -= (double)__bfloat162float(b);
        }
      }
    }
  }
}

// One orbit of a window step: the C(W, M) strings sharing the occupation
// outside the window.  Their addresses are R_O + F[c_lo][S]; every vector of
// the slab is rotated in registers by the step's Givens rotations.
template <typename R, int CS, int NST, int W, int M>
__device__ __forceinline__ void win_orbit(uint32_t desc, const uint16_t* F, cx_t<R>* const* base,
                                          size_t st_stride, const int (&cbr)[CS + 1], int KV,
                                          int kv_eff, const WProg<R>& prog, int ga, int gb) {
  using C = cx_t<R>;
  constexpr int NS = cbinom(W, M);
  const int RO = desc & 0xFFFF, clo = (desc >> 16) & 0xFF;
  const uint16_t* Fc = F + (clo << W);
  // element offsets (and, in a cluster, the owning CTA) of the orbit
  int ad[NS];
  int own[CS > 1 ? NS : 1];
  win_offsets<W, M>(Fc, ad, std::make_integer_sequence<int, NS>{});
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    int e = RO + ad[k];
    if constexpr (CS > 1) {
      int o = 0, b0 = 0;
#pragma unroll
      for (int r = 1; r < CS; ++r)
        if (e >= cbr[r]) {
          o = r;
          b0 = cbr[r];
        }
      own[k] = o;
      ad[k] = (e - b0) * KV;
    } else {
      ad[k] = e * KV;
    }
  }
  for (int kv = 0; kv < kv_eff; ++kv) {
    C v[NST][NS];
#pragma unroll
    for (int x = 0; x < NST; ++x)
#pragma unroll
      for (int k = 0; k < NS; ++k)
        v[x][k] = base[CS > 1 ? own[k] : 0][x * st_stride + ad[k] + kv];
    for (int q = ga; q < gb; ++q) {
      const R c = prog.c[q], sr = prog.sr[q], si = prog.si[q];
      switch (prog.u[q]) {
        case 0: win_pairs<W, M, 0, R, NST, NS>(v, c, sr, si); break;
        case 1: win_pairs<W, M, 1, R, NST, NS>(v, c, sr, si); break;
        case 2: win_pairs<W, M, 2, R, NST, NS>(v, c, sr, si); break;
        case 3: win_pairs<W, M, 3, R, NST, NS>(v, c, sr, si); break;
        case 4: win_pairs<W, M, 4, R, NST, NS>(v, c, sr, si); break;
        case 5: win_pairs<W, M, 5, R, NST, NS>(v, c, sr, si); break;
        case 6: win_pairs<W, M, 6, R, NST, NS>(v, c, sr, si); break;
        default: break;
      }
    }
#pragma unroll
    for (int x = 0; x < NST; ++x)
#pragma unroll
      for (int k = 0; k < NS; ++k)
        base[CS > 1 ? own[k] : 0][x * st_stride + ad[k] + kv] = v[x][k];
  }
}

// ------------------------------------------------ transition reduction
// One orbit of a transition pass: the C(4, M) strings O u S for the
// subset Q = {q_0 < .. < q_3}.  For every local pair (a, b) with b in S and
// a not in S, a^dag_{q_a} a_{q_b} maps S to S' = S - b + a with the sign
// (-1)^(#occupied orbitals strictly between q_a and q_b): the part inside Q
// is a compile-time constant, the part from O is folded into the loaded
// amplitudes (omega(S) = prod over j in S of (-1)^{G_j}, G_j the parity of
// O between q_0 and q_j, so omega(S) omega(S') is the O parity of the pair).
// acc[2 (a*4 + b)], acc[2 (a*4 + b) + 1] += Re, Im of conj(g[S']) psi[S].
template <typename R, int M, int J, int NS>
__device__ __forceinline__ void t_term(const cx_t<R> (&ps)[NS], const cx_t<R> (&pg)[NS],
                                       R (&acc)[32], uint32_t keep) {
  constexpr int k = J / 16, a = (J / 4) % 4, b = J % 4;
  if constexpr (k < NS) {
    constexpr int S = win_mask(4, M, k);
    constexpr int slot = a * 4 + b;
    if constexpr ((S >> b) & 1) {
      if constexpr (a == b) {
        if (keep & (1u << slot)) {  // uniform per pass: diagonals are owned once
          acc[2 * slot] = fma(pg[k].x, ps[k].x, fma(pg[k].y, ps[k].y, acc[2 * slot]));
          acc[2 * slot + 1] = fma(pg[k].x, ps[k].y, fma(-pg[k].y, ps[k].x, acc[2 * slot + 1]));
        }
      } else if constexpr (!((S >> a) & 1)) {
        constexpr int k2 = win_index(4, M, S ^ (1 << a) ^ (1 << b));
        constexpr int lo = a < b ? a : b, hi = a < b ? b : a;
        constexpr bool neg = cpopc(S & ((1 << hi) - 1) & ~((2 << lo) - 1)) & 1;
        constexpr R sg = neg ? R(-1) : R(1);
        if (keep & (1u << slot)) {  // uniform per pass: each pair is owned once
          // acc += sg * conj(g[k2]) * psi[k], as four fused multiply-adds
          const R gx = sg * pg[k2].x, gy = sg * pg[k2].y;
          acc[2 * slot] = fma(gx, ps[k].x, fma(gy, ps[k].y, acc[2 * slot]));
          acc[2 * slot + 1] = fma(gx, ps[k].y, fma(-gy, ps[k].x, acc[2 * slot + 1]));
        }
      }
    }
  }
}
template <typename R, int M, int NS, int... J>
__device__ __forceinline__ void t_terms(const cx_t<R> (&ps)[NS], const cx_t<R> (&pg)[NS],
                                        R (&acc)[32], uint32_t keep,
                                        std::integer_sequence<int, J...>) {
  (t_term<R, M, J, NS>(ps, pg, acc, keep), ...);
}
template <int M, int K>
__device__ __forceinline__ int t_flip(int gb) {
  constexpr int S = win_mask(4, M, K);
  int f = 0;
#pragma unroll
  for (int j = 1; j < 4; ++j)
    if ((S >> j) & 1) f ^= (gb >> j) & 1;
  return f;
}
template <int M, int... K>
__device__ __forceinline__ void t_flips(int gb, int (&fl)[sizeof...(K)],
                                        std::integer_sequence<int, K...>) {
  ((fl[K] = t_flip<M, K>(gb)), ...);
}
template <typename R, int CS, int M>
__device__ __forceinline__ void t_orbit(const TRecord& rc, cx_t<R>* const* base, size_t st_stride,
                                        const int (&cbr)[CS + 1], int KV, int kv_eff,
                                        R (&acc)[32], uint32_t keep) {
  using C = cx_t<R>;
  constexpr int NS = cbinom(4, M);
  int ad[NS], own[CS > 1 ? NS : 1];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int e = rc.addr[k];
    if constexpr (CS > 1) {
      int o = 0, b0 = 0;
#pragma unroll
      for (int r = 1; r < CS; ++r)
        if (e >= cbr[r]) {
          o = r;
          b0 = cbr[r];
        }
      own[k] = o;
      ad[k] = (e - b0) * KV;
    } else {
      ad[k] = e * KV;
    }
  }
  int fl[NS];
  t_flips<M>(rc.gbits, fl, std::make_integer_sequence<int, NS>{});
  for (int kv = 0; kv < kv_eff; ++kv) {
    C ps[NS], pg[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      C* b0 = base[CS > 1 ? own[k] : 0];
      ps[k] = b0[ad[k] + kv];
      pg[k] = b0[st_stride + ad[k] + kv];
      if (fl[k]) {
        ps[k].x = -ps[k].x;
        ps[k].y = -ps[k].y;
        pg[k].x = -pg[k].x;
        pg[k].y = -pg[k].y;
      }
    }
    t_terms<R, M, NS>(ps, pg, acc, keep, std::make_integer_sequence<int, 6 * 16>{});
  }
}

// Warp reduction of 32 values by recursive halving: afterwards lane l holds
// the sum over the warp of value l.
template <typename R>
__device__ __forceinline__ R warp_transpose_sum(R (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const bool up = lane & s;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const R send = up ? v[i] : v[i + s];
      const R keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, s);
    }
  }
  return v[0];
}

// Items [lo, hi) (classes of equal work, in descending order of work, each
// a multiple of 32 long) are dealt in chunks of 32: chunk c goes to cluster
// rank c % cs, and a rank's chunks go to its NT / 32 warps round by round,
// in warp order on even rounds and in reverse order on odd rounds, so the
// work evens out over ranks and warps and no warp mixes two classes.
// Item of round R for thread t of rank `rank`, or -1 past the end; rounds
// run while dealt_round<NT>(lo, hi, R, rank, cs).
template <int NT>
__device__ __forceinline__ int dealt_item(int lo, int hi, int R, int t, int rank, int cs) {
  constexpr int NW = NT / 32;
  const int w = t >> 5;
  const int k = R * NW + ((R & 1) ? NW - 1 - w : w);
  const int o = lo + 32 * (rank + cs * k) + (t & 31);
  return o < hi ? o : -1;
}
template <int NT>
__device__ __forceinline__ bool dealt_round(int lo, int hi, int R, int rank, int cs) {
  return lo + 32 * (rank + cs * R * (NT / 32)) < hi;
}

template <typename R, int W, bool WIN>
struct ProgOf {
  using type = GProg<R>;
};
template <typename R, int W>
struct ProgOf<R, W, true> {
  using type = WProg<R>;
};


// Cross-term tables for the slab vectors o = v0 .. v0+nv-1 (other-spin
// strings): w[kv][x] = sum_{y in I_o} X[y][x] (this = beta) or X[x][y]
// (this = alpha), and tab[kv][c][v] = exp(i sum_{bits b of v} w[kv][8c + b]).
// Ends with a block barrier.
template <typename R>
__device__ void build_cross_tables(const SweepGeom& g, const Mat& X, int v0, int nv,
                                   double* w, cx_t<R>* tab, int tid, int nthr) {
  for (int idx = tid; idx < nv * g.norb; idx += nthr) {
    int kv = idx / g.norb, x = idx - kv * g.norb;
    double s = 0;
    uint32_t m = g.masks_other[v0 + kv];
    while (m) {
      int y = __ffs(m) - 1;
      m &= m - 1;
      s += g.dir == 1 ? X.v[y * g.norb + x] : X.v[x * g.norb + y];
    }
    w[kv * kMaxOrb + x] = s;
  }
  __syncthreads();
  const int per = g.nchunk * 256;
  for (int idx = tid; idx < nv * per; idx += nthr) {
    int kv = idx / per, e = idx - kv * per;
    int c = e >> 8, v = e & 255;
    double s = 0;
    while (v) {
      int b = __ffs(v) - 1;
      v &= v - 1;
      int x = 8 * c + b;
      if (x < g.norb) s += w[kv * kMaxOrb + x];
    }
    tab[idx] = expi<R>(s);
  }
  __syncthreads();
}

// Asynchronous copy of one complex element from global to shared memory
// (8 bytes for complex64, 16 for complex128; both addresses aligned to the
// element size).
__device__ __forceinline__ void cp_async_elem(cx_t<float>* dst, const cx_t<float>* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(cx_t<double>* dst, const cx_t<double>* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

template <typename R>
__device__ __forceinline__ cx_t<R> ld_ea(const void* p, int64_t i) {
  if (!p) return mk<R>(1, 0);
  return reinterpret_cast<const cx_t<R>*>(p)[i];
}

// W == 0: one shared-memory pass per Givens rotation (pair lists);
// W > 0: one pass per window step, orbits rotated in registers.
// One slab of a sweep (see launch_sweep): load, Givens rotations, epilogue.
// NT threads per CTA.  SPLIT (two states, no cluster): during the Givens
// phase the first half of the CTA rotates state 0 and the second half state
// 1, each half synchronising on its own named barrier.
template <typename R, int CS, int NST, bool VJP, int W, int NT, bool SPLIT, typename P,
          bool TC = false>
__device__ __forceinline__ void sweep_body(const SweepGeom& g, const P& prog, const Mat& X,
                                           const int slab, const int rank,
                                           unsigned char* smraw) {
  static_assert(!VJP || NST == 2, "reverse mode carries two states");
  static_assert(!SPLIT || (NST == 2 && W > 0), "split mode: two states, window sweeps");
  constexpr int kThreads = NT;
  using C = cx_t<R>;
  C* sm = reinterpret_cast<C*>(smraw);
  const int KV = 1 << g.lgKV;
  const int v0 = slab * KV;
  const int kv_eff = min(KV, g.nvec - v0);
  // element ranges of the cluster ranks (registers; rank is runtime)
  int cbr[CS + 1];
#pragma unroll
  for (int r = 0; r <= CS; ++r) cbr[r] = g.cb[r];
  int e0 = 0, e1 = cbr[CS];
#pragma unroll
  for (int r = 0; r < CS; ++r)
    if (r == rank) {
      e0 = cbr[r];
      e1 = cbr[r + 1];
    }
  const int nel = max(0, e1 - e0);
  const int tid = threadIdx.x;
  const size_t st_stride = (size_t)g.chunk * KV;  // elements per state
  C* tab = sm + NST * st_stride;                  // cross tables, KV sets
  double* w = reinterpret_cast<double*>(tab + (g.has_x ? ((size_t)g.nchunk * 256 << g.lgKV) : 0));

  C* base[CS];
  if constexpr (CS > 1) {
    cg::cluster_group cl = cg::this_cluster();
    for (int r = 0; r < CS; ++r) base[r] = cl.map_shared_rank(sm, r);
  } else {
    base[0] = sm;
  }

  // ---- load this CTA's part of the slab: asynchronous element copies
  //      straight into shared memory (no register round trip, so the strided
  //      column gathers of an alpha slab all overlap)
  for (int s = 0; s < NST; ++s) {
    const C* gs = reinterpret_cast<const C*>(g.st[s]);
    C* ss = sm + s * st_stride;
    if (g.dir == 1) {
      for (int idx = tid; idx < kv_eff * nel; idx += kThreads) {
        int kv = idx / nel, el = idx - kv * nel;
        cp_async_elem(ss + (size_t)el * KV + kv, gs + (int64_t)(v0 + kv) * g.d_b + e0 + el);
      }
    } else {
      for (int idx = tid; idx < (nel << g.lgKV); idx += kThreads) {
        int el = idx >> g.lgKV, kv = idx & (KV - 1);
        if (kv < kv_eff)
          cp_async_elem(ss + (size_t)el * KV + kv, gs + (int64_t)(e0 + el) * g.d_b + v0 + kv);
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();

  // ---- Givens rotations, in program order
  if constexpr (TC) {
    static_assert(W == tc::kW && NT == tc::kThreads && !SPLIT && sizeof(R) == 4,
                  "tensor-core steps: complex64, W = 6, 512 threads");
    // the step images go after the slab(s), 128-byte aligned; the epilogue's
    // tables reuse that space afterwards
    const uint32_t s0 = tc::smem_u32(smraw);
    const uint32_t sb = s0 + (uint32_t)(NST * st_stride * sizeof(C));
    unsigned char* bsm = smraw + (((sb + 127u) & ~127u) - s0);
    tc_window_steps<CS, NST>(g, prog, base, cbr, KV, kv_eff, st_stride, rank, bsm);
  } else if constexpr (W == 0) {
    const int items = g.npp << g.lgKV;
    const int per = (items + CS - 1) / CS;
    const int lo = rank * per, hi = min(items, lo + per);
    for (int k = 0; k < prog.m; ++k) {
      const uint32_t* list = g.pairs + (int64_t)prog.p[k] * g.npp;
      const R c = prog.c[k], sr = prog.sr[k], si = prog.si[k];
      for (int it = lo + tid; it < hi; it += kThreads) {
        int t = it >> g.lgKV, kv = it & (KV - 1);
        if (kv >= kv_eff) continue;
        uint32_t pr = __ldg(list + t);
        int src = pr & 0xFFFF, dst = pr >> 16;
        int os = 0, od = 0, bs0 = 0, bd0 = 0;
        if constexpr (CS > 1) {
  #pragma unroll
          for (int r = 1; r < CS; ++r) {
            if (src >= cbr[r]) {
              os = r;
              bs0 = cbr[r];
            }
            if (dst >= cbr[r]) {
              od = r;
              bd0 = cbr[r];
            }
          }
        }
        size_t ls = (size_t)(src - bs0) * KV + kv;
        size_t ld = (size_t)(dst - bd0) * KV + kv;
  #pragma unroll
        for (int s = 0; s < NST; ++s) {
          C* ps = base[os] + s * st_stride + ls;
          C* pd = base[od] + s * st_stride + ld;
          C x = *ps, y = *pd;
          givens2<R>(x, y, c, sr, si);
          *ps = x;
          *pd = y;
        }
      }
      if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    }
  } else if constexpr (SPLIT) {
    // half h of every CTA rotates state h (one state per thread: the wider
    // single-state window fits the registers).  In one CTA each half meets
    // on its own named barrier 1 + h; in a cluster every step ends with the
    // cluster barrier.
    constexpr int HT = NT / 2;
    const int half = tid / HT, ltid = tid - half * HT;
    C* bs[CS];
#pragma unroll
    for (int r = 0; r < CS; ++r) bs[r] = base[r] + half * st_stride;
    for (int st = 0; st < prog.nsteps; ++st) {
      const int a = prog.a[st];
      const int ga = prog.g0[st], gb = prog.g0[st + 1];
      const int o0 = g.orb_off[a], o1 = g.orb_off[a + 1];
      const uint16_t* F = g.offs + (size_t)a * g.offs_stride;
      int lo = o0, hi = o1, drank = 0, dcs = 1;
      const uint32_t* olist = g.orbits;
      if constexpr (CS > 1) {
        if (g.blocked && a + W <= g.norb - g.lgcs) {
          olist = g.orb_grp;
          lo = __ldg(g.orb_goff + a * 9 + rank);
          hi = __ldg(g.orb_goff + a * 9 + rank + 1);
        } else {
          drank = rank;
          dcs = CS;
        }
      }
      for (int rd = 0; dealt_round<HT>(lo, hi, rd, drank, dcs); ++rd) {
        const int o = dealt_item<HT>(lo, hi, rd, ltid, drank, dcs);
        if (o < 0) continue;
        const uint32_t desc = __ldg(olist + o);
        switch (desc >> 24) {
          case 1: win_orbit<R, CS, 1, W, 1>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 2: win_orbit<R, CS, 1, W, 2>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 3: win_orbit<R, CS, 1, W, 3>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 4: if constexpr (W > 4) win_orbit<R, CS, 1, W, 4>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 5: if constexpr (W > 5) win_orbit<R, CS, 1, W, 5>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          default: break;
        }
      }
      if constexpr (CS > 1)
        cg::this_cluster().sync();
      else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "r"(HT) : "memory");
    }
    if constexpr (CS == 1) __syncthreads();
  } else {
    for (int st = 0; st < prog.nsteps; ++st) {
      const int a = prog.a[st];
      const int ga = prog.g0[st], gb = prog.g0[st + 1];
      const int o0 = g.orb_off[a], o1 = g.orb_off[a + 1];
      const uint16_t* F = g.offs + (size_t)a * g.offs_stride;
      int lo = o0, hi = o1, drank = rank, dcs = CS;
      const uint32_t* olist = g.orbits;
      if (CS > 1 && g.blocked && a + W <= g.norb - g.lgcs) {
        // window clear of the top orbitals: this rank's own orbits
        olist = g.orb_grp;
        lo = __ldg(g.orb_goff + a * 9 + rank);
        hi = __ldg(g.orb_goff + a * 9 + rank + 1);
        drank = 0;
        dcs = 1;
      }
      for (int rd = 0; dealt_round<kThreads>(lo, hi, rd, drank, dcs); ++rd) {
        const int o = dealt_item<kThreads>(lo, hi, rd, tid, drank, dcs);
        if (o < 0) continue;
        const uint32_t desc = __ldg(olist + o);
        switch (desc >> 24) {
          case 1: win_orbit<R, CS, NST, W, 1>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 2: win_orbit<R, CS, NST, W, 2>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 3: win_orbit<R, CS, NST, W, 3>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 4: if constexpr (W > 4) win_orbit<R, CS, NST, W, 4>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          case 5: if constexpr (W > 5) win_orbit<R, CS, NST, W, 5>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb); break;
          default: break;
        }
      }
      if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    }
  }

  const int tper = g.nchunk * 256;
  if constexpr (!VJP) {
    // ---- epilogue: phases, store
    if (g.has_x) build_cross_tables<R>(g, X, v0, kv_eff, w, tab, tid, kThreads);
    const int tot = g.dir == 1 ? kv_eff * nel : (nel << g.lgKV);
    for (int idx = tid; idx < tot; idx += kThreads) {
      int kv, el;
      if (g.dir == 1) {
        kv = idx / nel;
        el = idx - kv * nel;
      } else {
        el = idx >> g.lgKV;
        kv = idx & (KV - 1);
        if (kv >= kv_eff) continue;
      }
      const int o = v0 + kv, e = e0 + el;
      C f = cmul<R>(ld_ea<R>(g.ea_other, o), ld_ea<R>(g.ea_this, e));
      if (g.has_x) {
        uint32_t m = __ldg(g.masks_this + e);
        const C* tk = tab + kv * tper;
        for (int c = 0; c < g.nchunk; ++c) f = cmul<R>(f, tk[c * 256 + ((m >> (8 * c)) & 255)]);
      }
#pragma unroll
      for (int s = 0; s < NST; ++s) {
        C v = cmul<R>(f, sm[s * st_stride + (size_t)el * KV + kv]);
        C* gs = reinterpret_cast<C*>(g.st[s]);
        if (g.dir == 1)
          gs[(int64_t)o * g.d_b + e] = v;
        else
          gs[(int64_t)e * g.d_b + o] = v;
      }
    }
  } else {
    // ---- reverse-mode epilogue
    // (a) the diagonal layer of the (inverse) rotation, in shared memory
    for (int idx = tid; idx < (nel << g.lgKV); idx += kThreads) {
      int el = idx >> g.lgKV, kv = idx & (KV - 1);
      if (kv >= kv_eff) continue;
      C f = cmul<R>(ld_ea<R>(g.ea_other, v0 + kv), ld_ea<R>(g.ea_this, e0 + el));
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        C* q = sm + s * st_stride + (size_t)el * KV + kv;
        *q = cmul<R>(f, *q);
      }
    }
    if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    // (b) T[p][q] += sum over the slab of sign * conj(g[dst]) * psi[src] for
    //     every pair (src, dst = src^{q->p}) of the E_pq list of this spin
    if (g.T && g.npass > 0) {
      // subset passes: per-thread partial sums of the 16 local slots, one
      // warp reduction per pass, per-CTA sums in shared memory
      R* tsm = reinterpret_cast<R*>(w + (g.has_x ? (kMaxOrb << g.lgKV) : 0));
      for (int i = tid; i < g.npass * 32; i += kThreads) tsm[i] = 0;
      __syncthreads();
      const int lane = tid & 31;
      for (int ip = 0; ip < g.npass; ++ip) {
        const TPassDev pd = g.tpass[ip];
        R acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0;
        int lo = pd.rec0, hi = pd.rec1, drank = rank, dcs = CS;
        const TRecord* rlist = g.trec;
        if (CS > 1 && g.blocked && pd.q[3] < g.norb - g.lgcs) {
          // subset clear of the top orbitals: this rank's own records
          rlist = g.trec_grp;
          lo = __ldg(g.tgoff + ip * 9 + rank);
          hi = __ldg(g.tgoff + ip * 9 + rank + 1);
          drank = 0;
          dcs = 1;
        }
        for (int rd = 0; dealt_round<kThreads>(lo, hi, rd, drank, dcs); ++rd) {
          const int o = dealt_item<kThreads>(lo, hi, rd, tid, drank, dcs);
          if (o < 0) continue;
          TRecord rc;
          *reinterpret_cast<uint4*>(&rc) = __ldg(reinterpret_cast<const uint4*>(rlist + o));
          switch (rc.m) {
            case 1: t_orbit<R, CS, 1>(rc, base, st_stride, cbr, KV, kv_eff, acc, pd.keep); break;
            case 2: t_orbit<R, CS, 2>(rc, base, st_stride, cbr, KV, kv_eff, acc, pd.keep); break;
            case 3: t_orbit<R, CS, 3>(rc, base, st_stride, cbr, KV, kv_eff, acc, pd.keep); break;
            case 4: t_orbit<R, CS, 4>(rc, base, st_stride, cbr, KV, kv_eff, acc, pd.keep); break;
            default: break;
          }
        }
        const R v = warp_transpose_sum<R>(acc, lane);
        if (pd.keep & (1u << (lane >> 1))) atomicAdd(tsm + ip * 32 + lane, v);
      }
      __syncthreads();
      for (int i = tid; i < g.npass * 32; i += kThreads) {
        const TPassDev pd = g.tpass[i >> 5];
        const int slot = (i & 31) >> 1;
        if (!(pd.keep & (1u << slot))) continue;
        const int p = pd.q[slot >> 2], q = pd.q[slot & 3];
        atomicAdd(g.T + 2 * (p * g.norb + q) + (i & 1), (double)tsm[i]);
      }
    } else if (g.T) {
      const int lane = tid & 31;
      const int nw = (g.nx + 31) / 32;
      const int gw = rank * (kThreads / 32) + (tid >> 5);
      const int nlist = g.norb * g.norb;
      for (int L = gw; L < nlist; L += CS * (kThreads / 32)) {
        const int cnt = g.xcount[L];
        const uint32_t* lp = g.xpairs + (int64_t)L * g.nx;
        const uint32_t* ls = g.xsign + (int64_t)L * nw;
        R ar = 0, ai = 0;
        // four list entries per lane in flight: the loads of the pair list
        // (L2) are independent of the shared-memory arithmetic
        constexpr int U4 = 4;
        for (int t0 = 0; t0 < cnt; t0 += 32 * U4) {
          uint32_t pr[U4], sw[U4];
#pragma unroll
          for (int u = 0; u < U4; ++u) {
            const int t = t0 + u * 32 + lane;
            pr[u] = t < cnt ? __ldg(lp + t) : 0u;
            sw[u] = t < cnt ? __ldg(ls + (t >> 5)) : 0u;
          }
#pragma unroll
          for (int u = 0; u < U4; ++u) {
            const int t = t0 + u * 32 + lane;
            if (t >= cnt) continue;
            const uint32_t sb = (sw[u] >> (t & 31)) & 1u;
            const int src = pr[u] & 0xFFFF, dst = pr[u] >> 16;
            int os = 0, od = 0, bs0 = 0, bd0 = 0;
            if constexpr (CS > 1) {
#pragma unroll
              for (int r = 1; r < CS; ++r) {
                if (src >= cbr[r]) {
                  os = r;
                  bs0 = cbr[r];
                }
                if (dst >= cbr[r]) {
                  od = r;
                  bd0 = cbr[r];
                }
              }
            }
            const C* ps = base[os] + (size_t)(src - bs0) * KV;
            const C* pg = base[od] + st_stride + (size_t)(dst - bd0) * KV;
            R br = 0, bi = 0;
            for (int kv = 0; kv < kv_eff; ++kv) {
              C a = ps[kv], b = pg[kv];
              br = fma(b.x, a.x, fma(b.y, a.y, br));
              bi = fma(b.x, a.y, fma(-b.y, a.x, bi));
            }
            if (sb) {
              br = -br;
              bi = -bi;
            }
            ar += br;
            ai += bi;
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          ar += __shfl_xor_sync(0xFFFFFFFFu, ar, off);
          ai += __shfl_xor_sync(0xFFFFFFFFu, ai, off);
        }
        if (lane == 0) {
          atomicAdd(g.T + 2 * L, (double)ar);
          atomicAdd(g.T + 2 * L + 1, (double)ai);
        }
      }
    }
    // (c) W = Im(conj(g) psi) (invariant under the diagonal gate that
    //     follows), then the second phase, then store both states
    if (g.has_x) build_cross_tables<R>(g, X, v0, kv_eff, w, tab, tid, kThreads);
    const int tot = g.dir == 1 ? kv_eff * nel : (nel << g.lgKV);
    for (int idx = tid; idx < tot; idx += kThreads) {
      int kv, el;
      if (g.dir == 1) {
        kv = idx / nel;
        el = idx - kv * nel;
      } else {
        el = idx >> g.lgKV;
        kv = idx & (KV - 1);
        if (kv >= kv_eff) continue;
      }
      const int o = v0 + kv, e = e0 + el;
      const int64_t gi = g.dir == 1 ? (int64_t)o * g.d_b + e : (int64_t)e * g.d_b + o;
      C ps = sm[(size_t)el * KV + kv];
      C pg = sm[st_stride + (size_t)el * KV + kv];
      if (g.W) reinterpret_cast<R*>(g.W)[gi] = pg.x * ps.y - pg.y * ps.x;
      C f = cmul<R>(ld_ea<R>(g.ea2_other, o), ld_ea<R>(g.ea2_this, e));
      if (g.has_x) {
        uint32_t m = __ldg(g.masks_this + e);
        const C* tk = tab + kv * tper;
        for (int c = 0; c < g.nchunk; ++c) f = cmul<R>(f, tk[c * 256 + ((m >> (8 * c)) & 255)]);
      }
      reinterpret_cast<C*>(g.st[0])[gi] = cmul<R>(f, ps);
      reinterpret_cast<C*>(g.st[1])[gi] = cmul<R>(f, pg);
    }
    // remote CTAs may still read this CTA's shared memory in (b)
    if constexpr (CS > 1) cg::this_cluster().sync();
  }
}

template <typename R, int CS, int NST, bool VJP, int W, int NT, bool SPLIT, bool TC = false>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
    k_sweep(const SweepGeom g, const __grid_constant__ typename ProgOf<R, W, (W > 0)>::type prog,
            const __grid_constant__ Mat X) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  sweep_body<R, CS, NST, VJP, W, NT, SPLIT, typename ProgOf<R, W, (W > 0)>::type, TC>(
      g, prog, X, blockIdx.x / CS, rank, smraw);
}

// Batched sweep: one persistent launch over the slabs of many jobs (one job
// per circuit), taken from an atomic work counter in job order.
template <typename R, int NST, bool VJP, int W, int NT, bool SPLIT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
    k_sweep_batch(const SweepJob* jobs, int njobs, int total, int* counter) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_item, s_job;
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(counter, 1);
      int lo = 0, hi = njobs - 1;
      while (lo < hi) {  // last job with item0 <= it
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].item0 <= it) lo = mid; else hi = mid - 1;
      }
      s_item = it;
      s_job = lo;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= total) break;
    const SweepJob& J = jobs[s_job];
    sweep_body<R, 1, NST, VJP, W, NT, SPLIT>(J.g, *reinterpret_cast<const WProg<R>*>(J.prog),
                                             *J.X, it - J.item0, 0, smraw);
    __syncthreads();
  }
}

// Transition-reduction passes of a space (built once, on the host; see
// tpass_tables_host).
static void build_tpass_tables(Space* sp) {
  if (sp->tbuilt) return;
  std::vector<TPass>& passes = sp->tpass_h;
  std::vector<TRecord>& recs = sp->trec_h;
  tpass_tables_host(sp->norb, sp->nocc, passes, recs, sp->rkey_h);
  std::vector<TPassDev> pd(passes.size());
  for (size_t i = 0; i < passes.size(); ++i) {
    for (int j = 0; j < 4; ++j) pd[i].q[j] = passes[i].q[j];
    pd[i].keep = passes[i].keep;
    pd[i].rec0 = passes[i].rec0;
    pd[i].rec1 = passes[i].rec1;
  }
  if (!pd.empty()) {
    FS_CUDA(cudaMalloc(&sp->tpass, pd.size() * sizeof(TPassDev)));
    FS_CUDA(cudaMemcpy(sp->tpass, pd.data(), pd.size() * sizeof(TPassDev),
                       cudaMemcpyHostToDevice));
    FS_CUDA(cudaMalloc(&sp->trec, std::max<size_t>(recs.size(), 1) * sizeof(TRecord)));
    if (!recs.empty())
      FS_CUDA(cudaMemcpy(sp->trec, recs.data(), recs.size() * sizeof(TRecord),
                         cudaMemcpyHostToDevice));
  }
  sp->npass = (int)pd.size();
  sp->tbuilt = true;
}

// Window tables of a space for width W (built once, on the host; see
// window_tables_host).
static void build_window_tables(Space* sp, int W) {
  Space::Win& wt = sp->win[W];
  if (wt.built) return;
  std::vector<uint32_t>& orbits = wt.orb_h;
  std::vector<int>& off = wt.off_h;
  std::vector<uint16_t> offs;
  window_tables_host(sp->norb, sp->nocc, W, orbits, off, offs, wt.okey_h);
  FS_CUDA(cudaMalloc(&wt.orbits, std::max<size_t>(orbits.size(), 1) * 4));
  FS_CUDA(cudaMalloc(&wt.off, off.size() * sizeof(int)));
  FS_CUDA(cudaMalloc(&wt.offs, offs.size() * 2));
  if (!orbits.empty())
    FS_CUDA(cudaMemcpy(wt.orbits, orbits.data(), orbits.size() * 4, cudaMemcpyHostToDevice));
  FS_CUDA(cudaMemcpy(wt.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  FS_CUDA(cudaMemcpy(wt.offs, offs.data(), offs.size() * 2, cudaMemcpyHostToDevice));
  wt.built = true;
}

// Orbit and record lists regrouped by cluster rank for clusters of 2^b CTAs
// with the blocked layout (built once per space and b).
static void build_window_groups(Space* sp, int W, int b) {
  Space::Win& wt = sp->win[W];
  if (wt.gorb[b]) return;
  std::vector<uint32_t> gorb;
  std::vector<int> goff;
  window_groups_host(wt.orb_h, wt.off_h, wt.okey_h, b, gorb, goff);
  FS_CUDA(cudaMalloc(&wt.gorb[b], std::max<size_t>(gorb.size(), 1) * 4));
  FS_CUDA(cudaMalloc(&wt.goff[b], std::max<size_t>(goff.size(), 1) * sizeof(int)));
  if (!gorb.empty())
    FS_CUDA(cudaMemcpy(wt.gorb[b], gorb.data(), gorb.size() * 4, cudaMemcpyHostToDevice));
  if (!goff.empty())
    FS_CUDA(cudaMemcpy(wt.goff[b], goff.data(), goff.size() * sizeof(int),
                       cudaMemcpyHostToDevice));
}

static void build_tpass_groups(Space* sp, int b) {
  if (sp->tgrec[b] || sp->tpass_h.empty()) return;
  std::vector<TRecord> grec;
  std::vector<int> goff;
  tpass_groups_host(sp->tpass_h, sp->trec_h, sp->rkey_h, b, grec, goff);
  FS_CUDA(cudaMalloc(&sp->tgrec[b], std::max<size_t>(grec.size(), 1) * sizeof(TRecord)));
  FS_CUDA(cudaMalloc(&sp->tgoff[b], std::max<size_t>(goff.size(), 1) * sizeof(int)));
  if (!grec.empty())
    FS_CUDA(cudaMemcpy(sp->tgrec[b], grec.data(), grec.size() * sizeof(TRecord),
                       cudaMemcpyHostToDevice));
  if (!goff.empty())
    FS_CUDA(cudaMemcpy(sp->tgoff[b], goff.data(), goff.size() * sizeof(int),
                       cudaMemcpyHostToDevice));
}

template <typename R>
static WProg<R> make_wprog(const RotProgram& rp, int N, int W) {
  WProg<R> w;
  std::vector<WinStep> steps = schedule_windows(rp, N, W);
  int ng = 0;
  for (size_t st = 0; st < steps.size(); ++st) {
    w.a[st] = (int8_t)steps[st].a;
    w.g0[st] = (int16_t)ng;
    for (int k : steps[st].givens) {
      w.u[ng] = (int8_t)(rp.g[k].p - steps[st].a);
      w.c[ng] = (R)rp.g[k].c;
      w.sr[ng] = (R)rp.g[k].s.real();
      w.si[ng] = (R)rp.g[k].s.imag();
      ++ng;
    }
  }
  w.nsteps = (int)steps.size();
  w.g0[w.nsteps] = (int16_t)ng;
  return w;
}

template <typename R>
static GProg<R> make_prog(const RotProgram& rp) {
  GProg<R> p;
  p.m = (int)rp.g.size();
  for (int k = 0; k < p.m; ++k) {
    p.p[k] = (int8_t)rp.g[k].p;
    p.c[k] = (R)rp.g[k].c;
    p.sr[k] = (R)rp.g[k].s.real();
    p.si[k] = (R)rp.g[k].s.imag();
  }
  return p;
}

template <typename R, int CS, int NST, bool VJP, int W, int NT, bool SPLIT, typename P,
          bool TC = false>
static void launch_sweep_t(const SweepGeom& g, const P& prog, const Mat& X,
                           int nslabs, size_t smem, cudaStream_t st) {
  auto kern = k_sweep<R, CS, NST, VJP, W, NT, SPLIT, TC>;
  FS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  static const char* names[2][2][2] = {  // [f64][reverse][beta]
      {{"sweep_alpha_f32", "sweep_beta_f32"}, {"sweep_vjp_alpha_f32", "sweep_vjp_beta_f32"}},
      {{"sweep_alpha_f64", "sweep_beta_f64"}, {"sweep_vjp_alpha_f64", "sweep_vjp_beta_f64"}}};
  ProfScope ps(names[sizeof(R) == 8][VJP][g.dir], st);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nslabs * CS));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CS > 1 ? 1 : 0;
  FS_CUDA(cudaLaunchKernelEx(&cfg, kern, g, prog, X));
}

template <typename R, int NST, bool VJP, int W, int NT, typename P, bool SPLIT = false>
static void dispatch_cs(int CS, const SweepGeom& g, const P& prog, const Mat& X,
                        int nslabs, size_t smem, cudaStream_t st) {
  switch (CS) {
    case 1: launch_sweep_t<R, 1, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    case 2: launch_sweep_t<R, 2, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    case 4: launch_sweep_t<R, 4, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    case 8: launch_sweep_t<R, 8, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    default: FS_REQUIRE(false, FS_ERR_UNSUPPORTED, "cluster size out of range");
  }
}

// Window width of the register-blocked sweep per precision and state count,
// chosen so one orbit of every vector fits in registers.
template <typename R, int NST>
constexpr int window_width() {
  return sizeof(R) == 4 ? (NST == 1 ? 6 : 5) : (NST == 1 ? 5 : 4);
}

static void set_window_geom(SweepGeom& g, Space* sp, int W) {
  build_window_tables(sp, W);
  const Space::Win& wt = sp->win[W];
  g.orbits = wt.orbits;
  g.orb_off = wt.off;
  if (g.blocked) {
    build_window_groups(sp, W, g.lgcs);
    g.orb_grp = wt.gorb[g.lgcs];
    g.orb_goff = wt.goff[g.lgcs];
  }
  g.offs = wt.offs;
  g.offs_stride = (sp->nocc + 1) << W;
}

// Kernel choice: window sweeps when the orbitals allow a window; forward
// sweeps on 256 threads when a slab is small enough for two CTAs per SM
// (their window-step barriers then overlap), else 512; reverse sweeps in
// split mode (one half-CTA per state) unless the vector spans a cluster (in a
// cluster the joint form measured faster: the split form gains little when
// every step ends on the cluster barrier).
// Gather indices of the tensor-core steps (see TcSeg), built once per space:
// b = 0 for the whole orbit list of each window position, b = 1 for the two
// rank groups of 2-CTA blocked clusters.  Row o of class m holds the
// addresses R_O + F[a][c_lo][S] of the orbit's strings, S in ascending
// local-mask order (the order of the compound matrices).
static void build_tc_index(Space* sp, int b) {
  Space::Win& wt = sp->win[tc::kW];
  if (wt.tc_seg[b]) return;
  const int W = tc::kW, N = sp->norb, n = sp->nocc;
  const int npos = N - W + 1;
  const int ranks = 1 << b;
  // in-window rank offsets F, as in window_tables_host
  std::vector<uint32_t> orbits;
  std::vector<int> off;
  std::vector<uint16_t> offs;
  std::vector<uint8_t> okey;
  window_tables_host(N, n, W, orbits, off, offs, okey);
  std::vector<uint32_t> gorb;
  std::vector<int> goff;
  if (b > 0) window_groups_host(orbits, off, okey, b, gorb, goff);
  static const int order[5] = {3, 2, 4, 1, 5};
  std::vector<uint16_t> idx;
  std::vector<TcSeg> seg((size_t)npos * ranks);
  int mx = 0;
  for (int a = 0; a < npos; ++a)
    for (int r = 0; r < ranks; ++r) {
      const uint32_t* list = b ? gorb.data() : orbits.data();
      const int lo = b ? goff[a * 9 + r] : off[a], hi = b ? goff[a * 9 + r + 1] : off[a + 1];
      TcSeg& sg = seg[(size_t)a * ranks + r];
      sg.start = (int)idx.size();
      for (int i = 0; i < 5; ++i) {
        const int m = order[i];
        const int ns = (int)cbinom(W, m), pad = (ns + 7) / 8 * 8;
        int cnt = 0;
        for (int k = lo; k < hi; ++k) {
          const uint32_t desc = list[k];
          if ((int)(desc >> 24) != m) continue;
          const int RO = desc & 0xFFFF, clo = (desc >> 16) & 0xFF;
          const uint16_t* Fc = offs.data() + (((size_t)a * (n + 1) + clo) << W);
          for (int j = 0; j < pad; ++j)
            idx.push_back(j < ns ? (uint16_t)(RO + Fc[win_mask(W, m, j)]) : (uint16_t)0);
          ++cnt;
        }
        sg.cnt[i] = cnt;
      }
      while (idx.size() % 8) idx.push_back(0);
      sg.len = (int)idx.size() - sg.start;
      sg.pad_ = 0;
      mx = std::max(mx, 2 * sg.len);
    }
  FS_CUDA(cudaMalloc(&wt.tc_idx[b], std::max<size_t>(idx.size(), 8) * sizeof(uint16_t)));
  if (!idx.empty())
    FS_CUDA(cudaMemcpy(wt.tc_idx[b], idx.data(), idx.size() * sizeof(uint16_t),
                       cudaMemcpyHostToDevice));
  FS_CUDA(cudaMalloc(&wt.tc_seg[b], seg.size() * sizeof(TcSeg)));
  FS_CUDA(cudaMemcpy(wt.tc_seg[b], seg.data(), seg.size() * sizeof(TcSeg),
                     cudaMemcpyHostToDevice));
  wt.tc_seg_max[b] = (mx + 15) / 16 * 16;
}

// Tensor-core sweep of one program (complex64, W = 6, 1 or 2 CTAs per
// vector): the step images are built on the device first, into context
// scratch that the sweep then reads (stream order keeps consecutive sweeps
// apart).
template <int NST, bool VJP>
static void dispatch_tc(Ctx* ctx, Space* sthis, int CS, const SweepGeom& g0, const RotProgram& rp,
                        const Mat& X, int nslabs, size_t smem, cudaStream_t st) {
  SweepGeom g = g0;
  set_window_geom(g, sthis, tc::kW);
  Space::Win& wt = sthis->win[tc::kW];
  build_tc_index(sthis, 0);
  g.tc_seg_full = wt.tc_seg[0];
  g.tc_idx_full = wt.tc_idx[0];
  if (CS > 1) {
    build_tc_index(sthis, 1);
    g.tc_seg_grp = wt.tc_seg[1];
    g.tc_idx_grp = wt.tc_idx[1];
  }
  const WProg<double> wpd = make_wprog<double>(rp, sthis->norb, tc::kW);
  const WProg<float> wpf = make_wprog<float>(rp, sthis->norb, tc::kW);
  unsigned char* img = (unsigned char*)scratch(
      ctx, "tc_steps", (size_t)std::max(1, wpd.nsteps) * tc::kStepBytes);
  if (wpd.nsteps > 0) {
    ProfScope ps("tc_step_images", st);
    k_tc_bmats<<<wpd.nsteps, 256, 0, st>>>(wpd, img);
    FS_CUDA(cudaGetLastError());
  }
  g.tc_b = img;
  if (CS == 1)
    launch_sweep_t<float, 1, NST, VJP, tc::kW, tc::kThreads, false, WProg<float>, true>(
        g, wpf, X, nslabs, smem, st);
  else
    launch_sweep_t<float, 2, NST, VJP, tc::kW, tc::kThreads, false, WProg<float>, true>(
        g, wpf, X, nslabs, smem, st);
}

template <typename R, int NST, bool VJP>
static void dispatch_prog(Space* sthis, int CS, const SweepGeom& g0, const RotProgram& rp,
                          const Mat& X, int nslabs, size_t smem, bool two_per_sm,
                          cudaStream_t st) {
  if constexpr (NST == 1) {
    constexpr int W = window_width<R, 1>();
    if (sthis->norb >= W && sthis->dim > 1) {
      SweepGeom g = g0;
      set_window_geom(g, sthis, W);
      auto prog = make_wprog<R>(rp, sthis->norb, W);
      if (two_per_sm)
        dispatch_cs<R, NST, VJP, W, 256>(CS, g, prog, X, nslabs, smem, st);
      else
        dispatch_cs<R, NST, VJP, W, 512>(CS, g, prog, X, nslabs, smem, st);
      return;
    }
  } else {
    constexpr int WS = window_width<R, 1>();
    constexpr int WJ = window_width<R, 2>();
    if (CS == 1 && sthis->norb >= WS && sthis->dim > 1) {
      SweepGeom g = g0;
      set_window_geom(g, sthis, WS);
      auto prog = make_wprog<R>(rp, sthis->norb, WS);
      launch_sweep_t<R, 1, NST, VJP, WS, 512, true>(g, prog, X, nslabs, smem, st);
      return;
    }
    if (sthis->norb >= WJ && sthis->dim > 1) {
      SweepGeom g = g0;
      set_window_geom(g, sthis, WJ);
      auto prog = make_wprog<R>(rp, sthis->norb, WJ);
      dispatch_cs<R, NST, VJP, WJ, 512>(CS, g, prog, X, nslabs, smem, st);
      return;
    }
  }
  auto prog = make_prog<R>(rp);
  dispatch_cs<R, NST, VJP, 0, 512>(CS, g0, prog, X, nslabs, smem, st);
}

// Split of each vector over the CS ranks of a cluster.  Preferred: rank r
// holds the strings whose occupation of the top b = log2(CS) orbitals reads
// r (a contiguous address range of C(N - b, n - popcount(r)) strings), so
// that the orbits of windows and subsets clear of those orbitals stay
// within one CTA; else (the largest such block does not fit) equal chunks.
template <typename Fits>
static void set_cluster_layout(SweepGeom& g, const Space* sp, int CS, Fits&& fits) {
  g.blocked = 0;
  g.lgcs = 0;
  g.cb[0] = 0;
  if (CS > 1) {
    int b = 0;
    while ((1 << b) < CS) ++b;
    int64_t mx = 0;
    std::vector<int64_t> bs(CS);
    for (int r = 0; r < CS; ++r) {
      const int k = sp->nocc - __builtin_popcount(r);
      bs[r] = (k < 0 || k > sp->norb - b) ? 0 : (int64_t)binom_host(sp->norb - b, k);
      mx = std::max(mx, bs[r]);
    }
    if (sp->norb >= 3 && b <= 3 && fits((int)mx)) {
      g.blocked = 1;
      g.lgcs = b;
      g.chunk = (int)mx;
      for (int r = 0; r < CS; ++r) g.cb[r + 1] = g.cb[r] + (int)bs[r];
      return;
    }
  }
  g.chunk = (g.d + CS - 1) / CS;
  for (int r = 1; r <= CS; ++r) g.cb[r] = std::min(g.d, r * g.chunk);
}

void launch_sweep(Ctx* ctx, const Space* sa, const Space* sb, int dir, void* st0,
                  void* st1, int nst, int dtype, const RotProgram& rp,
                  const PhaseDev& ph, cudaStream_t st, const RevArgs* rev) {
  FS_REQUIRE((nst == 2) == (rev != nullptr), FS_ERR_ARG, "reverse mode needs two states");
  const Space* sthis = dir == 0 ? sa : sb;
  const Space* sother = dir == 0 ? sb : sa;
  FS_REQUIRE(sthis->dim <= kMaxSweepDim, FS_ERR_UNSUPPORTED,
             "string dimension above 65535 is not supported by the sweep kernels");
  FS_REQUIRE((int)rp.g.size() <= kMaxGivens, FS_ERR_ARG, "too many Givens rotations");
  SweepGeom g{};
  g.st[0] = st0;
  g.st[1] = st1;
  g.d_b = sb->dim;
  g.dir = dir;
  g.d = (int)sthis->dim;
  g.nvec = (int)sother->dim;
  g.pairs = sthis->pairs;
  g.npp = sthis->npp;
  g.masks_this = sthis->masks;
  g.masks_other = sother->masks;
  g.norb = sthis->norb;
  g.nchunk = (sthis->norb + 7) / 8;
  g.ea_this = dir == 0 ? ph.ea_a : ph.ea_b;
  g.ea_other = dir == 0 ? ph.ea_b : ph.ea_a;
  g.has_x = ph.has_x;
  if (rev) {
    g.ea2_this = dir == 0 ? rev->ea2_a : rev->ea2_b;
    g.ea2_other = dir == 0 ? rev->ea2_b : rev->ea2_a;
    g.xpairs = sthis->xpairs;
    g.xsign = sthis->xsign;
    g.xcount = sthis->xcount;
    g.nx = sthis->nx;
    g.T = sthis->nx > 0 ? rev->T : nullptr;
    g.W = rev->W;
    if (g.T && sthis->norb >= 4 && sthis->nocc >= 1) {
      build_tpass_tables(const_cast<Space*>(sthis));
      g.tpass = sthis->tpass;
      g.trec = sthis->trec;
      g.npass = sthis->npass;
    }
  }
  g.status = ctx->d_status;
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  const size_t maxsm = (size_t)ctx->prop.sharedMemPerBlockOptin;
  const size_t tab_per_kv = ph.has_x ? g.nchunk * 256 * csz : 0;
  const size_t fixed = ph.has_x ? kMaxOrb * sizeof(double) : 0;
  const size_t tsum = (size_t)g.npass * 32 * (csz / 2);  // per-CTA pass sums
  auto smem_for = [&](int CS, int KV) {
    size_t chunk = (g.d + CS - 1) / CS;
    return (size_t)KV * (chunk * csz * nst + tab_per_kv + fixed) + tsum;
  };
  // tensor-core window steps: complex64, a window of 6 orbitals, the vector
  // on 1 CTA or a blocked pair (the step images take 2 x 35 KB)
  if (dtype == FS_C64 && ctx->sweep_engine == FS_SWEEP_TENSOR && sthis->norb >= tc::kW &&
      sthis->dim > 1 && ctx->prop.major >= 10) {
    Space* sw0 = const_cast<Space*>(sthis);
    build_tc_index(sw0, 0);
    for (int CS = 1; CS <= 2; CS *= 2) {
      if (CS > 1) build_tc_index(sw0, 1);
      const Space::Win& wt = sthis->win[tc::kW];
      const int cap = CS > 1 ? std::max(wt.tc_seg_max[0], wt.tc_seg_max[1]) : wt.tc_seg_max[0];
      auto smem_tc = [&](size_t chunk, int KV) {
        return (size_t)KV * chunk * csz * nst +
               std::max<size_t>(128 + 2 * (size_t)tc::kStepBytes + 2 * (size_t)cap,
                                (size_t)KV * (tab_per_kv + fixed) + tsum);
      };
      SweepGeom gt = g;
      gt.tc_idx_cap = cap;
      set_cluster_layout(gt, sthis, CS, [&](int chunk) { return smem_tc(chunk, 1) <= maxsm; });
      if (CS > 1 && !gt.blocked) continue;
      if (smem_tc(gt.chunk, 1) > maxsm) continue;
      int want = std::max(1, gt.nvec / (2 * ctx->prop.multiProcessorCount));
      int lg = 0;
      while ((2 << lg) <= std::min(want, kMaxKV) && smem_tc(gt.chunk, 2 << lg) <= maxsm) ++lg;
      gt.lgKV = lg;
      if (gt.blocked && gt.npass > 0) {
        build_tpass_groups(const_cast<Space*>(sthis), gt.lgcs);
        gt.trec_grp = sthis->tgrec[gt.lgcs];
        gt.tgoff = sthis->tgoff[gt.lgcs];
      }
      const int KV = 1 << lg;
      const int nslabs = (gt.nvec + KV - 1) / KV;
      // more than half an SM's shared memory: one CTA per SM, so that no two
      // CTAs (of different clusters) ever wait on one SM's tensor memory
      const size_t smem = std::max(smem_tc(gt.chunk, KV),
                                   (size_t)ctx->prop.sharedMemPerMultiprocessor / 2 + 1024);
      Space* sw = const_cast<Space*>(sthis);
      if (nst == 1)
        dispatch_tc<1, false>(ctx, sw, CS, gt, rp, ph.X, nslabs, smem, st);
      else
        dispatch_tc<2, true>(ctx, sw, CS, gt, rp, ph.X, nslabs, smem, st);
      return;
    }
  }
  int CS = 1;
  while (CS <= 8 && smem_for(CS, 1) > maxsm) CS *= 2;
  FS_REQUIRE(CS <= 8, FS_ERR_UNSUPPORTED, "state vector too large for a cluster of 8");
  // two CTAs per SM for single-state sweeps whose slab fits half the SM
  const size_t half_sm = (size_t)ctx->prop.sharedMemPerMultiprocessor / 2 - 1024;
  const bool two_per_sm = nst == 1 && CS == 1 && smem_for(1, 1) <= half_sm;
  const size_t budget = two_per_sm ? half_sm : maxsm;
  // vectors per slab: fit the budget, keep >= 2 slabs per SM when possible
  int want = std::max(1, g.nvec / (2 * ctx->prop.multiProcessorCount));
  int lg = 0;
  while ((2 << lg) <= std::min(want, kMaxKV) && smem_for(CS, 2 << lg) <= budget) ++lg;
  g.lgKV = lg;
  set_cluster_layout(g, sthis, CS, [&](int chunk) {
    return (size_t)(chunk * csz * nst + tab_per_kv + fixed) + tsum <= maxsm;
  });
  if (g.blocked && g.npass > 0) {
    build_tpass_groups(const_cast<Space*>(sthis), g.lgcs);
    g.trec_grp = sthis->tgrec[g.lgcs];
    g.tgoff = sthis->tgoff[g.lgcs];
  }
  const int KV = 1 << lg;
  const int nslabs = (g.nvec + KV - 1) / KV;
  const size_t smem = std::max<size_t>(
      (size_t)KV * ((size_t)g.chunk * csz * nst + tab_per_kv + fixed) + tsum, 16);
  Space* sw = const_cast<Space*>(sthis);
  if (dtype == FS_C64) {
    if (nst == 1) dispatch_prog<float, 1, false>(sw, CS, g, rp, ph.X, nslabs, smem, two_per_sm, st);
    else dispatch_prog<float, 2, true>(sw, CS, g, rp, ph.X, nslabs, smem, false, st);
  } else {
    if (nst == 1) dispatch_prog<double, 1, false>(sw, CS, g, rp, ph.X, nslabs, smem, two_per_sm, st);
    else dispatch_prog<double, 2, true>(sw, CS, g, rp, ph.X, nslabs, smem, false, st);
  }
}

// ------------------------------------------------------- batched sweeps
size_t wprog_bytes(int dtype) {
  return dtype == FS_C64 ? sizeof(WProg<float>) : sizeof(WProg<double>);
}

int batch_window(int dtype, int nst) {
  return dtype == FS_C64 ? (nst == 1 ? window_width<float, 1>() : window_width<float, 1>())
                         : (nst == 1 ? window_width<double, 1>() : window_width<double, 1>());
}

// One circuit's sweep as a job of a batched launch: one CTA per slab (no
// cluster), window program for the batch window width, slab sized to
// `budget` bytes of shared memory.
// Autotuner of the batched sweeps' slab width: one circuit's sweep as a
// one-job launch of the batched kernel, on scratch states (and scratch W
// and T for the reverse sweeps), for every slab width 2^0 .. 2^lgmax that
// fits the stage's budget; CUDA events on a private stream, the fastest
// mean of two launches after one warm-up wins and is cached per sector and
// sweep kind.  Runs before any capture.
template <typename SmemFor>
static int tune_batch_slab(Ctx* ctx, const SweepGeom& g0, const std::vector<unsigned char>& prog,
                           int nst, int dtype, bool rev, int lgmax, SmemFor&& smem_for,
                           const std::array<int, 8>& key) {
  if (!ctx->tune_stream)
    FS_CUDA(cudaStreamCreateWithFlags(&ctx->tune_stream, cudaStreamNonBlocking));
  cudaStream_t ts = ctx->tune_stream;
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  const size_t nstate = (size_t)g0.d * g0.nvec;
  char* st = (char*)scratch(ctx, "tune_states", nstate * csz * nst);
  FS_CUDA(cudaMemsetAsync(st, 0, nstate * csz * nst, ts));
  // device copies of the program, a zero cross matrix and the job
  char* dev = (char*)scratch(ctx, "tune_job", prog.size() + sizeof(Mat) + sizeof(SweepJob) + 1024);
  char* dprog = dev;
  Mat* dX = (Mat*)(dev + (prog.size() + 255) / 256 * 256);
  SweepJob* djob = (SweepJob*)((char*)dX + (sizeof(Mat) + 255) / 256 * 256);
  int* dcounter = (int*)scratch(ctx, "tune_counter", sizeof(int));
  FS_CUDA(cudaMemcpyAsync(dprog, prog.data(), prog.size(), cudaMemcpyHostToDevice, ts));
  FS_CUDA(cudaMemsetAsync(dX, 0, sizeof(Mat), ts));
  SweepGeom g = g0;
  g.st[0] = st;
  g.st[1] = nst == 2 ? st + nstate * csz : nullptr;
  if (rev) {
    g.T = (double*)scratch(ctx, "tune_T", (size_t)2 * kMaxOrb * kMaxOrb * sizeof(double));
    g.W = g0.W ? scratch(ctx, "tune_W", nstate * (csz / 2)) : nullptr;
  }
  cudaEvent_t e0, e1;
  FS_CUDA(cudaEventCreate(&e0));
  FS_CUDA(cudaEventCreate(&e1));
  std::vector<float> ms(lgmax + 1, 0.f);
  int best = 0;
  for (int lg = 0; lg <= lgmax; ++lg) {
    g.lgKV = lg;
    SweepJob j{};
    j.g = g;
    j.prog = dprog;
    j.X = dX;
    j.item0 = 0;
    const int nslabs = (g.nvec + (1 << lg) - 1) >> lg;
    const size_t smem = smem_for(1 << lg);
    FS_CUDA(cudaMemcpyAsync(djob, &j, sizeof(j), cudaMemcpyHostToDevice, ts));
    launch_sweep_batch(ctx, dtype, nst, nullptr, 0, 0, nullptr, smem, ts);  // attribute
    float tot = 0;
    for (int r = 0; r < 3; ++r) {
      FS_CUDA(cudaMemsetAsync(dcounter, 0, sizeof(int), ts));
      if (r == 1) FS_CUDA(cudaEventRecord(e0, ts));
      launch_sweep_batch(ctx, dtype, nst, djob, 1, nslabs, dcounter, smem, ts);
    }
    FS_CUDA(cudaEventRecord(e1, ts));
    FS_CUDA(cudaEventSynchronize(e1));
    FS_CUDA(cudaEventElapsedTime(&tot, e0, e1));
    ms[lg] = tot / 2;
    if (ms[lg] < ms[best]) best = lg;
  }
  FS_CUDA(cudaEventDestroy(e0));
  FS_CUDA(cudaEventDestroy(e1));
  ctx->sweep_tune[key] = best;
  ctx->sweep_tune_ms[key] = ms;
  return best;
}

void plan_batch_sweep(Ctx* ctx, Space* sa, Space* sb, int dir, void* st0, void* st1, int nst,
                      int dtype, const RotProgram& rp, const PhaseDev& ph, const RevArgs* rev,
                      size_t budget, BatchSweepPlan& out) {
  Space* sthis = dir == 0 ? sa : sb;
  Space* sother = dir == 0 ? sb : sa;
  const int W = batch_window(dtype, nst);
  FS_REQUIRE(sthis->norb >= W && sthis->dim > 1 && sthis->dim <= kMaxSweepDim,
             FS_ERR_UNSUPPORTED, "batched sweeps need norb >= 6 and 2 <= dim <= 65535");
  SweepGeom& g = out.g;
  g = SweepGeom{};
  g.st[0] = st0;
  g.st[1] = st1;
  g.d_b = sb->dim;
  g.dir = dir;
  g.d = (int)sthis->dim;
  g.nvec = (int)sother->dim;
  g.pairs = sthis->pairs;
  g.npp = sthis->npp;
  g.masks_this = sthis->masks;
  g.masks_other = sother->masks;
  g.norb = sthis->norb;
  g.nchunk = (sthis->norb + 7) / 8;
  g.ea_this = dir == 0 ? ph.ea_a : ph.ea_b;
  g.ea_other = dir == 0 ? ph.ea_b : ph.ea_a;
  g.has_x = ph.has_x;
  if (rev) {
    g.ea2_this = dir == 0 ? rev->ea2_a : rev->ea2_b;
    g.ea2_other = dir == 0 ? rev->ea2_b : rev->ea2_a;
    g.T = rev->T;
    g.W = rev->W;
    build_tpass_tables(sthis);
    g.tpass = sthis->tpass;
    g.trec = sthis->trec;
    g.npass = sthis->npass;
  }
  set_window_geom(g, sthis, W);
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  const size_t tab_per_kv = ph.has_x ? g.nchunk * 256 * csz : 0;
  const size_t fixed = ph.has_x ? kMaxOrb * sizeof(double) : 0;
  const size_t tsum = (size_t)g.npass * 32 * (csz / 2);
  auto smem_for = [&](int KV) {
    return (size_t)KV * ((size_t)g.d * csz * nst + tab_per_kv + fixed) + tsum;
  };
  FS_REQUIRE(smem_for(1) <= budget, FS_ERR_UNSUPPORTED, "batched sweep slab does not fit");
  g.chunk = g.d;
  g.cb[0] = 0;
  g.cb[1] = g.d;
  out.prog.resize(wprog_bytes(dtype));
  if (dtype == FS_C64) {
    auto w = make_wprog<float>(rp, sthis->norb, W);
    memcpy(out.prog.data(), &w, sizeof(w));
  } else {
    auto w = make_wprog<double>(rp, sthis->norb, W);
    memcpy(out.prog.data(), &w, sizeof(w));
  }
  // slab width: the widest that fits the budget (at most 64 vectors), or the
  // autotuned width for this sector and sweep kind
  int lgmax = 0;
  while ((2 << lgmax) <= std::min(g.nvec, kMaxKV) && smem_for(2 << lgmax) <= budget) ++lgmax;
  const std::array<int, 8> key = {sthis->norb, sthis->nocc, sother->nocc, dtype, nst,
                                  rev != nullptr, ph.has_x, (int)(budget >> 10)};
  int lg = -1;
  auto it = ctx->sweep_tune.find(key);
  if (it != ctx->sweep_tune.end()) {
    lg = std::min(it->second, lgmax);
  } else if (ctx->batch_tuning && lgmax > 0) {
    lg = tune_batch_slab(ctx, g, out.prog, nst, dtype, rev != nullptr, lgmax, smem_for, key);
  }
  if (lg < 0) {  // untuned: about eight slabs per circuit
    const int want = std::max(1, g.nvec / 8);
    lg = 0;
    while ((2 << lg) <= std::min(want, kMaxKV) && lg < lgmax) ++lg;
  }
  g.lgKV = lg;
  out.nslabs = (g.nvec + (1 << lg) - 1) >> lg;
  out.smem = smem_for(1 << lg);
}

template <typename R, int NST, bool VJP, int W, int NT, bool SPLIT>
static void launch_batch_t(const SweepJob* jobs, int njobs, int total, int* counter, size_t smem,
                           int grid, cudaStream_t st) {
  auto kern = k_sweep_batch<R, NST, VJP, W, NT, SPLIT>;
  if (!jobs) {  // attribute only (called before a stream capture); only ever
                // raised, since several stages share one kernel
    cudaFuncAttributes fa;
    FS_CUDA(cudaFuncGetAttributes(&fa, kern));
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
      FS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return;
  }
  kern<<<grid, NT, smem, st>>>(jobs, njobs, total, counter);
  FS_CUDA(cudaGetLastError());
}

void launch_sweep_batch(Ctx* ctx, int dtype, int nst, const SweepJob* jobs, int njobs, int total,
                        int* counter, size_t smem, cudaStream_t st) {
  const int sms = ctx->prop.multiProcessorCount;
  const size_t half_sm = (size_t)ctx->prop.sharedMemPerMultiprocessor / 2 - 1024;
  if (dtype == FS_C64) {
    constexpr int W = window_width<float, 1>();
    if (nst == 1) {
      if (smem <= half_sm)
        launch_batch_t<float, 1, false, W, 256, false>(jobs, njobs, total, counter, smem, 2 * sms, st);
      else
        launch_batch_t<float, 1, false, W, 512, false>(jobs, njobs, total, counter, smem, sms, st);
    } else {
      launch_batch_t<float, 2, true, W, 512, true>(jobs, njobs, total, counter, smem, sms, st);
    }
  } else {
    constexpr int W = window_width<double, 1>();
    if (nst == 1) {
      if (smem <= half_sm)
        launch_batch_t<double, 1, false, W, 256, false>(jobs, njobs, total, counter, smem, 2 * sms, st);
      else
        launch_batch_t<double, 1, false, W, 512, false>(jobs, njobs, total, counter, smem, sms, st);
    } else {
      launch_batch_t<double, 2, true, W, 512, true>(jobs, njobs, total, counter, smem, sms, st);
    }
  }
}

// ------------------------------------------------------------------ phase
// One streaming pass: psi[i][j] *= ea_a[i] ea_b[j] exp(i sum X[p][q]) with
// the cross tables built per row from the alpha string.
template <typename R>
__global__ void __launch_bounds__(256)
    k_phase(cx_t<R>* vec, int64_t da, int64_t db, const uint32_t* ma,
            const uint32_t* mb, int norb, int nchunk, const void* ea_a,
            const void* ea_b, int has_x, const __grid_constant__ Mat X) {
  using C = cx_t<R>;
  __shared__ double w[kMaxOrb];
  __shared__ C tab[4 * 256];
  SweepGeom g{};
  g.dir = 1;
  g.norb = norb;
  g.nchunk = nchunk;
  g.has_x = has_x;
  g.masks_other = ma;
  for (int64_t i = blockIdx.x; i < da; i += gridDim.x) {
    C fa = ld_ea<R>(ea_a, i);
    if (has_x) {
      __syncthreads();
      build_cross_tables<R>(g, X, (int)i, 1, w, tab, threadIdx.x, blockDim.x);
    }
    C* row = vec + i * db;
    for (int64_t j = threadIdx.x; j < db; j += blockDim.x) {
      C f = cmul<R>(fa, ld_ea<R>(ea_b, j));
      if (has_x) {
        uint32_t m = __ldg(mb + j);
        for (int c = 0; c < nchunk; ++c) f = cmul<R>(f, tab[c * 256 + ((m >> (8 * c)) & 255)]);
      }
      row[j] = cmul<R>(f, row[j]);
    }
  }
}

void launch_phase(const Space* sa, const Space* sb, void* vec, int dtype,
                  const PhaseDev& ph, cudaStream_t st) {
  ProfScope ps(dtype == FS_C64 ? "phase_f32" : "phase_f64", st);
  int nchunk = (sa->norb + 7) / 8;
  unsigned grid = (unsigned)std::min<int64_t>(sa->dim, 4096);
  if (dtype == FS_C64)
    k_phase<float><<<grid, 256, 0, st>>>((float2*)vec, sa->dim, sb->dim, sa->masks,
                                         sb->masks, sa->norb, nchunk, ph.ea_a,
                                         ph.ea_b, ph.has_x, ph.X);
  else
    k_phase<double><<<grid, 256, 0, st>>>((double2*)vec, sa->dim, sb->dim, sa->masks,
                                          sb->masks, sa->norb, nchunk, ph.ea_a,
                                          ph.ea_b, ph.has_x, ph.X);
  FS_CUDA(cudaGetLastError());
}

// Per-string factors (FP64 arithmetic, stored in the state precision).
template <typename R>
__global__ void k_string_phase(cx_t<R>* out, const uint32_t* masks, int64_t dim,
                               int norb, const __grid_constant__ StrPhase f) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= dim) return;
  uint32_t m = masks[e];
  double re = 1, im = 0, ang = 0;
  for (int p = 0; p < norb; ++p) {
    if (!((m >> p) & 1u)) continue;
    if (f.use_d) {
      double dr = f.d[2 * p], di = f.d[2 * p + 1];
      double nr = re * dr - im * di;
      im = re * di + im * dr;
      re = nr;
    }
    if (f.use_lam) ang -= f.t * f.lam[p];
    if (f.use_j)
      for (int q = 0; q < norb; ++q)
        if ((m >> q) & 1u) ang -= 0.5 * f.t * f.J.v[p * norb + q];
  }
  double r = ang - 6.283185307179586 * rint(ang * 0.15915494309189535);
  double s, c;
  sincos(r, &s, &c);
  out[e] = mk<R>((R)(re * c - im * s), (R)(re * s + im * c));
}

void preload_phase_kernels() {
  cudaFuncAttributes fa;
  FS_CUDA(cudaFuncGetAttributes(&fa, k_string_phase<float>));
  FS_CUDA(cudaFuncGetAttributes(&fa, k_string_phase<double>));
  FS_CUDA(cudaFuncGetAttributes(&fa, k_phase<float>));
  FS_CUDA(cudaFuncGetAttributes(&fa, k_phase<double>));
}

void launch_string_phase(const Space* sp, void* out, int dtype, const StrPhase& f,
                         cudaStream_t st) {
  ProfScope ps("string_phase", st);
  unsigned grid = (unsigned)((sp->dim + 127) / 128);
  if (dtype == FS_C64)
    k_string_phase<float><<<grid, 128, 0, st>>>((float2*)out, sp->masks, sp->dim,
                                                 sp->norb, f);
  else
    k_string_phase<double><<<grid, 128, 0, st>>>((double2*)out, sp->masks, sp->dim,
                                                  sp->norb, f);
  FS_CUDA(cudaGetLastError());
}

// ----------------------------------------------- Hartree-Fock closed form
// v[e] = det(R[I_e, 0..n-1]) by Gaussian elimination with partial pivoting,
// FP64.
__global__ void k_slater_minors(const uint32_t* masks, int64_t dim, int norb, int n,
                                const __grid_constant__ CMat R, double2* v) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= dim) return;
  v[e] = slater_minor(masks[e], norb, n, R.v);
}

template <typename R>
__global__ void k_outer(cx_t<R>* vec, const double2* va, const double2* vb, int64_t da,
                        int64_t db) {
  int64_t n = da * db;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = k / db, j = k - i * db;
    double2 a = va[i], b = vb[j];
    vec[k] = mk<R>((R)(a.x * b.x - a.y * b.y), (R)(a.x * b.y + a.y * b.x));
  }
}

void launch_slater(Ctx* ctx, const Space* sa, const Space* sb, void* vec, int dtype,
                   const CMat& R, cudaStream_t st) {
  ProfScope ps("slater", st, 3);
  double2* va = (double2*)scratch(ctx, "slater_a", sa->dim * 16);
  double2* vb = (double2*)scratch(ctx, "slater_b", sb->dim * 16);
  k_slater_minors<<<(unsigned)((sa->dim + 63) / 64), 64, 0, st>>>(
      sa->masks, sa->dim, sa->norb, sa->nocc, R, va);
  FS_CUDA(cudaGetLastError());
  k_slater_minors<<<(unsigned)((sb->dim + 63) / 64), 64, 0, st>>>(
      sb->masks, sb->dim, sb->norb, sb->nocc, R, vb);
  FS_CUDA(cudaGetLastError());
  int64_t n = sa->dim * sb->dim;
  unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
  if (dtype == FS_C64)
    k_outer<float><<<grid, 256, 0, st>>>((float2*)vec, va, vb, sa->dim, sb->dim);
  else
    k_outer<double><<<grid, 256, 0, st>>>((double2*)vec, va, vb, sa->dim, sb->dim);
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
