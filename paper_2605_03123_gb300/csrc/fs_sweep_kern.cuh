// Device side of the Givens-rotation sweeps (kernels and their launch
// templates), shared by the translation units that instantiate them: the
// complex64 forward, reverse and batched kernels compile in units of their
// own, in parallel (see fs_sweep.cu for the sweep design).
#pragma once
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <tuple>
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

// One Givens update of the pair (x, y) in the form its coefficients are
// kept in: complex128 directly, complex64 as three in-place shears
// (x += tau y; y += sig x; x += tau y), each a complex multiply-add of two
// fused multiply-adds per part.
__device__ __forceinline__ void givens_upd(cx_t<double>& x, cx_t<double>& y, GCoef<double> k) {
  givens2<double>(x, y, k.c, k.sr, k.si);
}
__device__ __forceinline__ void givens_upd(cx_t<float>& x, cx_t<float>& y, GCoef<float> k) {
  x.x = fmaf(-k.ti, y.y, fmaf(k.tr, y.x, x.x));
  x.y = fmaf(k.ti, y.x, fmaf(k.tr, y.y, x.y));
  y.x = fmaf(-k.gi, x.y, fmaf(k.gr, x.x, y.x));
  y.y = fmaf(k.gi, x.x, fmaf(k.gr, x.y, y.y));
  x.x = fmaf(-k.ti, y.y, fmaf(k.tr, y.x, x.x));
  x.y = fmaf(k.ti, y.x, fmaf(k.tr, y.y, x.y));
}

template <int W, int M, int U, int J, typename R, int NV, int NS>
__device__ __forceinline__ void win_pair(cx_t<R> (&v)[NV][NS], GCoef<R> k) {
  constexpr int sm = win_src_mask(W, M, U, J);
  constexpr int a = win_index(W, M, sm);
  constexpr int b = win_index(W, M, sm ^ (1 << U) ^ (1 << (U + 1)));
#pragma unroll
  for (int x = 0; x < NV; ++x) givens_upd(v[x][a], v[x][b], k);
}
template <int W, int M, int U, typename R, int NV, int NS, int... J>
__device__ __forceinline__ void win_pairs_seq(cx_t<R> (&v)[NV][NS], GCoef<R> k,
                                              std::integer_sequence<int, J...>) {
  (win_pair<W, M, U, J, R, NV, NS>(v, k), ...);
}
template <int W, int M, int U, typename R, int NV, int NS>
__device__ __forceinline__ void win_pairs(cx_t<R> (&v)[NV][NS], GCoef<R> k) {
  if constexpr (U + 1 < W)
    win_pairs_seq<W, M, U, R, NV, NS>(v, k, std::make_integer_sequence<int, win_npairs(W, M, U)>{});
}

// Window patterns.  The greedy window schedule of the adjacent
// decomposition (rows N-1 .. 1, columns 0 .. r-1) repeats a few u-sequences
// for every N: each is applied with compile-time pair indices, so a step
// costs one dispatch per orbit instead of one per rotation.  Steps with
// other sequences take the general loop.
template <int... U>
using useq = std::integer_sequence<int, U...>;
template <int W>
struct WinPatterns {
  using list = std::tuple<>;
};
template <>
struct WinPatterns<6> {
  using list = std::tuple<useq<2, 3, 4, 1, 2, 3, 0, 1, 2>, useq<2, 3, 4, 1, 2, 3, 0, 1, 2, 0, 1, 0>,
                          useq<3, 4, 2, 3, 1, 2, 0, 1>, useq<4, 3, 2, 1, 0>,
                          useq<0, 1, 2, 3, 4, 0, 1, 2, 3, 0, 1, 2, 0, 1, 0>>;
};
template <>
struct WinPatterns<5> {
  using list = std::tuple<useq<2, 3, 1, 2, 0, 1>, useq<3, 2, 1, 0>, useq<1, 2, 3, 0, 1, 2, 0, 1, 0>,
                          useq<0, 1, 2, 3, 0, 1, 2, 0, 1, 0>, useq<2, 1, 0>>;
};
template <>
struct WinPatterns<4> {
  using list = std::tuple<useq<1, 2, 0, 1>, useq<1, 2, 0, 1, 0>, useq<2, 1, 0>, useq<0, 1, 2, 0, 1, 0>>;
};
template <int W>
constexpr int win_npat() {
  return (int)std::tuple_size<typename WinPatterns<W>::list>::value;
}

template <int W, int M, typename R, int NV, int NS, int... U, int... K>
__device__ __forceinline__ void win_seq(cx_t<R> (&v)[NV][NS], const WProg<R>& prog, int ga,
                                        useq<U...>, std::integer_sequence<int, K...>) {
  (win_pairs<W, M, U, R, NV, NS>(v, prog.coef(ga + K)), ...);
}
template <int W, int M, typename R, int NV, int NS, int I>
__device__ __forceinline__ bool win_pattern(int pid, cx_t<R> (&v)[NV][NS], const WProg<R>& prog,
                                            int ga) {
  using S = typename std::tuple_element<I, typename WinPatterns<W>::list>::type;
  if (pid != I) return false;
  win_seq<W, M, R, NV, NS>(v, prog, ga, S{}, std::make_integer_sequence<int, (int)S::size()>{});
  return true;
}
// Applies pattern pid (true), or does nothing (false: no such pattern).
template <int W, int M, typename R, int NV, int NS, size_t... I>
__device__ __forceinline__ bool win_patterns(int pid, cx_t<R> (&v)[NV][NS], const WProg<R>& prog,
                                             int ga, std::index_sequence<I...>) {
  return (win_pattern<W, M, R, NV, NS, (int)I>(pid, v, prog, ga) || ...);
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


// The rotations ga .. gb-1 of a window step on NV register copies of an
// orbit: through the step's compile-time pattern when it has one (PAT: the
// complex64 single-CTA kernels on one copy; with two copies the unrolled
// code outgrows the instruction cache and measured slower, and the other
// kernels keep one loop to bound the build time), else one dispatch per
// rotation.
template <int W, int M, typename R, int NV, int NS, bool PAT>
__device__ __forceinline__ void win_apply(cx_t<R> (&v)[NV][NS], const WProg<R>& prog, int ga,
                                          int gb, int pid) {
  constexpr int npat = PAT ? win_npat<W>() : 0;
  if (win_patterns<W, M, R, NV, NS>(pid, v, prog, ga, std::make_index_sequence<(size_t)npat>{}))
    return;
  for (int q = ga; q < gb; ++q) {
    const GCoef<R> k = prog.coef(q);
    switch (prog.u[q]) {
      case 0: win_pairs<W, M, 0, R, NV, NS>(v, k); break;
      case 1: win_pairs<W, M, 1, R, NV, NS>(v, k); break;
      case 2: win_pairs<W, M, 2, R, NV, NS>(v, k); break;
      case 3: win_pairs<W, M, 3, R, NV, NS>(v, k); break;
      case 4: win_pairs<W, M, 4, R, NV, NS>(v, k); break;
      case 5: win_pairs<W, M, 5, R, NV, NS>(v, k); break;
      case 6: win_pairs<W, M, 6, R, NV, NS>(v, k); break;
      default: break;
    }
  }
}

// One orbit of a window step: the C(W, M) strings sharing the occupation
// outside the window.  Their addresses are R_O + F[c_lo][S]; every vector of
// the slab is rotated in registers by the step's Givens rotations.
template <typename R, int CS, int NST, int W, int M>
__device__ __forceinline__ void win_orbit(uint32_t desc, const uint16_t* F, cx_t<R>* const* base,
                                          size_t st_stride, const int (&cbr)[CS + 1], int KV,
                                          int kv_eff, const WProg<R>& prog, int ga, int gb,
                                          int pid) {
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
    win_apply<W, M, R, NST, NS, sizeof(R) == 4 && CS == 1 && NST == 1>(v, prog, ga, gb, pid);
#pragma unroll
    for (int x = 0; x < NST; ++x)
#pragma unroll
      for (int k = 0; k < NS; ++k)
        base[CS > 1 ? own[k] : 0][x * st_stride + ad[k] + kv] = v[x][k];
  }
}

// ------------------------------------------- packed two-lane window steps
// Complex64 kernels that rotate two amplitude sets under the same rotations
// (two vectors of a slab in the forward sweeps; psi and g of one vector in
// the reverse sweeps) keep them packed per string in a 16-byte cell
// (Re lane 0, Re lane 1, Im lane 0, Im lane 1), so that one shared-memory
// access moves both and each Givens update runs as packed two-lane FP32
// (fma.rn.f32x2) with no register shuffles.  Lane 0 of cell c is at float
// 4c, lane 1 at 4c + 1, imaginary parts 2 further.
//
// Packed Givens update of the pairs (x, y) of both lanes, the same
// operations as the one-lane shear update lane by lane (so the results are
// bit-identical): x += tau y; y += sig x; x += tau y, every amplitude
// updated in place.
__device__ __forceinline__ void givens2_pk(float2& xr, float2& xi, float2& yr, float2& yi,
                                           float2 tr, float2 ti, float2 nti, float2 gr,
                                           float2 gi, float2 ngi) {
  xr = __ffma2_rn(nti, yi, __ffma2_rn(tr, yr, xr));
  xi = __ffma2_rn(ti, yr, __ffma2_rn(tr, yi, xi));
  yr = __ffma2_rn(ngi, xi, __ffma2_rn(gr, xr, yr));
  yi = __ffma2_rn(gi, xr, __ffma2_rn(gr, xi, yi));
  xr = __ffma2_rn(nti, yi, __ffma2_rn(tr, yr, xr));
  xi = __ffma2_rn(ti, yr, __ffma2_rn(tr, yi, xi));
}
template <int W, int M, int U, int J, int NS>
__device__ __forceinline__ void win_pair_pk(float2 (&vr)[NS], float2 (&vi)[NS], float2 tr,
                                            float2 ti, float2 nti, float2 gr, float2 gi,
                                            float2 ngi) {
  constexpr int sm = win_src_mask(W, M, U, J);
  constexpr int a = win_index(W, M, sm);
  constexpr int b = win_index(W, M, sm ^ (1 << U) ^ (1 << (U + 1)));
  givens2_pk(vr[a], vi[a], vr[b], vi[b], tr, ti, nti, gr, gi, ngi);
}
template <int W, int M, int U, int NS, int... J>
__device__ __forceinline__ void win_pairs_pk_seq(float2 (&vr)[NS], float2 (&vi)[NS],
                                                 const WProg<float>& prog, int q,
                                                 std::integer_sequence<int, J...>) {
  const float2 tr = prog.tr2[q], ti = prog.ti2[q], nti = prog.nti2[q], gr = prog.gr2[q],
               gi = prog.gi2[q];
  const float2 ngi = __fmul2_rn(gi, make_float2(-1.f, -1.f));
  (win_pair_pk<W, M, U, J, NS>(vr, vi, tr, ti, nti, gr, gi, ngi), ...);
}
template <int W, int M, int U, int NS>
__device__ __forceinline__ void win_pairs_pk(float2 (&vr)[NS], float2 (&vi)[NS],
                                             const WProg<float>& prog, int q) {
  if constexpr (U + 1 < W)
    win_pairs_pk_seq<W, M, U, NS>(vr, vi, prog, q,
                                  std::make_integer_sequence<int, win_npairs(W, M, U)>{});
}
// One orbit of a window step in a packed slab, packed set kc (cell stride
// per string KC).
template <int W, int M>
__device__ __forceinline__ void win_orbit_pk(uint32_t desc, const uint16_t* F, float* smf, int KC,
                                             int kc, const WProg<float>& prog, int ga, int gb) {
  constexpr int NS = cbinom(W, M);
  const int RO = desc & 0xFFFF, clo = (desc >> 16) & 0xFF;
  const uint16_t* Fc = F + (clo << W);
  int ad[NS];
  win_offsets<W, M>(Fc, ad, std::make_integer_sequence<int, NS>{});
#pragma unroll
  for (int k = 0; k < NS; ++k) ad[k] = (RO + ad[k]) * KC;
  {
    float2 vr[NS], vi[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float4 t = reinterpret_cast<const float4*>(smf)[ad[k] + kc];
      vr[k] = make_float2(t.x, t.y);
      vi[k] = make_float2(t.z, t.w);
    }
    for (int q = ga; q < gb; ++q) {
      switch (prog.u[q]) {
        case 0: win_pairs_pk<W, M, 0, NS>(vr, vi, prog, q); break;
        case 1: win_pairs_pk<W, M, 1, NS>(vr, vi, prog, q); break;
        case 2: win_pairs_pk<W, M, 2, NS>(vr, vi, prog, q); break;
        case 3: win_pairs_pk<W, M, 3, NS>(vr, vi, prog, q); break;
        case 4: win_pairs_pk<W, M, 4, NS>(vr, vi, prog, q); break;
        case 5: win_pairs_pk<W, M, 5, NS>(vr, vi, prog, q); break;
        default: break;
      }
    }
#pragma unroll
    for (int k = 0; k < NS; ++k)
      reinterpret_cast<float4*>(smf)[ad[k] + kc] = make_float4(vr[k].x, vr[k].y, vi[k].x, vi[k].y);
  }
}
// Float index of Re of amplitude (state s, string el, vector kv) in a
// packed slab: one state, vector pairs (NST = 1), or psi and g (NST = 2).
template <int NST>
__device__ __forceinline__ size_t pk_re(int s, size_t el, int KV, int kv) {
  if constexpr (NST == 1)
    return 4 * (el * (size_t)(KV >> 1) + (size_t)(kv >> 1)) + (size_t)(kv & 1);
  else
    return 4 * (el * (size_t)KV + (size_t)kv) + (size_t)s;
}
// Quotient and remainder of idx by n along idx = i0, i0 + step, ...: one
// division when the walk starts, then an add and a compare per step.
struct DivWalk {
  int n, q, r, a, b;  // a = idx / n, b = idx % n
  __device__ __forceinline__ DivWalk(int i0, int step, int n_) : n(n_) {
    a = i0 / n;
    b = i0 - a * n;
    q = step / n;
    r = step - q * n;
  }
  __device__ __forceinline__ void next() {
    a += q;
    b += r;
    if (b >= n) {
      b -= n;
      ++a;
    }
  }
};
__device__ __forceinline__ void cp_async_4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
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
// DIAG: the diagonal slots are evaluated; KEEP: ownership is tested per slot
// (else every evaluated slot is owned).
template <typename R, int M, int J, int NS, bool DIAG, bool KEEP>
__device__ __forceinline__ void t_term(const cx_t<R> (&ps)[NS], const cx_t<R> (&pg)[NS],
                                       R (&acc)[32], uint32_t keep) {
  constexpr int k = J / 16, a = (J / 4) % 4, b = J % 4;
  if constexpr (k < NS) {
    constexpr int S = win_mask(4, M, k);
    constexpr int slot = a * 4 + b;
    if constexpr ((S >> b) & 1) {
      if constexpr (a == b) {
        if (DIAG && (!KEEP || (keep & (1u << slot)))) {  // uniform per pass: diagonals are owned once
          acc[2 * slot] = fma(pg[k].x, ps[k].x, fma(pg[k].y, ps[k].y, acc[2 * slot]));
          acc[2 * slot + 1] = fma(pg[k].x, ps[k].y, fma(-pg[k].y, ps[k].x, acc[2 * slot + 1]));
        }
      } else if constexpr (!((S >> a) & 1)) {
        constexpr int k2 = win_index(4, M, S ^ (1 << a) ^ (1 << b));
        constexpr int lo = a < b ? a : b, hi = a < b ? b : a;
        constexpr bool neg = cpopc(S & ((1 << hi) - 1) & ~((2 << lo) - 1)) & 1;
        constexpr R sg = neg ? R(-1) : R(1);
        if (!KEEP || (keep & (1u << slot))) {  // uniform per pass: each pair is owned once
          // acc += sg * conj(g[k2]) * psi[k], as four fused multiply-adds
          const R gx = sg * pg[k2].x, gy = sg * pg[k2].y;
          acc[2 * slot] = fma(gx, ps[k].x, fma(gy, ps[k].y, acc[2 * slot]));
          acc[2 * slot + 1] = fma(gx, ps[k].y, fma(-gy, ps[k].x, acc[2 * slot + 1]));
        }
      }
    }
  }
}
template <typename R, int M, int NS, bool DIAG, bool KEEP, int... J>
__device__ __forceinline__ void t_terms(const cx_t<R> (&ps)[NS], const cx_t<R> (&pg)[NS],
                                        R (&acc)[32], uint32_t keep,
                                        std::integer_sequence<int, J...>) {
  (t_term<R, M, J, NS, DIAG, KEEP>(ps, pg, acc, keep), ...);
}
template <typename R, int CS, int M, bool PK, bool DIAG = true, bool KEEP = true>
__device__ __forceinline__ void t_orbit(const TRecord& rc, cx_t<R>* const* base, size_t st_stride,
                                        const int (&cbr)[CS + 1], int KV, int kv0, int kv1,
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
  const uint32_t fls = rc.flips;
  for (int kv = kv0; kv < kv1; ++kv) {
    C ps[NS], pg[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if constexpr (PK) {
        // packed cell (Re psi, Re g, Im psi, Im g), signs flipped by omega
        const float4 t = reinterpret_cast<const float4*>(base[0])[ad[k] + kv];
        const uint32_t sg = ((fls >> k) & 1u) << 31;
        ps[k] = mk<R>(__uint_as_float(__float_as_uint(t.x) ^ sg),
                      __uint_as_float(__float_as_uint(t.z) ^ sg));
        pg[k] = mk<R>(__uint_as_float(__float_as_uint(t.y) ^ sg),
                      __uint_as_float(__float_as_uint(t.w) ^ sg));
      } else {
        C* b0 = base[CS > 1 ? own[k] : 0];
        ps[k] = b0[ad[k] + kv];
        pg[k] = b0[st_stride + ad[k] + kv];
        if ((fls >> k) & 1u) {
          ps[k].x = -ps[k].x;
          ps[k].y = -ps[k].y;
          pg[k].x = -pg[k].x;
          pg[k].y = -pg[k].y;
        }
      }
    }
    t_terms<R, M, NS, DIAG, KEEP>(ps, pg, acc, keep, std::make_integer_sequence<int, 6 * 16>{});
  }
}

// One record of a transition pass, by its class and whether the pass
// evaluates diagonal slots.  Every evaluated slot is accumulated; slots the
// pass does not own (pairs an inexact covering repeats, diagonals owned
// elsewhere) are dropped when the pass's sums are reduced, which costs a few
// repeated multiply-adds instead of a test per slot and string.
template <typename R, int CS, bool PK>
__device__ __forceinline__ void t_record(bool diag, const TRecord& rc, cx_t<R>* const* base,
                                         size_t st_stride, const int (&cbr)[CS + 1], int KV,
                                         int kv0, int kv1, R (&acc)[32], uint32_t keep) {
  if (!diag) {
    switch (rc.m) {
      case 1: t_orbit<R, CS, 1, PK, false, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
      case 2: t_orbit<R, CS, 2, PK, false, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
      case 3: t_orbit<R, CS, 3, PK, false, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
      case 4: t_orbit<R, CS, 4, PK, false, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
      default: break;
    }
    return;
  }
  switch (rc.m) {
    case 1: t_orbit<R, CS, 1, PK, true, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
    case 2: t_orbit<R, CS, 2, PK, true, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
    case 3: t_orbit<R, CS, 3, PK, true, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
    case 4: t_orbit<R, CS, 4, PK, true, false>(rc, base, st_stride, cbr, KV, kv0, kv1, acc, keep); break;
    default: break;
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
          bool TC = false, bool PK = false>
__device__ __forceinline__ void sweep_body(const SweepGeom& g, const P& prog, const Mat& X,
                                           const int slab, const int rank,
                                           unsigned char* smraw) {
  static_assert(!VJP || NST == 2, "reverse mode carries two states");
  static_assert(!SPLIT || (NST == 2 && W > 0), "split mode: two states, window sweeps");
  static_assert(!PK || (CS == 1 && sizeof(R) == 4 && W > 0 && !SPLIT && !TC),
                "packed slabs: complex64 window sweeps in one CTA");
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
  float* const smf = reinterpret_cast<float*>(smraw);
  // amplitude (state s, string el, vector kv) of the slab
  auto slab_get = [&](int s, size_t el, int kv) -> C {
    if constexpr (PK) {
      const size_t r = pk_re<NST>(s, el, KV, kv);
      return mk<R>(smf[r], smf[r + 2]);
    } else {
      return sm[s * st_stride + el * KV + kv];
    }
  };
  auto slab_set = [&](int s, size_t el, int kv, C v) {
    if constexpr (PK) {
      const size_t r = pk_re<NST>(s, el, KV, kv);
      smf[r] = v.x;
      smf[r + 2] = v.y;
    } else {
      sm[s * st_stride + el * KV + kv] = v;
    }
  };
  for (int s = 0; s < NST; ++s) {
    const C* gs = reinterpret_cast<const C*>(g.st[s]);
    C* ss = sm + s * st_stride;
    if constexpr (PK) {
      // the real and imaginary parts go to their lanes of the packed cells
      const float* gf = reinterpret_cast<const float*>(g.st[s]);
      if (g.dir == 1) {
        DivWalk dw(tid, kThreads, nel > 0 ? nel : 1);
        for (int idx = tid; idx < kv_eff * nel; idx += kThreads, dw.next()) {
          const int kv = dw.a, el = dw.b;
          const size_t r = pk_re<NST>(s, el, KV, kv);
          const float* src = gf + 2 * ((int64_t)(v0 + kv) * g.d_b + e0 + el);
          cp_async_4(smf + r, src);
          cp_async_4(smf + r + 2, src + 1);
        }
      } else {
        for (int idx = tid; idx < (nel << g.lgKV); idx += kThreads) {
          const int el = idx >> g.lgKV, kv = idx & (KV - 1);
          if (kv >= kv_eff) continue;
          const size_t r = pk_re<NST>(s, el, KV, kv);
          const float* src = gf + 2 * ((int64_t)(e0 + el) * g.d_b + v0 + kv);
          cp_async_4(smf + r, src);
          cp_async_4(smf + r + 2, src + 1);
        }
      }
      continue;
    }
    if (g.dir == 1) {
      DivWalk dw(tid, kThreads, nel > 0 ? nel : 1);
      for (int idx = tid; idx < kv_eff * nel; idx += kThreads, dw.next()) {
        const int kv = dw.a, el = dw.b;
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
      const int ga = prog.g0[st], gb = prog.g0[st + 1], pid = prog.pat[st];
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
          case 1: win_orbit<R, CS, 1, W, 1>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 2: win_orbit<R, CS, 1, W, 2>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 3: win_orbit<R, CS, 1, W, 3>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 4: if constexpr (W > 4) win_orbit<R, CS, 1, W, 4>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 5: if constexpr (W > 5) win_orbit<R, CS, 1, W, 5>(desc, F, bs, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
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
      const int ga = prog.g0[st], gb = prog.g0[st + 1], pid = prog.pat[st];
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
      if constexpr (PK) {
        // packed cells (vector pairs of one state, or psi and g); the work
        // items are (orbit, packed set) pairs, chunk by chunk of 32 orbits
        // (a class boundary never falls inside a chunk), so that short
        // vectors with few orbits per step still fill the CTA
        const int KC = NST == 1 ? (KV >> 1) : KV;
        const int nk = NST == 1 ? (kv_eff + 1) >> 1 : kv_eff;
        const int nit = (hi - lo) * nk;
        // the descriptor of the next round is loaded while this one runs
        auto item_orbit = [&](int it) {
          const int ch = it >> 5, oc = nk == 1 ? ch : ch / nk;
          return lo + (oc << 5) + (it & 31);
        };
        int it_next = dealt_round<kThreads>(0, nit, 0, 0, 1) ? dealt_item<kThreads>(0, nit, 0, tid, 0, 1) : -1;
        uint32_t desc_next = it_next >= 0 ? __ldg(olist + item_orbit(it_next)) : 0u;
        for (int rd = 0; dealt_round<kThreads>(0, nit, rd, 0, 1); ++rd) {
          const int it = it_next;
          const uint32_t desc = desc_next;
          it_next = dealt_round<kThreads>(0, nit, rd + 1, 0, 1)
                        ? dealt_item<kThreads>(0, nit, rd + 1, tid, 0, 1)
                        : -1;
          if (it_next >= 0) desc_next = __ldg(olist + item_orbit(it_next));
          if (it < 0) continue;
          const int ch = it >> 5, oc = nk == 1 ? ch : ch / nk;
          const int kc = ch - oc * nk;
          switch (desc >> 24) {
            case 1: win_orbit_pk<W, 1>(desc, F, smf, KC, kc, prog, ga, gb); break;
            case 2: win_orbit_pk<W, 2>(desc, F, smf, KC, kc, prog, ga, gb); break;
            case 3: win_orbit_pk<W, 3>(desc, F, smf, KC, kc, prog, ga, gb); break;
            case 4: if constexpr (W > 4) win_orbit_pk<W, 4>(desc, F, smf, KC, kc, prog, ga, gb); break;
            case 5: if constexpr (W > 5) win_orbit_pk<W, 5>(desc, F, smf, KC, kc, prog, ga, gb); break;
            default: break;
          }
        }
        __syncthreads();
        continue;
      }
      for (int rd = 0; dealt_round<kThreads>(lo, hi, rd, drank, dcs); ++rd) {
        const int o = dealt_item<kThreads>(lo, hi, rd, tid, drank, dcs);
        if (o < 0) continue;
        const uint32_t desc = __ldg(olist + o);
        switch (desc >> 24) {
          case 1: win_orbit<R, CS, NST, W, 1>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 2: win_orbit<R, CS, NST, W, 2>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 3: win_orbit<R, CS, NST, W, 3>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 4: if constexpr (W > 4) win_orbit<R, CS, NST, W, 4>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
          case 5: if constexpr (W > 5) win_orbit<R, CS, NST, W, 5>(desc, F, base, st_stride, cbr, KV, kv_eff, prog, ga, gb, pid); break;
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
    DivWalk dw(tid, kThreads, nel > 0 ? nel : 1);
    for (int idx = tid; idx < tot; idx += kThreads, dw.next()) {
      int kv, el;
      if (g.dir == 1) {
        kv = dw.a;
        el = dw.b;
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
        C v = cmul<R>(f, slab_get(s, (size_t)el, kv));
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
      for (int s = 0; s < 2; ++s) slab_set(s, (size_t)el, kv, cmul<R>(f, slab_get(s, (size_t)el, kv)));
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
      if constexpr (CS == 1 && PK) {
        // one CTA: each warp takes whole units (pass ip, chunks c = qq mod 4
        // of its (record, vector) items, 32 records a chunk, interleaved so
        // that the units of a pass carry the same mix of classes) and
        // reduces once per unit; units are dealt round-robin over the
        // warps in pass order, so the passes that also own diagonals (the
        // first ones of the covering) fall on different warps
        const int warp = tid >> 5, nkv = kv_eff;
        for (int u = warp; u < g.npass * 4; u += kThreads / 32) {
          const int ip = u >> 2, qq = u & 3;
          const TPassDev pd = g.tpass[ip];
          R acc[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] = 0;
          const int nch = ((pd.rec1 - pd.rec0) >> 5) * nkv;
          // chunk ch = (record chunk oc, vector kv0), walked without a
          // division per chunk; the record of the next chunk is loaded
          // while this one runs
          auto rec_of = [&](int oc) {
            return __ldg(reinterpret_cast<const uint4*>(g.trec + pd.rec0 + (oc << 5) + lane));
          };
          DivWalk cw(qq, 4, nkv);
          uint4 rnext = qq < nch ? rec_of(cw.a) : make_uint4(0, 0, 0, 0);
          for (int ch = qq; ch < nch; ch += 4) {
            const int kv0 = cw.b;
            cw.next();
            TRecord rc;
            *reinterpret_cast<uint4*>(&rc) = rnext;
            if (ch + 4 < nch) rnext = rec_of(cw.a);
            t_record<R, CS, PK>((pd.keep & 0x8421u) != 0, rc, base, st_stride, cbr, KV, kv0, kv0 + 1, acc, pd.keep);
          }
          const R v = warp_transpose_sum<R>(acc, lane);
          if (pd.keep & (1u << (lane >> 1))) atomicAdd(tsm + ip * 32 + lane, v);
        }
      } else {
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
        // packed slabs: (record, vector) items, chunk by chunk of 32 records
        // (short vectors with few records per pass still fill the CTA)
        const int nkv = PK ? kv_eff : 1;
        const int ilo = PK ? 0 : lo, ihi = PK ? (hi - lo) * nkv : hi;
        for (int rd = 0; dealt_round<kThreads>(ilo, ihi, rd, drank, dcs); ++rd) {
          const int it = dealt_item<kThreads>(ilo, ihi, rd, tid, drank, dcs);
          if (it < 0) continue;
          int o = it, kv0 = 0, kv1 = kv_eff;
          if constexpr (PK) {
            const int ch = it >> 5, oc = nkv == 1 ? ch : ch / nkv;
            o = lo + (oc << 5) + (it & 31);
            kv0 = ch - oc * nkv;
            kv1 = kv0 + 1;
          }
          TRecord rc;
          *reinterpret_cast<uint4*>(&rc) = __ldg(reinterpret_cast<const uint4*>(rlist + o));
          t_record<R, CS, PK>((pd.keep & 0x8421u) != 0, rc, base, st_stride, cbr, KV, kv0, kv1,
                              acc, pd.keep);
        }
        const R v = warp_transpose_sum<R>(acc, lane);
        if (pd.keep & (1u << (lane >> 1))) atomicAdd(tsm + ip * 32 + lane, v);
      }
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
              C a, b;
              if constexpr (PK) {
                a = slab_get(0, (size_t)src, kv);
                b = slab_get(1, (size_t)dst, kv);
              } else {
                a = ps[kv];
                b = pg[kv];
              }
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
    DivWalk dw(tid, kThreads, nel > 0 ? nel : 1);
    for (int idx = tid; idx < tot; idx += kThreads, dw.next()) {
      int kv, el;
      if (g.dir == 1) {
        kv = dw.a;
        el = dw.b;
      } else {
        el = idx >> g.lgKV;
        kv = idx & (KV - 1);
        if (kv >= kv_eff) continue;
      }
      const int o = v0 + kv, e = e0 + el;
      const int64_t gi = g.dir == 1 ? (int64_t)o * g.d_b + e : (int64_t)e * g.d_b + o;
      C ps = slab_get(0, (size_t)el, kv);
      C pg = slab_get(1, (size_t)el, kv);
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

template <typename R, int CS, int NST, bool VJP, int W, int NT, bool SPLIT, bool TC = false,
          bool PK = false>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
    k_sweep(const SweepGeom g, const __grid_constant__ typename ProgOf<R, W, (W > 0)>::type prog,
            const __grid_constant__ Mat X) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  sweep_body<R, CS, NST, VJP, W, NT, SPLIT, typename ProgOf<R, W, (W > 0)>::type, TC, PK>(
      g, prog, X, blockIdx.x / CS, rank, smraw);
}

// Batched sweep: one persistent launch over the slabs of many jobs (one job
// per circuit), taken from an atomic work counter in job order.
template <typename R, int NST, bool VJP, int W, int NT, bool SPLIT, bool PK = false>
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
    sweep_body<R, 1, NST, VJP, W, NT, SPLIT, WProg<R>, false, PK>(
        J.g, *reinterpret_cast<const WProg<R>*>(J.prog),
                                             *J.X, it - J.item0, 0, smraw);
    __syncthreads();
  }
}

// Window width of the register-blocked sweep per precision and state count,
// chosen so one orbit of every vector fits in registers.
template <typename R, int NST>
constexpr int window_width() {
  return sizeof(R) == 4 ? (NST == 1 ? 6 : 5) : (NST == 1 ? 5 : 4);
}

template <typename R, int CS, int NST, bool VJP, int W, int NT, bool SPLIT, typename P,
          bool TC = false, bool PK = false>
void launch_sweep_t(const SweepGeom& g, const P& prog, const Mat& X,
                           int nslabs, size_t smem, cudaStream_t st) {
  auto kern = k_sweep<R, CS, NST, VJP, W, NT, SPLIT, TC, PK>;
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
void dispatch_cs(int CS, const SweepGeom& g, const P& prog, const Mat& X,
                        int nslabs, size_t smem, cudaStream_t st) {
  switch (CS) {
    case 1: launch_sweep_t<R, 1, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    case 2: launch_sweep_t<R, 2, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    case 4: launch_sweep_t<R, 4, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    case 8: launch_sweep_t<R, 8, NST, VJP, W, NT, SPLIT>(g, prog, X, nslabs, smem, st); break;
    default: FS_REQUIRE(false, FS_ERR_UNSUPPORTED, "cluster size out of range");
  }
}

template <typename R, int NST, bool VJP, int W, int NT, bool SPLIT, bool PK = false>
void launch_batch_t(const SweepJob* jobs, int njobs, int total, int* counter, size_t smem,
                           int grid, cudaStream_t st) {
  auto kern = k_sweep_batch<R, NST, VJP, W, NT, SPLIT, PK>;
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

}  // namespace fs
