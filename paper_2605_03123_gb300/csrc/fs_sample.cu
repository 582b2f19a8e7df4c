// Sampling configurations.
//
// From a state (sample-based algorithms section): configuration a (row-major
// address i * dim_b + j) is drawn with probability |psi_a|^2 / ||psi||^2, as
// the inverse of the cumulative distribution in address order: for a uniform
// u the sample is the first a whose inclusive prefix sum of |psi|^2 exceeds
// u * ||psi||^2.  The prefix is held at three levels: groups of 256
// amplitudes, tiles of 256 groups, and the tiles.  One streaming pass
// (k_cdf_groups) writes each group's inclusive prefix inside its tile; one
// CTA (k_cdf_tiles) forms the inclusive prefix of the tile totals; one warp
// per shot (k_sample_state) then searches tile, group and amplitude.
//
// Arithmetic: complex128 states accumulate in FP64.  complex64 states
// accumulate in double-float pairs (hi + lo, FP32 each, a ~48-bit
// significand): the squares of FP32 components are split exactly with FMA
// and summed with error-free transformations, because GB300's FP64 rate is
// a small fraction of its FP32 rate and FP64 sums would hold the pass well
// below HBM speed.  Prefixes inside a tile and across tiles are built as
// E_{k+1} = E_k + T_k in sequence, so a group or tile of zero mass has a
// prefix equal to its predecessor's and no search can land on it; every
// search also clamps its target to [0, level total], so rounding differences
// between the levels never select a configuration of zero probability.
//
// From a Slater determinant (Slater-sampling section): for one spin with
// occupied columns Phi = U[:, occ] the configuration is a determinantal point
// process with kernel K = Phi Phi^dag (a projector of rank n).  The chain rule
// picks one orbital per step: p with probability w_p / sum(w), where w_q is
// the squared distance of row q of Phi from the span of the rows already
// picked.  Here w is updated by Gram-Schmidt against K's columns:
//   c_i(q) = (K_qp - sum_{l<i} c_l(q) conj(c_l(p))) / sqrt(w_p),
//   w_q   <- w_q - |c_i(q)|^2,
// which equals projecting the rows of Phi onto the complement of the picked
// row, at O(N i) per step.  One CTA per shot, FP64 (the decisions are
// integers taken in the paper's precision).
#include <algorithm>
#include <cmath>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

constexpr int kGroup = 256;       // amplitudes per group
constexpr int kTileGroups = 256;  // groups per tile

// --------------------------------------------------------- accumulators
// Double-float number h + l with |l| <= ulp(h) / 2 (normalised).
struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return dfl{s, b - (s - a)};
}
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfl{s, (a - (s - bb)) + (b - bb)};
}

template <typename R> struct Acc;

template <> struct Acc<float> {
  using T = dfl;
  static __device__ __forceinline__ T zero() { return dfl{0.f, 0.f}; }
  static __device__ __forceinline__ T add(T a, T b) {
    const dfl s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + (a.l + b.l));
  }
  static __device__ __forceinline__ T neg(T a) { return dfl{-a.h, -a.l}; }
  static __device__ __forceinline__ bool gt(T a, T b) {
    return a.h > b.h || (a.h == b.h && a.l > b.l);
  }
  static __device__ __forceinline__ bool ge(T a, T b) {
    return a.h > b.h || (a.h == b.h && a.l >= b.l);
  }
  static __device__ __forceinline__ bool pos(T a) { return a.h > 0.f; }
  static __device__ __forceinline__ bool finite(T a) { return isfinite(a.h) && isfinite(a.l); }
  // |z|^2 of a complex64 amplitude: the squares split exactly by FMA
  static __device__ __forceinline__ T prob(float2 z) {
    const float h1 = z.x * z.x, l1 = fmaf(z.x, z.x, -h1);
    const float h2 = z.y * z.y, l2 = fmaf(z.y, z.y, -h2);
    const dfl s = two_sum(h1, h2);
    return fast_two_sum(s.h, s.l + (l1 + l2));
  }
  // u * a for a uniform u = uh + ul split into two floats
  static __device__ __forceinline__ T scale(float uh, float ul, T a) {
    const float p = uh * a.h;
    const float e = fmaf(uh, a.h, -p) + (uh * a.l + ul * a.h);
    return fast_two_sum(p, e);
  }
  // the uniform of a shot, read and split on lane 0 only (FP64 issue is
  // scarce on GB300), then broadcast; NaN reads as 0
  static __device__ __forceinline__ void uniform(const double* u, int64_t s, int lane,
                                                 float& uh, float& ul) {
    float h = 0.f, l = 0.f;
    if (lane == 0) {
      const double x = u[s];
      if (x == x) {
        h = (float)x;
        l = (float)(x - (double)h);
      }
    }
    uh = __shfl_sync(0xffffffffu, h, 0);
    ul = __shfl_sync(0xffffffffu, l, 0);
  }
  static __device__ __forceinline__ T shfl_up(T a, int d) {
    return dfl{__shfl_up_sync(0xffffffffu, a.h, d), __shfl_up_sync(0xffffffffu, a.l, d)};
  }
  static __device__ __forceinline__ T shfl_xor(T a, int m) {
    return dfl{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
  }
};

template <> struct Acc<double> {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ bool gt(T a, T b) { return a > b; }
  static __device__ __forceinline__ bool ge(T a, T b) { return a >= b; }
  static __device__ __forceinline__ bool pos(T a) { return a > 0.0; }
  static __device__ __forceinline__ bool finite(T a) { return isfinite(a); }
  static __device__ __forceinline__ T prob(double2 z) { return fma(z.x, z.x, z.y * z.y); }
  static __device__ __forceinline__ T scale(double u, double, T a) { return u * a; }
  static __device__ __forceinline__ void uniform(const double* u, int64_t s, int, double& uh,
                                                 double& ul) {
    const double x = u[s];
    uh = x == x ? x : 0.0;
    ul = 0.0;
  }
  static __device__ __forceinline__ T shfl_up(T a, int d) {
    return __shfl_up_sync(0xffffffffu, a, d);
  }
  static __device__ __forceinline__ T shfl_xor(T a, int m) {
    return __shfl_xor_sync(0xffffffffu, a, m);
  }
};

// ----------------------------------------------------- CDF of a state
// One CTA per tile (grid-stride), 8 warps; warp w sums groups w, w + 8, ...
// of the tile (each lane 8 amplitudes in 16-byte loads), then warp 0 turns
// the 256 group sums into the tile-local inclusive prefix gc[] and the tile
// total tsum[].
template <typename R>
__global__ void __launch_bounds__(256)
    k_cdf_groups(const cx_t<R>* __restrict__ v, int64_t n, int64_t ngroups, int64_t ntiles,
                 typename Acc<R>::T* __restrict__ gc, typename Acc<R>::T* __restrict__ tsum) {
  using A = Acc<R>;
  using T = typename A::T;
  __shared__ T gs[kTileGroups];
  __shared__ T lane_tot[32];
  __shared__ T lane_off[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int gi = warp; gi < kTileGroups; gi += 8) {
      const int64_t g = tile * kTileGroups + gi;
      T s = A::zero();
      if (g < ngroups) {
        const int64_t a0 = g * kGroup;
        if (a0 + kGroup <= n) {
          if constexpr (sizeof(R) == 4) {
            const float4* p4 = reinterpret_cast<const float4*>(v + a0);
            float4 q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = __ldcs(p4 + lane + 32 * k);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              s = A::add(s, A::prob(make_float2(q[k].x, q[k].y)));
              s = A::add(s, A::prob(make_float2(q[k].z, q[k].w)));
            }
          } else {
            cx_t<R> q[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) q[k] = __ldcs(v + a0 + lane + 32 * k);
#pragma unroll
            for (int k = 0; k < 8; ++k) s = A::add(s, A::prob(q[k]));
          }
        } else {
          for (int64_t a = a0 + lane; a < n; a += 32) s = A::add(s, A::prob(v[a]));
        }
      }
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) s = A::add(s, A::shfl_xor(s, m));
      if (lane == 0) gs[gi] = s;
    }
    __syncthreads();
    if (warp == 0) {
      // lane l: groups 8l .. 8l+7 in sequence; lane offsets chained in sequence
      T loc[8];
      T run = A::zero();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        run = A::add(run, gs[8 * lane + k]);
        loc[k] = run;
      }
      lane_tot[lane] = run;
      __syncwarp();
      if (lane == 0) {
        T e = A::zero();
        for (int l = 0; l < 32; ++l) {
          lane_off[l] = e;
          e = A::add(e, lane_tot[l]);
        }
        tsum[tile] = e;
      }
      __syncwarp();
      const T off = lane_off[lane];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t g = tile * kTileGroups + 8 * lane + k;
        if (g < ngroups) gc[g] = lane == 0 ? loc[k] : A::add(off, loc[k]);
      }
    }
    __syncthreads();
  }
}

// Inclusive prefix of the tile totals, one CTA of 1024 threads: each thread
// a contiguous chunk in sequence, chunk offsets chained in sequence.
template <typename R>
__global__ void __launch_bounds__(1024)
    k_cdf_tiles(const typename Acc<R>::T* __restrict__ tsum, int64_t ntiles,
                typename Acc<R>::T* __restrict__ tc) {
  using A = Acc<R>;
  using T = typename A::T;
  __shared__ T tot[1024];
  const int64_t chunk = (ntiles + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = min(ntiles, (int64_t)threadIdx.x * chunk), b1 = min(ntiles, b0 + chunk);
  T run = A::zero();
  for (int64_t t = b0; t < b1; ++t) run = A::add(run, tsum[t]);
  tot[threadIdx.x] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    T e = A::zero();
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const T x = tot[k];
      tot[k] = e;
      e = A::add(e, x);
    }
  }
  __syncthreads();
  const T acc = tot[threadIdx.x];
  const bool first = threadIdx.x == 0;
  T loc = A::zero();
  for (int64_t t = b0; t < b1; ++t) {
    loc = A::add(loc, tsum[t]);
    tc[t] = first ? loc : A::add(acc, loc);
  }
}

// First k in [lo, hi) with a[k] > x (a[k] >= x when ge), for an a whose
// a[hi - 1] satisfies the test: 32-ary search, each lane probing the end of
// one of 32 equal chunks.  The result k satisfies the test and k == lo or
// a[k - 1] fails it.
template <typename A>
__device__ __forceinline__ int64_t warp_search(const typename A::T* a, int64_t lo, int64_t hi,
                                               typename A::T x, bool ge, int lane) {
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t pos = lo + (int64_t)(lane + 1) * step - 1;
    bool ok = true;
    if (pos < hi - 1) {
      const typename A::T y = a[pos];
      ok = ge ? A::ge(y, x) : A::gt(y, x);
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    const int f = __ffs(m) - 1;  // m != 0: the last probe is at or beyond hi - 1
    const int64_t nlo = f == 0 ? lo : lo + (int64_t)f * step;
    const int64_t nhi = min(hi, lo + (int64_t)(f + 1) * step);
    lo = nlo;
    hi = nhi;
  }
  return lo;
}

// One warp per shot: tile, then group, then amplitude.
template <typename R>
__global__ void __launch_bounds__(256)
    k_sample_state(const cx_t<R>* __restrict__ v, int64_t n, int64_t ngroups, int64_t ntiles,
                   const typename Acc<R>::T* __restrict__ gc,
                   const typename Acc<R>::T* __restrict__ tc, const double* __restrict__ u,
                   int64_t shots, int64_t* __restrict__ out) {
  using A = Acc<R>;
  using T = typename A::T;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const T total = tc[ntiles - 1];
  const bool usable = A::finite(total) && A::pos(total);
  for (int64_t s = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); s < shots;
       s += warps) {
    if (!usable) {
      if (lane == 0) out[s] = -1;
      continue;
    }
    R uh, ul;
    A::uniform(u, s, lane, uh, ul);
    T x = A::scale(uh, ul, total);
    if (!A::pos(x)) x = A::zero();
    bool ge = false;
    if (!A::gt(total, x)) {
      x = total;
      ge = true;
    }
    // tile
    const int64_t t = warp_search<A>(tc, 0, ntiles, x, ge, lane);
    T xt = t > 0 ? A::add(x, A::neg(tc[t - 1])) : x;
    if (!A::pos(xt)) xt = A::zero();
    // group inside the tile
    const int64_t g0 = t * kTileGroups, g1 = min(ngroups, g0 + kTileGroups);
    const T ttot = gc[g1 - 1];
    ge = false;
    if (!A::gt(ttot, xt)) {
      xt = ttot;
      ge = true;
    }
    const int64_t g = warp_search<A>(gc, g0, g1, xt, ge, lane);
    T xg = g > g0 ? A::add(xt, A::neg(gc[g - 1])) : xt;
    if (!A::pos(xg)) xg = A::zero();
    // amplitude inside the group: lane l holds 8 consecutive amplitudes
    const int64_t a0 = g * kGroup + 8 * lane;
    const int64_t left = n - a0;
    const int cnt = left <= 0 ? 0 : (left >= 8 ? 8 : (int)left);
    T p[8];
    T own = A::zero();
    cx_t<R> z[8];
    if (cnt == 8) {
      if constexpr (sizeof(R) == 4) {
        const float4* p4 = reinterpret_cast<const float4*>(v + a0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 q = p4[k];
          z[2 * k] = make_float2(q.x, q.y);
          z[2 * k + 1] = make_float2(q.z, q.w);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) z[k] = v[a0 + k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) z[k] = k < cnt ? v[a0 + k] : cx_t<R>{};
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      p[k] = k < cnt ? A::prob(z[k]) : A::zero();
      own = A::add(own, p[k]);
    }
    T incl = own;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const T y = A::shfl_up(incl, d);
      if (lane >= d) incl = A::add(y, incl);
    }
    T excl = A::shfl_up(incl, 1);
    if (lane == 0) excl = A::zero();
    const unsigned has = __ballot_sync(0xffffffffu, A::pos(own));
    const unsigned crosses = __ballot_sync(0xffffffffu, A::gt(incl, xg)) & has;
    int f;
    bool scan;
    if (crosses) {
      f = __ffs(crosses) - 1;  // first crossing lane that holds mass
      scan = true;
    } else {
      f = has ? 31 - __clz(has) : 0;  // the last lane that holds mass
      scan = false;
    }
    if (lane == f) {
      int pick = -1, last = -1;
      T xl = A::add(xg, A::neg(excl));
      if (!A::pos(xl)) xl = A::zero();
      T run = A::zero();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (A::pos(p[k])) last = k;
        run = A::add(run, p[k]);
        if (scan && pick < 0 && A::pos(p[k]) && A::gt(run, xl)) pick = k;
      }
      if (pick < 0) pick = last;
      out[s] = pick < 0 ? -1 : a0 + pick;
    }
  }
}

// ------------------------------------------------- Slater determinants
// K[p][q] = sum_j Phi[p][j] conj(Phi[q][j]) (FP64), Phi = U[:, occ] (N x n).
__global__ void k_projector(double2* __restrict__ K, const double2* __restrict__ Phi, int N,
                            int n) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  const int p = (int)(idx / N), q = (int)(idx - (int64_t)p * N);
  double re = 0, im = 0;
  for (int j = 0; j < n; ++j) {
    const double2 a = Phi[(int64_t)p * n + j], b = Phi[(int64_t)q * n + j];
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.y, b.x, fma(-a.x, b.y, im));
  }
  K[idx] = make_double2(re, im);
}

// One CTA per shot (grid-stride).  Thread t owns rows [t R, t R + R).  C
// (n x N complex, the Gram-Schmidt coefficients) lives in shared memory when
// it fits, else in this CTA's slot of global scratch.
__global__ void __launch_bounds__(256)
    k_sample_slater(const double2* __restrict__ K, int N, int n, const double* __restrict__ u,
                    int64_t shots, uint64_t* __restrict__ out, int words,
                    double2* __restrict__ cglob, int c_in_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int64_t cbytes = c_in_smem ? (int64_t)n * N * 16 : 0;
  double2* C = c_in_smem ? reinterpret_cast<double2*>(smraw)
                         : cglob + (int64_t)blockIdx.x * n * N;
  double* w = reinterpret_cast<double*>(smraw + cbytes);          // N
  double* wtot = w + N;                                           // 8 warp totals
  unsigned long long* mask = reinterpret_cast<unsigned long long*>(wtot + 8);  // words
  int* pick_sm = reinterpret_cast<int*>(mask + words);  // pick, thread, scan flag
  double* wp_sm = reinterpret_cast<double*>(pick_sm + 4);         // w of the pick
  const int B = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (B + 31) >> 5;
  const int R = (N + B - 1) / B;
  const int r0 = min(N, tid * R), r1 = min(N, r0 + R);
  for (int64_t s = blockIdx.x; s < shots; s += gridDim.x) {
    for (int q = r0; q < r1; ++q) w[q] = K[(int64_t)q * N + q].x;
    for (int k = tid; k < words; k += B) mask[k] = 0ull;
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      // inverse CDF over the orbitals in increasing order
      double own = 0;
      for (int q = r0; q < r1; ++q) own += w[q];
      double incl = own;
      for (int d = 1; d < 32; d <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      if (lane == 31) wtot[warp] = incl;
      __syncthreads();
      double woff = 0, total = 0;
      for (int k = 0; k < nw; ++k) {
        if (k < warp) woff += wtot[k];
        total += wtot[k];
      }
      incl += woff;
      const double excl = incl - own;
      double x = u[s * n + i] * total;
      if (!(x > 0)) x = 0;
      const bool ge = !(x < total);
      if (ge) x = total;
      const bool has = own > 0;
      const bool cr = has && (ge ? incl >= x : incl > x);
      // first crossing thread with mass, else the last thread with mass
      const unsigned mc = __ballot_sync(0xffffffffu, cr), mh = __ballot_sync(0xffffffffu, has);
      __syncthreads();  // everyone has read wtot
      if (lane == 0) {
        reinterpret_cast<int*>(wtot)[2 * warp] = mc ? (__ffs(mc) - 1) : -1;
        reinterpret_cast<int*>(wtot)[2 * warp + 1] = mh ? (31 - __clz(mh)) : -1;
      }
      __syncthreads();
      if (tid == 0) {
        int chosen = -1, scan = 1;
        for (int k = 0; k < nw && chosen < 0; ++k) {
          const int f = reinterpret_cast<int*>(wtot)[2 * k];
          if (f >= 0) chosen = 32 * k + f;
        }
        if (chosen < 0) {
          scan = 0;
          for (int k = nw - 1; k >= 0 && chosen < 0; --k) {
            const int f = reinterpret_cast<int*>(wtot)[2 * k + 1];
            if (f >= 0) chosen = 32 * k + f;
          }
        }
        if (chosen < 0) {  // no mass left: impossible for orthonormal columns
          chosen = 0;
          scan = 0;
        }
        pick_sm[1] = chosen;
        pick_sm[2] = scan;
      }
      __syncthreads();
      if (tid == pick_sm[1]) {
        const int scan = pick_sm[2];
        double xl = x - excl;
        if (!(xl > 0)) xl = 0;
        int pick = -1, last = -1;
        double run = 0;
        for (int q = r0; q < r1; ++q) {
          const double wq = w[q];
          if (wq > 0) last = q;
          run += wq;
          if (scan && pick < 0 && wq > 0 && (ge ? run >= xl : run > xl)) pick = q;
        }
        if (pick < 0) pick = last >= 0 ? last : 0;
        pick_sm[0] = pick;
        wp_sm[0] = w[pick];
        mask[pick >> 6] |= 1ull << (pick & 63);
      }
      __syncthreads();
      const int p = pick_sm[0];
      const double rinv = 1.0 / sqrt(wp_sm[0]);
      const double2* Kp = K + (int64_t)p * N;
      for (int q = r0; q < r1; ++q) {
        const double2 kpq = Kp[q];  // K_qp = conj(K_pq)
        double ar = kpq.x, ai = -kpq.y;
        for (int l = 0; l < i; ++l) {
          const double2 cq = C[(int64_t)l * N + q], cp = C[(int64_t)l * N + p];
          // cq * conj(cp)
          ar -= fma(cq.x, cp.x, cq.y * cp.y);
          ai -= fma(cq.y, cp.x, -cq.x * cp.y);
        }
        const double cre = ar * rinv, cim = ai * rinv;
        C[(int64_t)i * N + q] = make_double2(cre, cim);
        const double wn = w[q] - fma(cre, cre, cim * cim);
        w[q] = q == p ? 0.0 : (wn > 0 ? wn : 0.0);
      }
      __syncthreads();
    }
    for (int k = tid; k < words; k += B) out[s * words + k] = mask[k];
    __syncthreads();
  }
}

// ------------------------------------------------------------- launch
void sample_state(Ctx* ctx, const void* vec, int dtype, int64_t n, const double* u,
                  int64_t shots, int64_t* out, cudaStream_t st) {
  if (shots == 0) return;
  const int64_t ngroups = (n + kGroup - 1) / kGroup;
  const int64_t ntiles = (ngroups + kTileGroups - 1) / kTileGroups;
  const size_t acc = 8;  // dfl and double are both 8 bytes
  char* ws = (char*)scratch(ctx, "sample_cdf", (size_t)(ngroups + 2 * ntiles) * acc);
  const int sms = ctx->prop.multiProcessorCount;
  const unsigned g1 = (unsigned)std::min<int64_t>(ntiles, (int64_t)1 << 30);
  const int g3 = (int)std::max<int64_t>(
      1, std::min<int64_t>((shots + 7) / 8, (int64_t)sms * 16));
  if (dtype == FS_C64) {
    using T = Acc<float>::T;
    T* gc = (T*)ws;
    T* ts = gc + ngroups;
    T* tc = ts + ntiles;
    {
      ProfScope ps("sample_cdf", st);
      k_cdf_groups<float><<<g1, 256, 0, st>>>((const float2*)vec, n, ngroups, ntiles, gc, ts);
    }
    {
      ProfScope ps("sample_cdf_tiles", st);
      k_cdf_tiles<float><<<1, 1024, 0, st>>>(ts, ntiles, tc);
    }
    ProfScope ps("sample_search", st);
    k_sample_state<float><<<g3, 256, 0, st>>>((const float2*)vec, n, ngroups, ntiles, gc, tc, u,
                                              shots, out);
  } else {
    using T = Acc<double>::T;
    T* gc = (T*)ws;
    T* ts = gc + ngroups;
    T* tc = ts + ntiles;
    {
      ProfScope ps("sample_cdf", st);
      k_cdf_groups<double><<<g1, 256, 0, st>>>((const double2*)vec, n, ngroups, ntiles, gc, ts);
    }
    {
      ProfScope ps("sample_cdf_tiles", st);
      k_cdf_tiles<double><<<1, 1024, 0, st>>>(ts, ntiles, tc);
    }
    ProfScope ps("sample_search", st);
    k_sample_state<double><<<g3, 256, 0, st>>>((const double2*)vec, n, ngroups, ntiles, gc, tc,
                                               u, shots, out);
  }
  FS_CUDA(cudaGetLastError());
}

void sample_slater(Ctx* ctx, const std::vector<zd>& Phi, int N, int n, const double* u,
                   int64_t shots, uint64_t* out, cudaStream_t st) {
  if (shots == 0) return;
  const int words = (N + 63) / 64;
  const size_t kbytes = (size_t)N * N * 16, pbytes = (size_t)N * n * 16;
  const int B = std::min(256, ((N + 31) / 32) * 32);
  const size_t base = (size_t)N * 8 + 8 * 8 + (size_t)words * 8 + 16 + 16;
  const size_t cbytes = (size_t)n * N * 16;
  const size_t smem_max = ctx->prop.sharedMemPerBlockOptin;
  const bool c_smem = base + cbytes <= smem_max;
  const size_t smem = c_smem ? base + cbytes : base;
  FS_REQUIRE(smem <= smem_max, FS_ERR_UNSUPPORTED, "norb too large for the Slater sampler");
  const int sms = ctx->prop.multiProcessorCount;
  int64_t grid = std::min<int64_t>(shots, c_smem ? (int64_t)sms * 32 : (int64_t)sms * 2);
  if (!c_smem)  // global coefficient slots: at most 4 GiB of them
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, ((int64_t)4 << 30) / (int64_t)cbytes));
  grid = std::max<int64_t>(grid, 1);
  char* ws = (char*)scratch(ctx, "slater",
                            kbytes + pbytes + (c_smem ? 0 : (size_t)grid * cbytes));
  double2* K = (double2*)ws;
  double2* P = (double2*)(ws + kbytes);
  double2* Cg = c_smem ? nullptr : (double2*)(ws + kbytes + pbytes);
  if (pbytes) FS_CUDA(cudaMemcpyAsync(P, Phi.data(), pbytes, cudaMemcpyHostToDevice, st));
  {
    ProfScope ps("slater_projector", st);
    const int64_t nn = (int64_t)N * N;
    k_projector<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(K, P, N, n);
  }
  FS_CUDA(cudaFuncSetAttribute(k_sample_slater, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  ProfScope ps("slater_sample", st);
  k_sample_slater<<<(unsigned)grid, B, smem, st>>>(K, N, n, u, shots, out, words, Cg,
                                                   c_smem ? 1 : 0);
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
