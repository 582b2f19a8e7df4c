// Device-side helpers shared by the fsgpu kernels: complex arithmetic on
// float2/double2, binomials, and error checking.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace fs {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <typename R> using cx_t = typename Cx<R>::T;

template <typename R>
__host__ __device__ __forceinline__ cx_t<R> mk(R re, R im) {
  cx_t<R> z;
  z.x = re;
  z.y = im;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ cx_t<R> cmul(cx_t<R> a, cx_t<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cx_t<R> cmulc(cx_t<R> a, cx_t<R> b) {
  return mk<R>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// One Givens update on the pair (x, y), x the amplitude of I (p occupied,
// q empty) and y that of I' = I^{p->q}, for G = [[c, s], [-s*, c]]:
//   x' = c x + s y,   y' = -s* x + c y.
template <typename R>
__device__ __forceinline__ void givens2(cx_t<R>& x, cx_t<R>& y, R c, R sr, R si) {
  cx_t<R> xn, yn;
  xn.x = fma(c, x.x, fma(sr, y.x, -si * y.y));
  xn.y = fma(c, x.y, fma(sr, y.y, si * y.x));
  yn.x = fma(c, y.x, -fma(sr, x.x, si * x.y));
  yn.y = fma(c, y.y, fma(si, x.x, -sr * x.y));
  x = xn;
  y = yn;
}

// Binomial coefficient C(n, k) (0 outside 0 <= k <= n).

__host__ __device__ inline uint64_t binom_host(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

}  // namespace fs
