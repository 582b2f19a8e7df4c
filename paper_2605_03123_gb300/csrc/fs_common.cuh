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

// exp(i x) for an FP64 angle: reduced to [-pi, pi] in FP64, then evaluated
// in the precision of the state.
template <typename R>
__device__ __forceinline__ cx_t<R> expi(double x);
template <>
__device__ __forceinline__ cx_t<float> expi<float>(double x) {
  double r = x - 6.283185307179586 * rint(x * 0.15915494309189535);
  float s, c;
  sincosf((float)r, &s, &c);
  return mk<float>(c, s);
}
template <>
__device__ __forceinline__ cx_t<double> expi<double>(double x) {
  double r = x - 6.283185307179586 * rint(x * 0.15915494309189535);
  double s, c;
  sincos(r, &s, &c);
  return mk<double>(c, s);
}

// det(R[rows of mask, columns 0 .. n-1]) for an N x N complex matrix R
// (row-major, interleaved re/im), by Gaussian elimination with partial
// pivoting in FP64: the amplitude of string `mask` in the Slater
// determinant of the first n columns of R.
__device__ inline double2 slater_minor(uint32_t mask, int norb, int n, const double* Rv) {
  double2 a[32 * 32];
  int r = 0;
  for (int p = 0; p < norb; ++p)
    if ((mask >> p) & 1u) {
      for (int c = 0; c < n; ++c)
        a[r * n + c] = make_double2(Rv[2 * (p * norb + c)], Rv[2 * (p * norb + c) + 1]);
      ++r;
    }
  double dr = 1, di = 0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = hypot(a[k * n + k].x, a[k * n + k].y);
    for (int i = k + 1; i < n; ++i) {
      const double h = hypot(a[i * n + k].x, a[i * n + k].y);
      if (h > best) {
        best = h;
        piv = i;
      }
    }
    if (best == 0) return make_double2(0, 0);
    if (piv != k) {
      for (int c = 0; c < n; ++c) {
        const double2 t = a[k * n + c];
        a[k * n + c] = a[piv * n + c];
        a[piv * n + c] = t;
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
  return make_double2(dr, di);
}

// Binomial coefficient C(n, k) (0 outside 0 <= k <= n).

__host__ __device__ inline uint64_t binom_host(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

}  // namespace fs
