// Device helpers shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace prd {

// Weideman expansion coefficients of the Faddeeva function (host-computed at
// prd_create, uploaded to constant memory of each translation unit that
// evaluates W): a_k, k = 1..N, and the scale L.
struct WeidemanConst {
  double a64[36];
  float a32[20];
  double L64;
  float L32;
};

template <typename T> struct Cx { T re, im; };

template <typename T> __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// w(x + i y), y >= 0, from Weideman's rational expansion in Z = (L+iz)/(L-iz):
//   w = 2 p(Z)/(L - i z)^2 + 1/(sqrt(pi)(L - i z)),  p(Z) = sum_k a_k Z^(k-1).
template <typename T> __device__ __forceinline__ Cx<T> faddeeva(T x, T y, const WeidemanConst& wc);

template <> __device__ __forceinline__ Cx<double> faddeeva<double>(double x, double y, const WeidemanConst& wc) {
  const double L = wc.L64;
  // L - i z = (L + y) - i x ;  L + i z = (L - y) + i x
  const double dr = L + y, di = -x;
  const double nr = L - y, ni = x;
  const double inv = 1.0 / (dr * dr + di * di);
  const double Zr = (nr * dr + ni * di) * inv, Zi = (ni * dr - nr * di) * inv;
  double pr = wc.a64[35], pi = 0.0;
#pragma unroll
  for (int k = 34; k >= 0; --k) {
    const double t = pr * Zr - pi * Zi + wc.a64[k];
    pi = pr * Zi + pi * Zr;
    pr = t;
  }
  // 1/d and 1/d^2
  const double ir = dr * inv, ii = -di * inv;           // 1/d
  const double i2r = ir * ir - ii * ii, i2i = 2.0 * ir * ii;
  const double s = 0.56418958354775628695;              // 1/sqrt(pi)
  return {2.0 * (pr * i2r - pi * i2i) + s * ir, 2.0 * (pr * i2i + pi * i2r) + s * ii};
}

template <> __device__ __forceinline__ Cx<float> faddeeva<float>(float x, float y, const WeidemanConst& wc) {
  const float L = wc.L32;
  const float dr = L + y, di = -x;
  const float nr = L - y, ni = x;
  const float inv = 1.0f / (dr * dr + di * di);
  const float Zr = (nr * dr + ni * di) * inv, Zi = (ni * dr - nr * di) * inv;
  float pr = wc.a32[19], pi = 0.0f;
#pragma unroll
  for (int k = 18; k >= 0; --k) {
    const float t = pr * Zr - pi * Zi + wc.a32[k];
    pi = pr * Zi + pi * Zr;
    pr = t;
  }
  const float ir = dr * inv, ii = -di * inv;
  const float i2r = ir * ir - ii * ii, i2i = 2.0f * ir * ii;
  const float s = 0.564189583547756f;
  return {2.0f * (pr * i2r - pi * i2i) + s * ir, 2.0f * (pr * i2i + pi * i2r) + s * ii};
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace prd
