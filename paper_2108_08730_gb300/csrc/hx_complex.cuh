// Small complex helpers on float2 / double2 (interleaved re, im).
#pragma once

#include <cuda_runtime.h>

namespace hx {

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };

__device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }
template <class C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return cmk(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return cmk(a.x - b.x, a.y - b.y); }
template <class C, class T> __device__ __forceinline__ C cscale(T s, C a) { return cmk(s * a.x, s * a.y); }
// acc + s * a   (s real)
template <class C, class T> __device__ __forceinline__ C cfmar(T s, C a, C acc) {
  return cmk(fma(s, a.x, acc.x), fma(s, a.y, acc.y));
}
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a * b
template <class C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  return cmk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// i * s * a  (s real)
template <class C, class T> __device__ __forceinline__ C cscale_i(T s, C a) { return cmk(-s * a.y, s * a.x); }
template <class C> __device__ __forceinline__ C crcp(C a) {
  auto d = a.x * a.x + a.y * a.y;
  return cmk(a.x / d, -a.y / d);
}

}  // namespace hx
