// Interleaved complex helpers (double2 / float2) for the device code.
#pragma once
#include <cuda_runtime.h>

namespace bf {

template <typename R>
struct Cx;

template <>
struct Cx<double> {
  using V = double2;
  __host__ __device__ static inline V make(double x, double y) { return make_double2(x, y); }
};
template <>
struct Cx<float> {
  using V = float2;
  __host__ __device__ static inline V make(float x, float y) { return make_float2(x, y); }
};

// acc += a * b
template <typename V>
__device__ __forceinline__ void cmac(V& acc, const V a, const V b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename V>
__device__ __forceinline__ void cmac_conj(V& acc, const V a, const V b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 to_d2(const double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(const float2 v) { return make_double2(v.x, v.y); }

template <typename V>
__device__ __forceinline__ V from_d2(const double2 v);
template <>
__device__ __forceinline__ double2 from_d2<double2>(const double2 v) { return v; }
template <>
__device__ __forceinline__ float2 from_d2<float2>(const double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

}  // namespace bf
