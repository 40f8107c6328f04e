// Complex helpers shared by the FP64 (double2) and FP32 (float2) kernels.
#pragma once
#include <cuda_runtime.h>

namespace hk {

template <class C>
struct RealOf;
template <>
struct RealOf<double2> {
  typedef double type;
};
template <>
struct RealOf<float2> {
  typedef float type;
};

__device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }

template <class C>
__device__ __forceinline__ C cmul(C a, C b) {
  return mkc(fmar(a.x, b.x, -a.y * b.y), fmar(a.x, b.y, a.y * b.x));
}

// Round a double2 to the kernel's complex type.
template <class C>
__device__ __forceinline__ C from_d2(double2 v);
template <>
__device__ __forceinline__ double2 from_d2<double2>(double2 v) {
  return v;
}
template <>
__device__ __forceinline__ float2 from_d2<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

}  // namespace hk
