// Complex helpers shared by the FP64 (double2), FP32 (float2) and double-float (df64c) kernels.
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
// acc + a b
template <class C>
__device__ __forceinline__ C cmac(C a, C b, C acc) {
  return mkc(fmar(a.x, b.x, fmar(-a.y, b.y, acc.x)), fmar(a.x, b.y, fmar(a.y, b.x, acc.y)));
}

// Double-float numbers (a value as the unevaluated sum h + l of two floats, |l| <= ulp(h)/2)
// for the transform stages of DF64 plans: about 48 significant bits from FP32 arithmetic,
// which runs 64 times faster than FP64 on this GPU. The building blocks are the error-free
// transformations of Knuth (two-sum) and Dekker (fast two-sum for |a| >= |b|) and the FMA form
// of the exact product; addition is the "sloppy" double-float sum (error bounded relative to
// |a| + |b|, the bound the FFT's normwise error analysis needs).
struct df64 {
  float h, l;
  df64() = default;
  __host__ __device__ constexpr df64(float hh, float ll) : h(hh), l(ll) {}
  __host__ __device__ df64(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  return fast_two_sum(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.h, -a.l); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
// a b + c with one rounding step less than the product followed by the sum
__device__ __forceinline__ df64 fmar(df64 a, df64 b, df64 c) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  const float s = p + c.h;
  const float bb = s - p;
  e += (p - (s - bb)) + (c.h - bb);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  e += c.l;
  return fast_two_sum(s, e);
}

struct __align__(16) df64c {
  df64 x, y;
};
template <>
struct RealOf<df64c> {
  typedef df64 type;
};
__device__ __forceinline__ df64c mkc(df64 x, df64 y) {
  df64c r;
  r.x = x;
  r.y = y;
  return r;
}

// Read-only loads of the complex types.
__device__ __forceinline__ double2 ldgc(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldgc(const float2* p) { return __ldg(p); }
__device__ __forceinline__ df64c ldgc(const df64c* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return mkc(df64(v.x, v.y), df64(v.z, v.w));
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
template <>
__device__ __forceinline__ df64c from_d2<df64c>(double2 v) {
  return mkc(df64(v.x), df64(v.y));
}

}  // namespace hk
