// Small vector and compensated-arithmetic helpers for the device code.
#pragma once

#include <cuda_runtime.h>

namespace dem {

template <typename T>
struct V3 {
  T x, y, z;
};

template <typename T>
__host__ __device__ __forceinline__ V3<T> mk(T x, T y, T z) {
  return V3<T>{x, y, z};
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) {
  return mk(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) {
  return mk(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> operator-(V3<T> a) {
  return mk(-a.x, -a.y, -a.z);
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> operator*(T s, V3<T> a) {
  return mk(s * a.x, s * a.y, s * a.z);
}
template <typename T>
__host__ __device__ __forceinline__ T dot(V3<T> a, V3<T> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ double vsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }

template <typename T>
__device__ __forceinline__ T vnorm(V3<T> a) {
  return vsqrt(dot(a, a));
}

// ---- error-free transformations (Knuth TwoSum, FMA-based TwoProduct) -------
// They let FP32 hardware carry ~48 significant bits where the DEM state needs
// them; see e.g. Ogita, Rump & Oishi, "Accurate sum and dot product" (2005).

struct ff {  // unevaluated sum hi + lo, |lo| <= ulp(hi)/2 after normalisation
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return ff{s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return ff{s, e};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = a * b;
  float e = __fmaf_rn(a, b, -p);
  return ff{p, e};
}
// (hi, lo) + b
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  s.lo += a.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

// Kahan's compensated summation (Kahan 1965), the compensation kept as a
// correction term: sum = h + l.  The rounding error of each addition is
// carried into the next one; the order of the additions is fixed.
__device__ __forceinline__ void kahan(float& h, float& l, float b) {
  const float y = b + l;
  const float t = h + y;
  l = y - (t - h);
  h = t;
}

// Compensated accumulator of a 3-vector (order fixed by the caller).
struct Acc3 {
  float hx, hy, hz, lx, ly, lz;
  __device__ __forceinline__ void zero() { hx = hy = hz = lx = ly = lz = 0.f; }
  __device__ __forceinline__ void add(V3<float> v) {
    kahan(hx, lx, v.x);
    kahan(hy, ly, v.y);
    kahan(hz, lz, v.z);
  }
};

}  // namespace dem
