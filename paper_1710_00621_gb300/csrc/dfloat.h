// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32 numbers
// (about 48 significand bits), computed on the FP32 pipe with the error-free
// transformations of Dekker and Knuth (TwoSum, FastTwoSum, and the exact product
// a b = p + e with p = fl(a b), e = fma(a, b, -p)).  Sums and products are the
// "sloppy" double-float forms (relative error a few times 2^-48), enough for the
// FP64-accurate transforms of CMBWS_FP32X2.  Conversions from and to double run on
// the FP64 pipe and are kept out of inner loops.
#pragma once

#include <cuda_runtime.h>

namespace cmbws {

struct df {
  float h, l;
  df() = default;
  __host__ __device__ constexpr df(float h_, float l_) : h(h_), l(l_) {}
  __device__ df(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
  __device__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_from(double v) { return df(v); }
__device__ __forceinline__ double df_to(df a) { return (double)a; }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return quick_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ df df_sub(df a, df b) {
  const df s = two_sum(a.h, -b.h);
  return quick_two_sum(s.h, s.l + (a.l - b.l));
}
// a * b - c
__device__ __forceinline__ df df_fms(df a, df b, df c) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const df s = two_sum(p, -c.h);
  return quick_two_sum(s.h, s.l + (e - c.l));
}
// compensated accumulation acc_h + acc_l += a * b (Dot2 of Ogita, Rump and Oishi 2005)
__device__ __forceinline__ void dot2_acc(float& acc_h, float& acc_l, df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const df s = two_sum(acc_h, p);
  acc_h = s.h;
  acc_l += s.l + e;
}
// the rescaled Legendre recurrence step (A - A y) m1 - m2
__device__ __forceinline__ df df_recur(df A, df y, df m1, df m2) {
  const df ax = df_sub(A, df_mul(A, y));
  return df_fms(ax, m1, m2);
}

__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a, df b) { return df_sub(a, b); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df operator-(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = df_add(a, b); }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = df_sub(a, b); }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = df_mul(a, b); }

// complex double-float (16 bytes, the size of double2)
struct __align__(16) df2 {
  df x, y;
};

}  // namespace cmbws
