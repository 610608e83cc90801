// wf_common.cuh -- arithmetic types, complex helpers and reductions shared by the kernels.
//
// Three real types carry the spectral arithmetic:
//   double  FP64 (1/64-rate units on GB300: used where FP64 storage meets FP64 arithmetic)
//   float   FP32 (the inner solves of the mixed-precision path)
//   df32    a double-float pair (hi + lo, |lo| <= ulp(hi)/2, ~48-bit significand) evaluated on
//           the FP32 units with error-free transforms (Knuth two-sum, FMA two-product, as in
//           Dekker 1971 / the "double-double" literature); used to transform FP64-stored fields
//           at FP32-unit throughput.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define WF_HD __host__ __device__ __forceinline__
#define WF_D __device__ __forceinline__

// ------------------------------------------------------------------------------------------
// double-float
// ------------------------------------------------------------------------------------------
struct df32 {
  float hi, lo;
};

WF_D df32 df_make(float h, float l) { return df32{h, l}; }

// s + e = a + b exactly (Knuth two-sum, no magnitude assumption)
WF_D void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker fast two-sum)
WF_D void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// accurate double-float sum (relative error ~2^-46 even under cancellation)
WF_D df32 operator+(df32 a, df32 b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return df32{s, e};
}
WF_D df32 operator-(df32 a) { return df32{-a.hi, -a.lo}; }
WF_D df32 operator-(df32 a, df32 b) { return a + (-b); }
WF_D df32 operator*(df32 a, df32 b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);          // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return df32{s, t};
}
WF_D df32& operator+=(df32& a, df32 b) { return a = a + b; }
WF_D df32& operator-=(df32& a, df32 b) { return a = a - b; }
WF_D df32& operator*=(df32& a, df32 b) { return a = a * b; }

// FP64 <-> df32 (hi = nearest float, lo = nearest float of the remainder)
WF_D df32 df_from_double(double v) {
  float h = __double2float_rn(v);
  float l = __double2float_rn(v - (double)h);
  return df32{h, l};
}
WF_D double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

// Ask L2 to fetch [p, p + bytes) from HBM ahead of its use (a bulk prefetch: no registers or
// shared memory held, no completion to wait for).  p and bytes must be multiples of 16.
WF_D void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ------------------------------------------------------------------------------------------
// real-type traits: constants and conversion to/from the FP64 / FP32 storage types
// ------------------------------------------------------------------------------------------
template <class R> struct RT;
template <> struct RT<double> {
  WF_HD static double c(double v) { return v; }
  WF_D static double from_d(double v) { return v; }
  WF_D static double to_d(double v) { return v; }
  WF_D static double from_f(float v) { return (double)v; }
  WF_D static float to_f(double v) { return (float)v; }
  WF_D static double mul(double a, double b) { return a * b; }
};
template <> struct RT<float> {
  WF_HD static float c(double v) { return (float)v; }
  WF_D static float from_d(double v) { return __double2float_rn(v); }
  WF_D static double to_d(float v) { return (double)v; }
  WF_D static float from_f(float v) { return v; }
  WF_D static float to_f(float v) { return v; }
};
template <> struct RT<df32> {
  WF_D static df32 c(double v) { return df_from_double(v); }
  WF_D static df32 from_d(double v) { return df_from_double(v); }
  WF_D static double to_d(df32 v) { return df_to_double(v); }
  WF_D static df32 from_f(float v) { return df32{v, 0.f}; }
  WF_D static float to_f(df32 v) { return v.hi + v.lo; }
};

// ------------------------------------------------------------------------------------------
// complex over a real type
// ------------------------------------------------------------------------------------------
template <class R> struct __align__(2 * sizeof(R)) cx {
  R x, y;
};
template <class R> WF_D cx<R> mkc(R a, R b) { return cx<R>{a, b}; }
template <class R> WF_D cx<R> operator+(cx<R> a, cx<R> b) { return cx<R>{a.x + b.x, a.y + b.y}; }
template <class R> WF_D cx<R> operator-(cx<R> a, cx<R> b) { return cx<R>{a.x - b.x, a.y - b.y}; }
template <class R> WF_D cx<R> operator*(cx<R> a, cx<R> b) {
  return cx<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R> WF_D cx<R> scale(cx<R> a, R s) { return cx<R>{a.x * s, a.y * s}; }
template <class R> WF_D cx<R> conj(cx<R> a) { return cx<R>{a.x, -a.y}; }
template <class R> WF_D cx<R> mul_i(cx<R> a) { return cx<R>{-a.y, a.x}; }      // a * i
template <class R> WF_D cx<R> mul_mi(cx<R> a) { return cx<R>{a.y, -a.x}; }     // a * (-i)
// a * i * sign (sign = +1 or -1 at compile time)
template <int SIGN, class R> WF_D cx<R> mul_si(cx<R> a) {
  return SIGN > 0 ? mul_i(a) : mul_mi(a);
}

// loads/stores between FP64 / FP32 storage and the arithmetic type
template <class R> WF_D cx<R> ld_c(const double2* p) {
  double2 v = *p;
  return cx<R>{RT<R>::from_d(v.x), RT<R>::from_d(v.y)};
}
template <class R> WF_D cx<R> ld_c(const float2* p) {
  float2 v = *p;
  return cx<R>{RT<R>::from_f(v.x), RT<R>::from_f(v.y)};
}
template <class R> WF_D void st_c(double2* p, cx<R> v) { *p = make_double2(RT<R>::to_d(v.x), RT<R>::to_d(v.y)); }
template <class R> WF_D void st_c(float2* p, cx<R> v) { *p = make_float2(RT<R>::to_f(v.x), RT<R>::to_f(v.y)); }

// storage complex type for an arithmetic type: FP64 storage for double and df32, FP32 for float
template <class R> struct Store { using T = double2; using S = double; };
template <> struct Store<float> { using T = float2; using S = float; };

// ------------------------------------------------------------------------------------------
// dot-product accumulation.  For FP32 data the products are formed exactly (two-product) and
// accumulated in double-float; for FP64 data in FP64.  Either way the per-thread partial is
// returned as a double and the cross-thread sums are FP64.  Sums whose terms are all >= 0 (norms,
// <p, m p>, sum D T^2) add a 16-byte vector's few terms in the storage type first and pass that
// partial to add(): no cancellation, so the relative error stays a few units of FP32 rounding.
// ------------------------------------------------------------------------------------------
struct AccD {
  double s = 0.0;
  WF_D void add_prod(double a, double b) { s = fma(a, b, s); }
  WF_D void add(double a) { s += a; }
  WF_D double get() const { return s; }
};
struct AccF {
  float hi = 0.f, lo = 0.f;
  WF_D void add_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    float s, t;
    two_sum(hi, p, s, t);
    lo = __fadd_rn(lo, __fadd_rn(t, e));
    hi = s;
  }
  WF_D void add(float a) {
    float s, t;
    two_sum(hi, a, s, t);
    lo = __fadd_rn(lo, t);
    hi = s;
  }
  WF_D double get() const { return (double)hi + (double)lo; }
};
template <class S> struct AccFor { using T = AccD; };
template <> struct AccFor<float> { using T = AccF; };

// Block-wide sum of a double; result valid in thread 0.  `red` holds >= 32 doubles.
WF_D double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
