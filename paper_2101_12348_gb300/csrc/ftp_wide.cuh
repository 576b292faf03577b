// "Wide" arithmetic for the FP64-class steps of the roots kernel (assembly of
// MM', YM', Mbar and the Newton polish of the chosen phase).
//
// Two representations share one interface:
//   double / double2  - native FP64 (the FP64 path and the re-solve pass);
//   dd / ddc          - a float-float ("double-single") number hi + lo with
//                       |lo| <= ulp(hi)/2, about 48 significand bits, built
//                       from the error-free transformations TwoSum (Knuth)
//                       and TwoProduct via a fused multiply-add (Dekker's
//                       product with FMA).  It runs on the FP32 pipe, which
//                       on this GPU issues a warp instruction ~100x cheaper
//                       than the FP64 pipe.
// The transformations use __fadd_rn/__fsub_rn/__fmul_rn so the compiler can
// neither contract them into FMAs nor reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace ftp {
namespace wide {

struct dd {
  float hi, lo;
};
struct ddc {
  dd x, y;
};

// ---------------------------------------------------------- float-float core
__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return {s, e};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// multiply by a float (exact integers such as harmonic numbers included)
__device__ __forceinline__ dd dd_mulf(dd a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}
// Quotient q1 + q2 with q2 from the exact remainder a - b q1 (Dekker).  The
// two float quotients may be approximate (a few ulp): the remainder absorbs
// q1's error, and q2's error is ulp-level of a term ~2^-22 |q|, so the
// result keeps ~44 bits.
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  const float q1 = __fdividef(a.hi, b.hi);
  const dd r = dd_sub(a, dd_mulf(b, q1));
  const float q2 = __fdividef(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ dd dd_from_double(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------- generic interface
// W: real type, WC: complex type.
__device__ __forceinline__ double w_add(double a, double b) { return a + b; }
__device__ __forceinline__ dd w_add(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ double w_sub(double a, double b) { return a - b; }
__device__ __forceinline__ dd w_sub(dd a, dd b) { return dd_sub(a, b); }
__device__ __forceinline__ double w_mul(double a, double b) { return a * b; }
__device__ __forceinline__ dd w_mul(dd a, dd b) { return dd_mul(a, b); }
__device__ __forceinline__ double w_mulf(double a, float b) { return a * (double)b; }
__device__ __forceinline__ dd w_mulf(dd a, float b) { return dd_mulf(a, b); }
__device__ __forceinline__ double w_div(double a, double b) { return a / b; }
__device__ __forceinline__ dd w_div(dd a, dd b) { return dd_div(a, b); }
__device__ __forceinline__ float w_f(double a) { return (float)a; }
__device__ __forceinline__ float w_f(dd a) { return a.hi; }
__device__ __forceinline__ double w_d(double a) { return a; }
__device__ __forceinline__ double w_d(dd a) { return dd_to_double(a); }
template <typename W> __device__ __forceinline__ W w_zero();
template <> __device__ __forceinline__ double w_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ dd w_zero<dd>() { return {0.f, 0.f}; }
template <typename W> __device__ __forceinline__ W w_of(double v);
template <> __device__ __forceinline__ double w_of<double>(double v) { return v; }
template <> __device__ __forceinline__ dd w_of<dd>(double v) { return dd_from_double(v); }
template <typename W> __device__ __forceinline__ W w_off(float v);
template <> __device__ __forceinline__ double w_off<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ dd w_off<dd>(float v) { return {v, 0.f}; }

template <typename W> struct CT;
template <> struct CT<double> { using type = double2; };
template <> struct CT<dd> { using type = ddc; };

__device__ __forceinline__ double re(double2 a) { return a.x; }
__device__ __forceinline__ double im(double2 a) { return a.y; }
__device__ __forceinline__ dd re(ddc a) { return a.x; }
__device__ __forceinline__ dd im(ddc a) { return a.y; }
__device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ ddc mkc(dd x, dd y) { return {x, y}; }

template <typename W>
__device__ __forceinline__ typename CT<W>::type c_add(typename CT<W>::type a,
                                                      typename CT<W>::type b) {
  return mkc(w_add(re(a), re(b)), w_add(im(a), im(b)));
}
template <typename W>
__device__ __forceinline__ typename CT<W>::type c_sub(typename CT<W>::type a,
                                                      typename CT<W>::type b) {
  return mkc(w_sub(re(a), re(b)), w_sub(im(a), im(b)));
}
template <typename W>
__device__ __forceinline__ typename CT<W>::type c_mul(typename CT<W>::type a,
                                                      typename CT<W>::type b) {
  return mkc(w_sub(w_mul(re(a), re(b)), w_mul(im(a), im(b))),
             w_add(w_mul(re(a), im(b)), w_mul(im(a), re(b))));
}
__device__ __forceinline__ double w_neg(double a) { return -a; }
__device__ __forceinline__ dd w_neg(dd a) { return dd_neg(a); }
template <typename W>
__device__ __forceinline__ typename CT<W>::type c_conj(typename CT<W>::type a) {
  return mkc(re(a), w_neg(im(a)));
}
template <typename W>
__device__ __forceinline__ typename CT<W>::type c_mulf(typename CT<W>::type a, float k) {
  return mkc(w_mulf(re(a), k), w_mulf(im(a), k));
}
template <typename W>
__device__ __forceinline__ W c_abs2(typename CT<W>::type a) {
  return w_add(w_mul(re(a), re(a)), w_mul(im(a), im(a)));
}
template <typename W> __device__ __forceinline__ typename CT<W>::type c_zero() {
  return mkc(w_zero<W>(), w_zero<W>());
}

// ---------------------------------------------------------- shuffles
__device__ __forceinline__ double w_shfl_xor(double v, int o, int width) {
  return __shfl_xor_sync(0xffffffffu, v, o, width);
}
__device__ __forceinline__ dd w_shfl_xor(dd v, int o, int width) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o, width),
          __shfl_xor_sync(0xffffffffu, v.lo, o, width)};
}
__device__ __forceinline__ double w_shfl_up(double v, int o, int width) {
  return __shfl_up_sync(0xffffffffu, v, o, width);
}
__device__ __forceinline__ dd w_shfl_up(dd v, int o, int width) {
  return {__shfl_up_sync(0xffffffffu, v.hi, o, width),
          __shfl_up_sync(0xffffffffu, v.lo, o, width)};
}
__device__ __forceinline__ double w_shfl(double v, int src, int width) {
  return __shfl_sync(0xffffffffu, v, src, width);
}
__device__ __forceinline__ dd w_shfl(dd v, int src, int width) {
  return {__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width)};
}

}  // namespace wide
}  // namespace ftp
