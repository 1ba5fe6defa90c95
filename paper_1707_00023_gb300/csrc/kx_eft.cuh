// Compensated FP32 Gram-Schmidt update.
//
// The Arnoldi update x <- x - sum_i c_i v_i in FP32 rounds x once per
// column; with FP32 basis storage that accumulated rounding is the largest
// error of the FP32 path (measured in an FP32 emulation of restart in
// Krylov dimension at T = 400: the error falls about threefold when the
// update alone is carried in higher precision, and changes by less than 10 %
// when the dots, the stencil or a second orthogonalisation pass are).  Here
// x is carried as an unevaluated pair hi + lo.  Each column's step
// s = fl(hi + nc v) is one FMA; its rounding error is hi + nc v - s =
// fma(nc, v, hi - s), where hi - s is exact whenever s lies within a factor
// 2 of hi (Sterbenz's lemma), and the error collects in lo.  A step that
// changes x by more than that (a large coefficient against a small entry)
// keeps an error of the order of one FP32 rounding of that step.  Rounding
// hi + lo once when the column is stored gives the update close to FP32
// storage precision, at four FP32 operations a column instead of one.
#pragma once

namespace kx {

// hi + lo <- hi + lo + nc v
__device__ __forceinline__ void sub_fma(float& hi, float& lo, float nc, float v) {
  const float s = fmaf(nc, v, hi);
  lo += fmaf(nc, v, hi - s);
  hi = s;
}

// The same on two lanes at a time in packed FP32x2 operations (a - b as
// fma(b, -1, a), exact before its one rounding).
__device__ __forceinline__ void sub_fma2(float2& hi, float2& lo, float2 nc, float2 v) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 s = __ffma2_rn(nc, v, hi);     // fl(hi + nc v)
  const float2 d = __ffma2_rn(s, m1, hi);     // hi - s, exact when s is within a factor 2 of hi
  lo = __fadd2_rn(lo, __ffma2_rn(nc, v, d));  // + the rounding error of s
  hi = s;
}

__device__ __forceinline__ void sub_fma4(float4& hi, float4& lo, float nc, const float4& v) {
  const float2 n2 = make_float2(nc, nc);
  float2 h0 = make_float2(hi.x, hi.y), h1 = make_float2(hi.z, hi.w);
  float2 l0 = make_float2(lo.x, lo.y), l1 = make_float2(lo.z, lo.w);
  sub_fma2(h0, l0, n2, make_float2(v.x, v.y));
  sub_fma2(h1, l1, n2, make_float2(v.z, v.w));
  hi = make_float4(h0.x, h0.y, h1.x, h1.y);
  lo = make_float4(l0.x, l0.y, l1.x, l1.y);
}

}  // namespace kx
