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

__device__ __forceinline__ void sub_fma4(float4& hi, float4& lo, float nc, const float4& v) {
  sub_fma(hi.x, lo.x, nc, v.x);
  sub_fma(hi.y, lo.y, nc, v.y);
  sub_fma(hi.z, lo.z, nc, v.z);
  sub_fma(hi.w, lo.w, nc, v.w);
}

}  // namespace kx
