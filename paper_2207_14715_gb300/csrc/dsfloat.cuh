// Float-float ("double-single") arithmetic for the mixed form.
//
// A value is represented as hi + lo with |lo| <= ulp(hi)/2 (about 48 significant bits),
// built from the error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and
// TwoProduct through a fused multiply-add (Dekker 1971).  The mixed-form evaluation uses it
// for the values of the basis functions and of the determinant orbitals, which set ln|Psi|:
// on this part the FP64 pipe is ~64x slower than FP32, so double-precision accuracy is
// obtained from float instructions.
#pragma once

#include <cuda_runtime.h>

namespace vbq {

struct dsf {
  float hi, lo;
};

__device__ __forceinline__ dsf ds_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ dsf ds_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ dsf ds_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
// accurate sum (both parts through TwoSum): safe under cancellation
__device__ __forceinline__ dsf ds_add(dsf a, dsf b) {
  dsf s = ds_two_sum(a.hi, b.hi);
  const dsf t = ds_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = ds_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return ds_fast_two_sum(s.hi, s.lo);
}
// sum without the low-part TwoSum: enough when the operands do not cancel
__device__ __forceinline__ dsf ds_add_nc(dsf a, dsf b) {
  dsf s = ds_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return ds_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dsf ds_mul(dsf a, dsf b) {
  dsf p = ds_two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return ds_fast_two_sum(p.hi, p.lo);
}
// a + b for a float b (cancellation-safe)
__device__ __forceinline__ dsf ds_add_f(dsf a, float b) {
  dsf s = ds_two_sum(a.hi, b);
  s.lo += a.lo;
  return ds_fast_two_sum(s.hi, s.lo);
}
// a - b rounded to float (within one rounding of the exact difference): the difference of the
// high parts is exact through TwoSum, the low parts only add a small correction.
__device__ __forceinline__ float ds_diff_f(dsf a, dsf b) {
  const dsf d = ds_two_sum(a.hi, -b.hi);
  return d.hi + (d.lo + (a.lo - b.lo));
}
__device__ __forceinline__ dsf ds_neg(dsf a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dsf ds_sub(dsf a, dsf b) { return ds_add(a, ds_neg(b)); }
// 1/a: float reciprocal y0 of a.hi, then one Newton step y0 + y0 (1 - a y0) with the residual
// 1 - a y0 formed in float-float (its error is second order in the float error of y0).
__device__ __forceinline__ dsf ds_recip(dsf a) {
  const float y0 = 1.0f / a.hi;
  const dsf e = ds_add_f(ds_neg(ds_mul(a, dsf{y0, 0.0f})), 1.0f);
  return ds_add_f(ds_two_prod(y0, e.hi), y0);
}
// a/b: float quotient q0 = a.hi/b.hi, then one correction (a - b q0)/b.hi
__device__ __forceinline__ dsf ds_div(dsf a, dsf b) {
  const float q0 = a.hi / b.hi;
  const dsf r = ds_sub(a, ds_mul(b, dsf{q0, 0.0f}));
  return ds_add_f(dsf{r.hi / b.hi, 0.0f}, q0);
}
// sqrt(a), a >= 0: s0 = sqrt(a.hi) in float, then s0 + (a - s0^2)/(2 s0) (Newton's step on
// s^2 = a, residual exact through TwoProduct).
__device__ __forceinline__ dsf ds_sqrt(dsf a) {
  if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
  const float s0 = sqrtf(a.hi);
  const dsf r = ds_sub(a, ds_two_prod(s0, s0));
  return ds_add_f(dsf{r.hi / (2.0f * s0), 0.0f}, s0);
}
__device__ __forceinline__ dsf ds_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double ds_to_double(dsf a) { return (double)a.hi + (double)a.lo; }

// exp(-x) for x >= 0 given in float-float, relative error ~1e-14.
// Reduction (Cody and Waite): n = round(x / ln 2), r = x - n ln 2 with ln 2 split into three
// floats L1 + L2 + L3 (L1 has 15 significant bits, so n L1 and x_hi - n L1 are exact for the
// n that occur); then exp(-x) = 2^-n exp(-r), |r| <= ln2/2, with the Taylor series of exp(-r)
// to degree 13 (truncation < 2e-16) evaluated by Horner's rule in float-float.  Results below
// 2^-126 are flushed to zero.
__device__ __forceinline__ dsf ds_exp_neg(dsf x) {
  if (!(x.hi < 87.0f)) return {0.0f, 0.0f};
  const float L1 = 0x1.62e4p-1f, L2 = 0x1.7f7d1cp-20f, L3 = 0x1.ef357ap-45f;
  const float n = rintf(x.hi * 1.44269504089f);
  const float t1 = fmaf(-n, L1, x.hi);
  const dsf p2 = ds_two_prod(n, L2);
  dsf r = ds_two_sum(t1, -p2.hi);
  r.lo += (x.lo - p2.lo) - n * L3;
  r = ds_fast_two_sum(r.hi, r.lo);
  const dsf mr = {-r.hi, -r.lo};
  // 1/k!, k = 13..0, as float pairs
  const float chi[14] = {0x1.612462p-33f, 0x1.1eed8ep-29f, 0x1.ae6456p-26f, 0x1.27e4fcp-22f, 0x1.71de3ap-19f,
                         0x1.a01a02p-16f, 0x1.a01a02p-13f, 0x1.6c16c2p-10f, 0x1.111112p-7f,  0x1.555556p-5f,
                         0x1.555556p-3f, 0x1.0p-1f,       0x1.0p+0f,       0x1.0p+0f};
  const float clo[14] = {-0x1.8af25ep-58f, 0x1.ff1b12p-54f, 0x1.fd5138p-52f, -0x1.10ec14p-47f, 0x1.55b1ccp-45f,
                         -0x1.7f97fap-42f, -0x1.7f97fap-39f, -0x1.27d27ep-35f, -0x1.dddddep-32f, -0x1.555556p-30f,
                         -0x1.555556p-28f, 0.0f,            0.0f,            0.0f};
  dsf p = {chi[0], clo[0]};
#pragma unroll
  for (int k = 1; k < 14; ++k) p = ds_add_nc(ds_mul(p, mr), dsf{chi[k], clo[k]});
  const int ni = (int)n;
  const float scale = __int_as_float((127 - ni) << 23);  // 2^-n, exact for 0 <= n <= 126
  return {p.hi * scale, p.lo * scale};
}

}  // namespace vbq
