// stencil_ops.cuh -- the per-point update of Eq. 2 (Section 2) in the
// library's arithmetic forms.  Every operation is an explicit round-to-nearest
// intrinsic, so the compiler cannot contract or reorder it.
#pragma once

#include <cuda_runtime.h>

namespace heat {

// Eq. 2, exact reading: v = u + r*((ul - 2u) + ur), each operation rounded once.
// ul - 2u is issued as one fused multiply-add: 2u is exact in binary64 (for
// |u| <= DBL_MAX/2), so fma(-2, u, ul) rounds the same value ul - 2u once.
__device__ __forceinline__ double eq2_exact(double ul, double u, double ur, double r) {
  const double t1 = __fma_rn(-2.0, u, ul);
  const double t2 = __dadd_rn(t1, ur);
  const double t3 = __dmul_rn(r, t2);
  return __dadd_rn(u, t3);
}

// Eq. 2, fused reading: v = fma(r, (ul - 2u) + ur, u).
__device__ __forceinline__ double eq2_fma(double ul, double u, double ur, double r) {
  const double t1 = __fma_rn(-2.0, u, ul);
  const double t2 = __dadd_rn(t1, ur);
  return __fma_rn(r, t2, u);
}

// Eq. 2, exact reading, for r = +-2^k on operands screened so that every
// intermediate value is +0 or normal with room below (the integer-pipe tiles'
// screen): r * t2 is then exact and only moves t2's exponent, so it is done on
// the high word with an integer add (hi_add = k << 20) and a sign flip
// (hi_xor), +0 staying +0.  Three FP64-unit operations per point instead of
// four; the same bits as eq2_exact.
__device__ __forceinline__ double eq2_exact_pow2(double ul, double u, double ur, int hi_add, int hi_xor) {
  const double t2 = __dadd_rn(__fma_rn(-2.0, u, ul), ur);
  const int hi = __double2hiint(t2);
  const double t3 = __hiloint2double(hi == 0 ? 0 : ((hi + hi_add) ^ hi_xor), __double2loint(t2));
  return __dadd_rn(u, t3);
}

template <bool FMA>
__device__ __forceinline__ double eq2(double ul, double u, double ur, double r) {
  return FMA ? eq2_fma(ul, u, ur, r) : eq2_exact(ul, u, ur, r);
}

// Knuth's TwoSum: s = RN(a + b) and e with s + e == a + b exactly
// (no ordering assumption on |a|, |b|).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// One compensated binary32 step on a (hi, lo) pair:
//   d = ((hl - 2h) + hr) + ((ll - 2l) + lr);  inc = rf*d;
//   (s, e) = TwoSum(h, inc);  h' = s;  l' = l + e.
// 2h and 2l are exact in binary32 (below overflow), so the differences are
// issued as fused multiply-adds with one rounding each.
__device__ __forceinline__ void eq2_f32c(float hl, float h, float hr, float ll, float l, float lr, float rf,
                                         float &h_out, float &l_out) {
  const float dh = __fadd_rn(__fmaf_rn(-2.0f, h, hl), hr);
  const float dl = __fadd_rn(__fmaf_rn(-2.0f, l, ll), lr);
  const float d = __fadd_rn(dh, dl);
  const float inc = __fmul_rn(rf, d);
  float s, e;
  two_sum(h, inc, s, e);
  h_out = s;
  l_out = __fadd_rn(l, e);
}

// The same step on two points at once: each 64-bit operand holds two binary32
// values, and every operation but the product is the paired IEEE binary32
// operation with round-to-nearest (add/sub/fma .rn.f32x2), so each half is
// bitwise the scalar eq2_f32c.  The product rf*d is two scalar multiplies: a
// paired multiply feeding the paired add that follows was measured to round
// differently in some cases (as if the two had been fused), which the scalar
// form does not.  Paired instructions halve the issue slots the compensated
// update needs.
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ float f2_lo(unsigned long long v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return a;
}
__device__ __forceinline__ float f2_hi(unsigned long long v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return b;
}

__device__ __forceinline__ void eq2_f32c_x2(unsigned long long hl, unsigned long long h, unsigned long long hr,
                                            unsigned long long ll, unsigned long long l, unsigned long long lr,
                                            float rf, unsigned long long &h_out, unsigned long long &l_out) {
  // (-2, -2) built by a move, so that it is a register operand: an integer
  // literal in a paired floating-point instruction would not mean two -2.0f
  const unsigned long long m2 = f2_pack(-2.0f, -2.0f);
  const unsigned long long dh = f2_add(f2_fma(m2, h, hl), hr);
  const unsigned long long dl = f2_add(f2_fma(m2, l, ll), lr);
  const unsigned long long d = f2_add(dh, dl);
  const unsigned long long inc = f2_pack(__fmul_rn(rf, f2_lo(d)), __fmul_rn(rf, f2_hi(d)));
  // TwoSum(h, inc)
  const unsigned long long s = f2_add(h, inc);
  const unsigned long long bb = f2_sub(s, h);
  const unsigned long long e = f2_add(f2_sub(h, f2_sub(s, bb)), f2_sub(inc, bb));
  h_out = s;
  l_out = f2_add(l, e);
}

// End of a temporal block: the stored binary32 value RN(h + l).
__device__ __forceinline__ float f32c_store(float h, float l) { return __fadd_rn(h, l); }

}  // namespace heat
