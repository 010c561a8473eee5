// dp_emul.cuh -- IEEE 754 binary64 addition and multiplication, round to
// nearest-even, computed with integer operations only.
//
// Why: GB300's FP64 unit issues 2 lane-operations per clock per SM, 1/64 of the
// FP32 rate, while its integer pipes sit idle during the binary64 stencil.
// Points whose update is computed here run on the integer pipes concurrently
// with points computed by the FP64 unit, and give the same bits (both are the
// correctly rounded IEEE result).
//
// Domain: the fast routines handle finite operands whose exponent field is in
// 1..2046 (normal numbers) or that are +-0, with a normal or exactly zero
// result.  Anything else (subnormal operands or results, overflow, infinities,
// NaNs) sets `bad`; the caller then recomputes the point with the FP64 unit.
// The routines are written from the definition of binary64 (sign, 11-bit biased
// exponent, 52-bit fraction with an implicit leading 1) and of rounding to
// nearest with ties to even; they compile for the host too, so they are tested
// against the host's IEEE arithmetic.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define HEAT_HD __host__ __device__ __forceinline__
#else
#define HEAT_HD static inline
#endif

namespace heat {
namespace emul {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kAbs = 0x7fffffffffffffffull;
constexpr uint64_t kFrac = 0x000fffffffffffffull;
constexpr uint64_t kImpl = 0x0010000000000000ull;

HEAT_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

HEAT_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Round-and-pack.  s holds the significand with its leading 1 at bit 62 and
// ten guard bits below bit 10, bit 0 carrying the sticky OR of anything lower;
// e is the biased exponent of that leading 1.  Returns the correctly rounded
// binary64 with the given sign, flags results that are not normal.
HEAT_HD uint64_t round_pack(uint64_t sign, int e, uint64_t s, bool &bad) {
  s += 0x1ffull + ((s >> 10) & 1ull);  // nearest, ties to even
  const uint64_t sig = s >> 10;       // 2^52 .. 2^53 (2^53 when rounding carried)
  const uint64_t mag = (((uint64_t)(e - 1)) << 52) + sig;
  bad |= (e < 1) | (e > 2046) | (mag >= 0x7ff0000000000000ull);  // subnormal or overflow
  return sign | mag;
}

// a + b.  Zeros are handled; other exceptional inputs set bad.
HEAT_HD uint64_t add(uint64_t a, uint64_t b, bool &bad) {
  uint64_t ma = a & kAbs, mb = b & kAbs;
  if (ma < mb) {
    const uint64_t t = a; a = b; b = t;
    const uint64_t u = ma; ma = mb; mb = u;
  }
  const int ea = (int)(ma >> 52), eb = (int)(mb >> 52);
  bad |= (ea == 2047);
  if (mb == 0) {           // x + (+-0) = x; (+-0) + (+-0) goes to the FP64 unit (sign rules)
    bad |= (ma == 0);
    return a;
  }
  bad |= (eb == 0);        // subnormal operand
  const uint64_t sa = ((ma & kFrac) | kImpl) << 10;  // leading 1 at bit 62
  uint64_t sb = ((mb & kFrac) | kImpl) << 10;
  const int d = ea - eb;   // 0 .. 2046
  if (d > 0) {
    if (d < 64) {
      const uint64_t lost = sb << (64 - d);
      sb = (sb >> d) | (lost != 0);
    } else {
      sb = 1;              // only the sticky bit survives
    }
  }
  uint64_t s;
  if ((a ^ b) & kSign) {
    s = sa - sb;
    if (s == 0) return 0;  // exact cancellation: +0 under round-to-nearest
  } else {
    s = sa + sb;
  }
  const int lz = clz64(s);  // 0 (carry into bit 63) .. 62
  int e = ea;
  if (lz == 0) {
    s = (s >> 1) | (s & 1ull);
    e += 1;
  } else if (lz > 1) {
    s <<= (lz - 1);         // no nonzero bits below the sticky position are lost: exact
    e -= (lz - 1);
  }
  return round_pack(a & kSign, e, s, bad);
}

// Significand and exponent of a nonzero normal multiplier, prepared once.
struct Mul {
  uint64_t sig11;  // significand with its leading 1 at bit 63
  int exp;         // biased exponent
  uint64_t sign;
  bool pow2;       // the multiplier is +-2^k: the product only moves the exponent
};

HEAT_HD Mul prepare_mul(uint64_t r) {
  Mul m;
  m.sig11 = ((r & kFrac) | kImpl) << 11;
  m.exp = (int)((r & kAbs) >> 52);
  m.sign = r & kSign;
  m.pow2 = (r & kFrac) == 0;
  return m;
}

// r * b for a multiplier r prepared by prepare_mul (normal, nonzero).
HEAT_HD uint64_t mul(const Mul &m, uint64_t b, bool &bad) {
  const uint64_t mb = b & kAbs;
  const uint64_t sign = (b & kSign) ^ m.sign;
  if (mb == 0) return sign;  // r * (+-0) = signed zero
  const int eb = (int)(mb >> 52);
  bad |= (eb == 0) | (eb == 2047);
  if (m.pow2) {            // exact: same fraction, exponent eb + k
    const int e = eb + m.exp - 1023;
    bad |= (e < 1) | (e > 2046);
    return sign | ((uint64_t)(e & 2047) << 52) | (mb & kFrac);
  }
  const uint64_t sb = ((mb & kFrac) | kImpl) << 11;  // leading 1 at bit 63
  // 128-bit product of two significands in [2^63, 2^64): in [2^126, 2^128)
  const uint64_t hi = mulhi64(sb, m.sig11);
  const uint64_t lo = sb * m.sig11;
  int e = eb + m.exp - 1023;
  uint64_t s;
  if (hi >> 63) {          // product in [2^127, 2^128): leading 1 at bit 63 of hi
    s = (hi >> 1) | (hi & 1ull) | (lo != 0);
    e += 1;
  } else {                 // leading 1 at bit 62 of hi
    s = hi | (lo != 0);
  }
  return round_pack(sign, e, s, bad);
}

// Exactly 2x for normal x (exponent + 1), zero stays zero.
HEAT_HD uint64_t twice(uint64_t x, bool &bad) {
  const uint64_t mx = x & kAbs;
  if (mx == 0) return x;
  const int ex = (int)(mx >> 52);
  bad |= (ex == 0) | (ex >= 2046);
  return x + kImpl;
}

// Eq. 2, exact reading: v = u + r*((ul - 2u) + ur), each step rounded to nearest.
HEAT_HD uint64_t eq2_exact(uint64_t ul, uint64_t u, uint64_t ur, const Mul &m, bool &bad) {
  const uint64_t t1 = add(ul, twice(u, bad) ^ kSign, bad);
  const uint64_t t2 = add(t1, ur, bad);
  const uint64_t t3 = mul(m, t2, bad);
  return add(u, t3, bad);
}

}  // namespace emul
}  // namespace heat
