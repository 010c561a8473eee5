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

// ---------------------------------------------------------------------------
// Unpacked form, for whole temporal-blocking tiles on the integer pipes.
//
// A value is held as x = m * 2^e with m a signed (two's complement) 64-bit
// integer whose magnitude has its leading 1 at bit 59 (2^59 <= |m| <= 2^60,
// the 53-bit significand shifted left by 7, low 7 bits zero), or m = 0 (x = +0)
// with e very negative.  A tile's values are unpacked once, advanced T steps
// without packing, and packed once.  The tile's inputs are screened first
// (in_domain): zero or a normal magnitude within [2^(lo-1023), 2^(hi-1022)),
// bounds the host derives from T and r so that every intermediate result of
// the T steps is +0 or a normal, finite binary64 number (no -0: it cannot
// arise from such inputs).  Under that guarantee add/mul/eq2 below are the
// correctly rounded binary64 operations without any range test.
struct X {
  int64_t m;
  int32_t e;
  int32_t pad;
};

constexpr int32_t kZeroE = -(1 << 24);  // exponent of +0: below every other

HEAT_HD X unpack(uint64_t b) {  // b: +0 or normal
  const int be = (int)(b >> 52) & 2047;
  const int64_t mag = (int64_t)(((b & kFrac) | kImpl) << 7);
  X x;
  x.m = be ? ((b >> 63) ? -mag : mag) : 0;
  x.e = be ? be - 1082 : kZeroE;
  x.pad = 0;
  return x;
}

HEAT_HD uint64_t pack(X x) {
  const uint64_t mag = (uint64_t)(x.m < 0 ? -x.m : x.m) >> 7;
  // biased exponent e + 1082 for |m| in [2^59, 2^60); |m| = 2^60 carries into it
  const uint64_t v = ((uint64_t)(x.e + 1081) << 52) + mag;
  return x.m ? (((uint64_t)x.m & kSign) | v) : 0ull;
}

// Screen: +0, or a normal value with biased exponent in [lo, hi].
HEAT_HD bool in_domain(uint64_t b, int lo, int hi) {
  const int be = (int)(b >> 52) & 2047;
  return b == 0 || (be >= lo && be <= hi);
}

// Position of the most significant bit that differs from the sign bit (the
// leading 1 of |v| for v >= 0, of |v| - 1 for v < 0); -1 for v = 0 or -1.
HEAT_HD int msb_signed(int64_t v) {
#if defined(__CUDA_ARCH__)
  unsigned p;
  asm("bfind.s64 %0, %1;" : "=r"(p) : "l"(v));  // 0xffffffff when v is all sign bits
  return (int)p;
#else
  const uint64_t t = (uint64_t)(v ^ (v >> 63));
  return t ? 63 - __builtin_clzll(t) : -1;
#endif
}

// x + y, rounded to nearest-even.  The smaller-exponent operand is aligned to
// the other by an arithmetic right shift whose lost bits are kept as a sticky
// 1 in bit 0 (|A|, |B| <= 2^60, so |S| <= 2^61); the sum is shifted left until
// its leading bit sits at bit 61 and rounded at bit 9 with
// floor((S + 255 + bit9) / 2^9) * 2^9, which is round to nearest-even for two's
// complement values too, then moved to bit 59.  A negative power of two
// normalises one place high and rounds exactly to |m| = 2^60.
HEAT_HD X add(X x, X y) {
  const int d = x.e - y.e;
  const bool sw = d < 0;
  const int64_t A = sw ? y.m : x.m;
  const int64_t Bs = sw ? x.m : y.m;
  const int eb = sw ? y.e : x.e;
  const int sh = sw ? -d : d;
#if defined(__CUDA_ARCH__)
  // PTX clamps shift amounts above the register width (sh exceeds 2^24 against
  // a +0 operand): Bs >> sh is then all sign bits and B << sh is 0, the same
  // result as a shift by 63 with the sticky set
  int64_t B;
  asm("shr.s64 %0, %1, %2;" : "=l"(B) : "l"(Bs), "r"(sh));
  uint64_t Bb;
  asm("shl.b64 %0, %1, %2;" : "=l"(Bb) : "l"(B), "r"(sh));
  B |= (int64_t)(Bb != (uint64_t)Bs);  // sticky
#else
  const int shc = sh < 63 ? sh : 63;
  int64_t B = Bs >> shc;
  B |= (int64_t)(((uint64_t)B << shc) != (uint64_t)Bs);  // sticky
#endif
  const int64_t S = A + B;
  const int p = msb_signed(S);                           // -1 (S = 0) .. 61
  const int64_t Sn = (int64_t)((uint64_t)S << (61 - p));
  const int64_t q = (Sn + 255 + ((Sn >> 9) & 1)) & ~(int64_t)511;
  X r;
  r.m = q >> 2;
  r.e = p >= 0 ? eb + p - 59 : kZeroE;
  r.pad = 0;
  return r;
}

// A multiplier r (normal, nonzero) prepared for the unpacked form.
struct MulX {
  int64_t sig10;   // significand (in [2^52, 2^53)) shifted left by 10: in [2^62, 2^63)
  int e;           // r = sig * 2^e
  bool neg;
  bool pow2;       // r = +-2^k: the product only moves the exponent
};

HEAT_HD MulX prepare_mulx(uint64_t r) {
  MulX m;
  m.sig10 = (int64_t)(((r & kFrac) | kImpl) << 10);
  m.e = (int)((r & kAbs) >> 52) - 1075;
  m.neg = (r >> 63) != 0;
  m.pow2 = (r & kFrac) == 0;
  return m;
}

// |r| * x for r = +-2^k.
HEAT_HD X scale_mag(X x, const MulX &r) {
  X y;
  y.m = x.m;
  y.e = x.e + r.e + 52;
  y.pad = 0;
  return y;
}

// r * x for r = +-2^k.
HEAT_HD X scale(X x, const MulX &r) {
  X y = scale_mag(x, r);
  if (r.neg) y.m = -y.m;
  return y;
}

HEAT_HD int64_t mulhi_s64(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * b) >> 64);
#endif
}

// |r| * x, rounded to nearest-even, on the signed value: (m * 2^2) * (sig *
// 2^10) is a two's complement 128-bit product P with |P| in [2^123, 2^125).
// Its high word V = floor(P / 2^64) has the leading bit of |P| at bit 59 or
// 60 (found on the one's complement, as in add), so the 53 kept bits end at
// bit q = 7 or 8; V is rounded at q by floor((V + 2^(q-1) - 1 + (s | bit_q)) /
// 2^q) * 2^q with s = (low word != 0) -- round to nearest-even for two's
// complement values with the low word as the discarded fraction -- and shifted
// to a leading bit at 59.  A negative r negates the rounded result (rounding to
// nearest is symmetric): mul below; mul_mag leaves the sign of r out.
HEAT_HD X mul_mag(X x, const MulX &r) {
  const int64_t a = (int64_t)((uint64_t)x.m << 2);
  const int64_t V = mulhi_s64(a, r.sig10);
  const uint64_t lo = (uint64_t)a * (uint64_t)r.sig10;
  const int top = (int)(((uint64_t)(V ^ (V >> 63)) >> 60) & 1);  // leading bit at 60 (1) or 59 (0)
  // q = 7 + top: 2^(q-1) - 1 and the mask of bits q.. as selects of constants
  const int64_t half_m1 = top ? 127 : 63;
  const int64_t keep = top ? ~(int64_t)255 : ~(int64_t)127;
  const int64_t inc = half_m1 + (int64_t)((lo != 0) | ((V >> (7 + top)) & 1));
  const int64_t R = (V + inc) & keep;
  X y;
  y.m = R >> top;
  y.e = x.e + r.e + 52 + top;
  y.pad = 0;
  return y;
}

HEAT_HD X mul(X x, const MulX &r) {
  X y = mul_mag(x, r);
  if (r.neg) y.m = -y.m;
  return y;
}

// Eq. 2, exact reading, unpacked: u + r*((ul - 2u) + ur), each step rounded.
// POW2: r = +-2^k; NEG: r < 0 (the sign is fixed at compile time so that a
// step does not select it per point).
template <bool POW2, bool NEG>
HEAT_HD X eq2x(X ul, X u, X ur, const MulX &r) {
  X m2u;
  m2u.m = -u.m;  // -2u, exact
  m2u.e = u.e + 1;
  m2u.pad = 0;
  const X t2 = add(add(ul, m2u), ur);
  X p = POW2 ? scale_mag(t2, r) : mul_mag(t2, r);
  if (NEG) p.m = -p.m;
  return add(u, p);
}

// Screening bounds for T steps with multiplier r (normal, nonzero); false when
// no input passes.  Every value the steps produce is an integer multiple of
// the inputs' granularity g = 2^(emin - 52), shrunk by at most 2^(52 - e_r)
// per step through the rounded product (by exactly 2^e_r when r = +-2^e_r,
// whose products are exact), so a nonzero result is at least
// g * 2^(-T * shrink); magnitudes grow at most by (1 + 4|r|) per step.
HEAT_HD bool domain_bounds(uint64_t r, int T, int &lo, int &hi) {
  const int er = (int)((r & kAbs) >> 52) - 1023;  // |r| in [2^er, 2^(er+1))
  const bool pow2 = (r & kFrac) == 0;
  const int shrink = pow2 ? (er < 0 ? -er : 0) : (er < 52 ? 52 - er : 0);
  lo = 53 + T * shrink + 3;
  // ceil(log2(1 + 4|r|)) <= max(er + 3, 0) + 1
  const int grow = (er + 3 > 0 ? er + 3 : 0) + 1;
  hi = 2040 - T * (grow + 1) - (er > 0 ? er + 1 : 0);
  return lo <= hi;
}

}  // namespace emul
}  // namespace heat
