// Host check of the integer binary64 routines in csrc/dp_emul.cuh against the
// host's IEEE 754 arithmetic (compiled with -ffp-contract=off).  Prints
// "mismatches=<n> bad=<n> checked=<n>" per category.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2307_01117_gb300/csrc/dp_emul.cuh"

using namespace heat::emul;

static uint64_t bits(double x) { uint64_t u; std::memcpy(&u, &x, 8); return u; }
static double dbl(uint64_t u) { double x; std::memcpy(&x, &u, 8); return x; }

struct Tally { long mism = 0, bad = 0, n = 0; };

static void check_add(Tally &t, double a, double b) {
  bool bad = false;
  const uint64_t got = add(bits(a), bits(b), bad);
  const double want = a + b;
  t.n++;
  if (bad) { t.bad++; return; }
  if (got != bits(want)) {
    if (t.mism < 5) std::printf("add mismatch %a + %a: got %a want %a\n", a, b, dbl(got), want);
    t.mism++;
  }
}

static void check_mul(Tally &t, double r, double b) {
  bool bad = false;
  const Mul m = prepare_mul(bits(r));
  const uint64_t got = mul(m, bits(b), bad);
  const double want = r * b;
  t.n++;
  if (bad) { t.bad++; return; }
  if (got != bits(want)) {
    if (t.mism < 5) std::printf("mul mismatch %a * %a: got %a want %a\n", r, b, dbl(got), want);
    t.mism++;
  }
}

static void check_eq2(Tally &t, double ul, double u, double ur, double r) {
  bool bad = false;
  const Mul m = prepare_mul(bits(r));
  const uint64_t got = eq2_exact(bits(ul), bits(u), bits(ur), m, bad);
  const double want = u + r * ((ul - 2.0 * u) + ur);
  t.n++;
  if (bad) { t.bad++; return; }
  if (got != bits(want)) {
    if (t.mism < 5) std::printf("eq2 mismatch ul=%a u=%a ur=%a r=%a: got %a want %a\n", ul, u, ur, r, dbl(got), want);
    t.mism++;
  }
}

// ---- unpacked form (whole tiles) ----

static void check_addx(Tally &t, double a, double b) {
  const uint64_t got = pack(add(unpack(bits(a)), unpack(bits(b))));
  const double want = a + b;
  t.n++;
  if (got != bits(want)) {
    if (t.mism < 5) std::printf("addx mismatch %a + %a: got %a want %a\n", a, b, dbl(got), want);
    t.mism++;
  }
}

static void check_mulx(Tally &t, double r, double b) {
  const MulX m = prepare_mulx(bits(r));
  const X x = unpack(bits(b));
  const uint64_t got = pack(m.pow2 ? scale(x, m) : mul(x, m));
  const double want = r * b;
  t.n++;
  if (got != bits(want)) {
    if (t.mism < 5) std::printf("mulx mismatch %a * %a: got %a want %a\n", r, b, dbl(got), want);
    t.mism++;
  }
}

// T steps of Eq. 2 on a periodic ring, unpacked, against IEEE binary64 step by
// step; inputs must pass the screen for (r, T) (counted as skipped otherwise).
static void check_tile(Tally &t, std::vector<double> u, double r, int T) {
  int lo = 0, hi = 0;
  t.n++;
  if (!domain_bounds(bits(r), T, lo, hi)) { t.bad++; return; }
  for (double v : u)
    if (!in_domain(bits(v), lo, hi)) { t.bad++; return; }
  const size_t n = u.size();
  const MulX m = prepare_mulx(bits(r));
  std::vector<X> x(n), y(n);
  for (size_t i = 0; i < n; ++i) x[i] = unpack(bits(u[i]));
  std::vector<double> w(n);
  for (int s = 0; s < T; ++s) {
    for (size_t i = 0; i < n; ++i) {
      const size_t l = (i + n - 1) % n, rr = (i + 1) % n;
      w[i] = u[i] + r * ((u[l] - 2.0 * u[i]) + u[rr]);
      y[i] = m.pow2 ? (m.neg ? eq2x<true, true>(x[l], x[i], x[rr], m) : eq2x<true, false>(x[l], x[i], x[rr], m))
                    : (m.neg ? eq2x<false, true>(x[l], x[i], x[rr], m) : eq2x<false, false>(x[l], x[i], x[rr], m));
    }
    u.swap(w);
    x.swap(y);
  }
  for (size_t i = 0; i < n; ++i) {
    if (pack(x[i]) != bits(u[i])) {
      if (t.mism < 5) std::printf("tile mismatch r=%a T=%d i=%zu: got %a want %a\n", r, T, i, dbl(pack(x[i])), u[i]);
      t.mism++;
      return;
    }
  }
}

int main(int argc, char **argv) {
  long n = argc > 1 ? std::atol(argv[1]) : 2000000;
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> E(-60, 60), Esmall(-3, 3), D(0, 70);
  Tally ta, tm, te, tr, tt;
  for (long i = 0; i < n; ++i) {
    // random magnitudes over a wide range
    const double a = std::ldexp(U(g), E(g)), b = std::ldexp(U(g), E(g));
    check_add(ta, a, b);
    check_add(ta, a, -a * (1.0 + std::ldexp(U(g), -D(g))));     // near cancellation
    check_add(ta, a, std::ldexp(a, -D(g)));                     // exponent differences 0..70
    check_add(ta, a, -std::ldexp(a, -D(g)));
    check_mul(tm, std::ldexp(std::fabs(U(g)) + 0.5, Esmall(g)), b);
    check_mul(tm, 0.25, b);
    // Eq. 2 chains on nearby values (smooth fields) and on unrelated values
    const double u = U(g), r = 0.5 * std::fabs(U(g)) + 1e-3;
    check_eq2(te, u + 1e-3 * U(g), u, u + 1e-3 * U(g), r);
    check_eq2(te, U(g), U(g), U(g), r);
    check_eq2(te, (double)(i % 4000), (double)((i + 1) % 4000), (double)((i + 2) % 4000), 0.5);
    // raw random bit patterns (exceptional ones must be flagged, never wrong)
    const uint64_t x = g(), y = g();
    check_add(tr, dbl(x), dbl(y));
    check_mul(tr, std::ldexp(std::fabs(U(g)) + 0.5, E(g)), dbl(y));
  }
  // exact ties: 1 + 2^-53 (ties to even -> 1), 1 + 3*2^-53 (-> 1 + 2^-51), carries through all-ones
  check_add(tt, 1.0, std::ldexp(1.0, -53));
  check_add(tt, 1.0, 3.0 * std::ldexp(1.0, -53));
  check_add(tt, 1.0 + std::ldexp(1.0, -52), std::ldexp(1.0, -53));
  check_add(tt, std::nextafter(2.0, 0.0), std::ldexp(1.0, -53));
  check_add(tt, -1.0, std::ldexp(1.0, -54));
  check_add(tt, 1.5, -1.5);
  check_add(tt, 0.0, 3.0);
  check_add(tt, -0.0, 3.0);
  check_mul(tt, 1.0 + std::ldexp(1.0, -52), 1.0 + std::ldexp(1.0, -52));
  check_mul(tt, 3.0, 1.0 / 3.0);
  check_mul(tt, 0.1, -0.0);
  // unpacked form: single operations on normal operands with normal or zero results
  Tally xa, xm, xt, xe;
  for (long i = 0; i < n; ++i) {
    const double a = std::ldexp(U(g), E(g)), b = std::ldexp(U(g), E(g));
    check_addx(xa, a, b);
    check_addx(xa, a, -a);                                        // exact cancellation: +0
    check_addx(xa, a, -a * (1.0 + std::ldexp(U(g), -D(g))));
    check_addx(xa, a, std::ldexp(a, -D(g)));
    check_addx(xa, a, -std::ldexp(a, -D(g)));
    check_addx(xa, a, std::ldexp(b, -8 * D(g)));                 // exponent differences up to 560
    check_addx(xa, 0.0, b);
    check_mulx(xm, std::ldexp(std::fabs(U(g)) + 0.5, Esmall(g)) * (i & 1 ? -1.0 : 1.0), b);
    check_mulx(xm, (i & 2) ? -0.25 : 0.25, b);
    check_mulx(xm, 0.3, 0.0);
  }
  {
    const double e = std::ldexp(1.0, -53);
    const double pairs[][2] = {{1.0, e}, {1.0, 3 * e}, {1.0 + 2 * e, e}, {std::nextafter(2.0, 0.0), e},
                               {-1.0, e / 2}, {-1.0, -e}, {-1.0, -3 * e}, {1.5, -1.5}, {0.0, 3.0}, {3.0, 0.0},
                               {0.0, 0.0}, {-std::nextafter(2.0, 0.0), -e}, {std::ldexp(1.0, 600), 1.0},
                               {-std::ldexp(1.0, 600), 1.0}, {1.0, -std::ldexp(1.0, -600)}};
    for (auto &p : pairs) check_addx(xe, p[0], p[1]);
    check_mulx(xe, 1.0 + 2 * e, 1.0 + 2 * e);
    check_mulx(xe, 3.0, 1.0 / 3.0);
    check_mulx(xe, -3.0, 1.0 / 3.0);
    check_mulx(xe, std::nextafter(2.0, 0.0), std::nextafter(2.0, 0.0));
    // exact ties of the product (the discarded part is exactly half an ulp), both signs
    const double u52 = std::ldexp(1.0, -52);
    const double tie_x[] = {1.0 + u52, 1.0 + 3 * u52, 1.0 + 5 * u52, 2.0 - u52};
    const double tie_r[] = {3.0, 1.5, 0.75, -3.0, -1.5};
    for (double xv : tie_x)
      for (double rv : tie_r) {
        check_mulx(xe, rv, xv);
        check_mulx(xe, rv, -xv);
      }
  }
  // whole tiles: smooth, random, integer-valued (zero second differences), near
  // the screen's lower bound, mixed magnitudes; several r and T
  const double rs[] = {0.25, 0.5, 0.3, 0.123456789, 1e-3, -0.3, 2.0, 0.4999};
  const int Ts[] = {1, 4, 8, 12, 24, 40};
  for (long i = 0; i < std::max(1L, n / 2000); ++i) {
    for (double r : rs) {
      for (int T : Ts) {
        int lo = 0, hi = 0;
        if (!domain_bounds(bits(r), T, lo, hi)) continue;
        // deep blocks: r = 2^k only (for other r the screen then excludes ordinary data)
        if (T > 12 && (bits(r) & 0x000fffffffffffffull) != 0) continue;
        std::vector<double> a(64), b(64), c(64), d(64), f(64);
        const double base = U(g);
        for (int k = 0; k < 64; ++k) {
          a[k] = base + 1e-6 * std::sin(0.1 * k) + std::ldexp(U(g), -40);
          b[k] = U(g);
          c[k] = (double)((k * 7 + i) % 50);
          d[k] = std::ldexp(1.0 + std::fabs(U(g)), lo - 1023 + (int)(g() % 4));
          f[k] = std::ldexp(U(g), (int)(g() % 200) - 100);
        }
        check_tile(xt, a, r, T);
        check_tile(xt, b, r, T);
        check_tile(xt, c, r, T);
        check_tile(xt, d, r, T);
        check_tile(xt, f, r, T);
      }
    }
  }
  std::printf("addx mismatches=%ld bad=%ld checked=%ld\n", xa.mism, xa.bad, xa.n);
  std::printf("mulx mismatches=%ld bad=%ld checked=%ld\n", xm.mism, xm.bad, xm.n);
  std::printf("edgex mismatches=%ld bad=%ld checked=%ld\n", xe.mism, xe.bad, xe.n);
  std::printf("tile mismatches=%ld bad=%ld checked=%ld\n", xt.mism, xt.bad, xt.n);
  if (xa.mism || xm.mism || xe.mism || xt.mism) return 1;
  std::printf("add mismatches=%ld bad=%ld checked=%ld\n", ta.mism, ta.bad, ta.n);
  std::printf("mul mismatches=%ld bad=%ld checked=%ld\n", tm.mism, tm.bad, tm.n);
  std::printf("eq2 mismatches=%ld bad=%ld checked=%ld\n", te.mism, te.bad, te.n);
  std::printf("raw mismatches=%ld bad=%ld checked=%ld\n", tr.mism, tr.bad, tr.n);
  std::printf("edge mismatches=%ld bad=%ld checked=%ld\n", tt.mism, tt.bad, tt.n);
  return (ta.mism || tm.mism || te.mism || tr.mism || tt.mism) ? 1 : 0;
}
