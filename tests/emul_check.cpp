// Host check of the integer binary64 routines in csrc/dp_emul.cuh against the
// host's IEEE 754 arithmetic (compiled with -ffp-contract=off).  Prints
// "mismatches=<n> bad=<n> checked=<n>" per category.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

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
  std::printf("add mismatches=%ld bad=%ld checked=%ld\n", ta.mism, ta.bad, ta.n);
  std::printf("mul mismatches=%ld bad=%ld checked=%ld\n", tm.mism, tm.bad, tm.n);
  std::printf("eq2 mismatches=%ld bad=%ld checked=%ld\n", te.mism, te.bad, te.n);
  std::printf("raw mismatches=%ld bad=%ld checked=%ld\n", tr.mism, tr.bad, tr.n);
  std::printf("edge mismatches=%ld bad=%ld checked=%ld\n", tt.mism, tt.bad, tt.n);
  return (ta.mism || tm.mism || te.mism || tr.mism || tt.mism) ? 1 : 0;
}
