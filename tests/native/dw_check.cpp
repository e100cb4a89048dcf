// Host-side check of the double-word arithmetic in dw.cuh against extended
// precision (long double: 64-bit significand on x86-64, 113-bit on AArch64).
// Prints the largest observed error of each operation in units of the bound
// it must meet; test_dw_arith.py asserts every ratio <= 1.
#include <stdio.h>
#include <math.h>
#include <stdint.h>

#include "dw.cuh"

using mpcg::dw;
typedef long double ld;

static uint64_t state = 0x9E3779B97F4A7C15ULL;
static uint64_t next_u64() {   // splitmix64
  uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double uniform() { return (next_u64() >> 11) * (1.0 / 9007199254740992.0); }
// random double with exponent in [-emax, emax] and random sign
static double rnd(int emax) {
  const double m = 1.0 + uniform();
  const int e = (int)(next_u64() % (uint64_t)(2 * emax + 1)) - emax;
  return ((next_u64() & 1) ? -1.0 : 1.0) * ldexp(m, e);
}
static ld val(dw x) { return (ld)x.hi + (ld)x.lo; }
static dw rnd_dw(int emax) { return mpcg::dw_from_double(rnd(emax)); }

int main() {
  const ld u47 = ldexpl(1.0L, -47), u45 = ldexpl(1.0L, -45), u44 = ldexpl(1.0L, -44), u52 = ldexpl(1.0L, -52);
  double r_split = 0, r_back = 0, r_add = 0, r_mul = 0, r_fma = 0, r_div = 0, r_norm = 0;
  long fails_exact = 0;
  for (int it = 0; it < 200000; ++it) {
    const double d = rnd(90);
    const dw x = mpcg::dw_from_double(d);
    // split: hi + lo within 2^-47 of d, |lo| <= ulp(hi)
    const ld es = fabsl(val(x) - (ld)d) / (u47 * fabsl((ld)d));
    if (es > r_split) r_split = (double)es;
    const ld en = fabsl((ld)x.lo) / (ldexpl(1.0L, -23) * fabsl((ld)x.hi));
    if (en > r_norm) r_norm = (double)en;
    // assembling the pair back: within 2^-52 of the pair's exact value
    const double back = mpcg::dw_to_double(x.hi, x.lo);
    const ld eb = fabsl((ld)back - val(x)) / (u52 * fabsl(val(x)));
    if (eb > r_back) r_back = (double)eb;
    // the pair of a float-exact double assembles exactly
    const float f = (float)d;
    if (mpcg::dw_to_double(f, 0.f) != (double)f) ++fails_exact;
    const dw y = rnd_dw(30), z = rnd_dw(30), c = rnd_dw(60);
    const dw a = rnd_dw(30);
    // sums with cancellation too: y and its perturbed negative
    const dw yn = mpcg::dw_from_double(-(double)val(y) * (1.0 + ldexp(uniform(), -20)));
    for (int k = 0; k < 2; ++k) {
      const dw w = k ? yn : z;
      const ld ea = fabsl(val(y + w) - (val(y) + val(w))) / (u45 * (fabsl(val(y)) + fabsl(val(w))));
      if (ea > r_add) r_add = (double)ea;
    }
    const ld em = fabsl(val(y * z) - val(y) * val(z)) / (u45 * fabsl(val(y) * val(z)));
    if (em > r_mul) r_mul = (double)em;
    const dw fm = fma(a, z, c);
    const ld ef = fabsl(val(fm) - (val(c) + val(a) * val(z))) / (u44 * (fabsl(val(c)) + fabsl(val(a) * val(z))));
    if (ef > r_fma) r_fma = (double)ef;
    const ld ed = fabsl(val(y / z) - val(y) / val(z)) / (u44 * fabsl(val(y) / val(z)));
    if (ed > r_div) r_div = (double)ed;
  }
  // special values
  const dw zero = mpcg::dw_from_double(0.0), nzero = mpcg::dw_from_double(-0.0);
  const bool specials = zero.hi == 0.f && zero.lo == 0.f && signbit(nzero.hi) &&
                        mpcg::dw_to_double(0.f, 0.f) == 0.0 && mpcg::dw_to_double(1.f, 0.f) == 1.0 &&
                        mpcg::dw_to_double(-2.5f, 0.f) == -2.5 && (double)dw(3) == 3.0 &&
                        (double)mpcg::dw_from_double(0.1) != 0.0;
  printf("{\"split\": %.6g, \"lo_norm\": %.6g, \"assemble\": %.6g, \"add\": %.6g, \"mul\": %.6g, \"fma\": %.6g, "
         "\"div\": %.6g, \"exact_fails\": %ld, \"specials\": %d}\n",
         r_split, r_norm, r_back, r_add, r_mul, r_fma, r_div, fails_exact, specials ? 1 : 0);
  return 0;
}
