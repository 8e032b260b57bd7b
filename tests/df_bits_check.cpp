// Host check of the bit-level double-FP32 split and widening
// (csrc/df_bits.cuh) against the host's IEEE conversions: hi = fl32(x),
// lo = fl32(x - hi), and (double)f.  Prints the number of mismatches.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "df_bits.cuh"

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {             // splitmix64
  uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static uint32_t fbits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }
static uint64_t dbits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static double from_bits(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static float from_fbits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }

static long bad_split = 0, bad_widen = 0, checked = 0, on_bit_path = 0;
static void check(double x) {
  float hi, lo;
  ntu::df_split_real(x, hi, lo);
  const float rh = (float)x;
  const float rl = (float)(x - (double)rh);
  const int E = (int)((dbits(x) >> 52) & 0x7ff);
  if (E >= 950 && E <= 1149) ++on_bit_path;
  ++checked;
  if (fbits(hi) != fbits(rh) || fbits(lo) != fbits(rl)) {
    if (bad_split < 5) printf("split mismatch x=%a: %a %a vs %a %a\n", x, hi, lo, rh, rl);
    ++bad_split;
  }
}
static void check_widen(float f) {
  const double w = ntu::df_widen(f), r = (double)f;
  if (dbits(w) != dbits(r) && !(isnan(w) && isnan(r))) {
    if (bad_widen < 5) printf("widen mismatch f=%a: %a vs %a\n", f, w, r);
    ++bad_widen;
  }
}

int main() {
  // edge cases: zeros, the ends of the bit path, ties, carries into the exponent
  const double edges[] = {0.0, -0.0, 1.0, -1.0, 0x1p-73, -0x1p-73, 0x1.fffffffffffffp-74,
                          0x1p127, 0x1.fffffffffffffp126, -0x1.fffffffffffffp126,
                          1.0 + 0x1p-24, 1.0 + 0x1p-24 + 0x1p-52, 1.0 + 3 * 0x1p-24,
                          0x1.fffffffp0, 0x1.ffffffp0, 0x1.fffffe8p0, 0x1.ffffff8p0,
                          1.0 / 3.0, -2.0 / 3.0, 0x1p-1022, 0x1p-1074, HUGE_VAL, -HUGE_VAL,
                          NAN, 0x1p-126, 0x1p-149, 1e-30, 1e30};
  for (double x : edges) check(x);
  // every tie pattern of the low 29 bits around 2^28, for both parities of s
  for (uint64_t s = 0; s < 4; ++s)
    for (int64_t d = -3; d <= 3; ++d) {
      const uint64_t low = (uint64_t)((1 << 28) + d) & 0x1fffffff;
      check(from_bits((1023ull << 52) | (s << 29) | low));
      check(from_bits((1100ull << 52) | (0xfffffffull << 29 >> 0) | (s << 29) | low));
      check(-from_bits((960ull << 52) | ((0x7fffffull - s) << 29) | low));
    }
  // random bit patterns over all exponents, and random values of the ALS range
  for (long i = 0; i < 4000000; ++i) {
    const uint64_t b = next_u64();
    check(from_bits(b));
    const int E = 900 + (int)(next_u64() % 300);
    check(from_bits((b & 0x800fffffffffffffull) | ((uint64_t)E << 52)));
  }
  for (long i = 0; i < 2000000; ++i) check_widen(from_fbits((uint32_t)next_u64()));
  const float fedges[] = {0.0f, -0.0f, 1.0f, 0x1p-126f, 0x1p-149f, -0x1p-149f, 3.4e38f,
                          INFINITY, -INFINITY};
  for (float f : fedges) check_widen(f);
  printf("checked %ld (bit path %ld) split mismatches %ld widen mismatches %ld\n", checked,
         on_bit_path, bad_split, bad_widen);
  return (bad_split || bad_widen) ? 1 : 0;
}
