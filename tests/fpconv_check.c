/* Host check of the integer-pipe FP32 <-> FP64 conversions and of the FP32 x
 * FP64 product of the y solve (paper_2505_23940_b300/csrc/fpconv.cuh) against
 * the host's IEEE 754 arithmetic: every binary32 value widened; binary64 values
 * from every exponent of and around the binary32 range, with rounding ties,
 * narrowed; products over every binary32 exponent, the under- and overflow
 * boundaries and constructed rounding ties; the fast paths agree on every input
 * they do not flag and flag exactly the rest.
 * Prints "ok" and exits 0, or the first mismatch and exits 1. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "fpconv.cuh"

static uint64_t dbits(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
static double bitsd(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float bitsf(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

static uint64_t s = 0x9e3779b97f4a7c15ull;
static uint64_t next(void) {   /* splitmix64 */
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static int narrow_one(uint64_t b) {
  const double d = bitsd(b);
  const uint32_t got = fsconv_narrow_bits((uint32_t)(b >> 32), (uint32_t)b);
  /* the fast path agrees wherever it does not flag the input, and flags exactly the
     inputs outside the normal binary32 range other than zeros */
  uint32_t sp = 0;
  const uint32_t fast = fsconv_narrow_fast((uint32_t)(b >> 32), (uint32_t)b, &sp);
  const uint32_t e11 = (uint32_t)(b >> 52) & 0x7ffu;
  const int normal = e11 >= 897u && e11 <= 1150u, zero = (b << 1) == 0;
  if (sp != (uint32_t)!(normal || zero) || (!sp && fast != got)) {
    printf("narrow fast %016llx: special %u fast %08x full %08x\n", (unsigned long long)b, sp, fast, got);
    return 1;
  }
  const float want = (float)d;
  if (isnan(d)) {
    if (!isnan(bitsf(got))) { printf("narrow NaN %016llx -> %08x\n", (unsigned long long)b, got); return 1; }
    return 0;
  }
  if (got != fbits(want)) {
    printf("narrow %016llx (%.17g): got %08x want %08x\n", (unsigned long long)b, d, got, fbits(want));
    return 1;
  }
  return 0;
}

/* binary32 x binary64 product: the fast path agrees with the host's IEEE product (one rounding,
   to nearest even) wherever it does not flag the input, and flags exactly the inputs that are not
   normal or zero and the products that are not normal (a product just below the smallest normal
   that rounds up to it may be flagged as well) */
static int scale_one(uint32_t u, uint64_t e) {
  uint32_t hi, lo, sp = 0;
  fsconv_scale_fast(u, (uint32_t)(e >> 32), (uint32_t)e, &hi, &lo, &sp);
  const double want = (double)bitsf(u) * bitsd(e);
  const uint64_t wb = dbits(want), got = ((uint64_t)hi << 32) | lo;
  const uint32_t e8 = (u >> 23) & 0xffu;
  const uint64_t e11 = (e >> 52) & 0x7ffu, we = (wb >> 52) & 0x7ffu;
  const int fz = (u << 1) == 0, ez = (e << 1) == 0;
  const int fin = ((e8 >= 1u && e8 <= 254u) || fz) && ((e11 >= 1u && e11 <= 2046u) || ez);
  const int plain = fin && (fz || ez || (we >= 1u && we <= 2046u));
  if ((!sp && !plain) || (sp && plain && we != 1u) || (!sp && got != wb)) {
    printf("scale %08x x %016llx: special %u got %016llx want %016llx\n", u, (unsigned long long)e, sp,
           (unsigned long long)got, (unsigned long long)wb);
    return 1;
  }
  return 0;
}

static uint64_t inv_mod24(uint64_t a) {   /* a odd: a^-1 mod 2^24 by Newton's iteration */
  uint64_t x = a;
  for (int i = 0; i < 5; ++i) x = (x * (2 - a * x)) & 0xffffffull;
  return x;
}

static int check_scale(void) {
  /* every binary32 exponent against sampled binary64 exponents (edges, the ranges where the product
     leaves the normal range, random), random significands and both signs */
  for (uint32_t e8 = 0; e8 < 256u; ++e8) {
    uint64_t exps[80];
    int ne = 0;
    const uint64_t edge[] = {0, 1, 2, 1022, 1023, 1024, 2045, 2046, 2047};
    for (unsigned q = 0; q < sizeof(edge) / sizeof(edge[0]); ++q) exps[ne++] = edge[q];
    for (int d = -3; d <= 3; ++d) {
      const long lo_e = 150 - 24 - (long)e8 + d, hi_e = 2046 + 150 - 24 - (long)e8 + d;
      if (lo_e >= 0 && lo_e < 2048) exps[ne++] = (uint64_t)lo_e;
      if (hi_e >= 0 && hi_e < 2048) exps[ne++] = (uint64_t)hi_e;
    }
    while (ne < 80) exps[ne++] = next() & 0x7ffull;
    for (int q = 0; q < ne; ++q)
      for (int r = 0; r < 24; ++r) {
        const uint32_t u = ((uint32_t)(next() & 1u) << 31) | (e8 << 23) | (uint32_t)(next() & 0x7fffffu);
        const uint64_t e = ((next() & 1ull) << 63) | (exps[q] << 52) | (next() & 0xfffffffffffffull);
        if (scale_one(u, e)) return 1;
        if (scale_one(u & 0x80000000u, e) || scale_one(u, e & 0x8000000000000000ull)) return 1;   /* zeros */
      }
  }
  /* rounding ties and their neighbours at both alignments: significand products with
     P mod 2^24 = 2^23 (a tie when P >= 2^76) or 2^22 (a tie when P < 2^76) */
  for (int r = 0; r < 400000; ++r) {
    const uint64_t mf = (next() & 0x7fffffull) | 0x800001ull;   /* odd */
    const uint64_t inv = inv_mod24(mf);
    const uint64_t target = (r & 1) ? (1ull << 23) : (1ull << 22);
    const uint64_t low = (target * inv) & 0xffffffull;
    for (int dd = -1; dd <= 1; ++dd) {
      const uint64_t me = ((next() & 0xfffffffull) << 24) | ((low + (uint64_t)(long long)dd) & 0xffffffull);
      const uint32_t e8 = 100u + (uint32_t)(next() % 50u);
      const uint64_t e11 = 900u + next() % 200u;
      const uint32_t u = (e8 << 23) | (uint32_t)(mf & 0x7fffffu);
      const uint64_t e = (e11 << 52) | (me & 0xfffffffffffffull);
      if (scale_one(u, e)) return 1;
    }
  }
  /* random bit patterns (specials included) */
  for (long r = 0; r < 20000000; ++r)
    if (scale_one((uint32_t)next(), next())) return 1;
  return 0;
}

int main(void) {
  if (check_scale()) return 1;
  /* widening: all 2^32 inputs */
  for (uint64_t i = 0; i < (1ull << 32); ++i) {
    const uint32_t u = (uint32_t)i;
    uint32_t hi, lo;
    fsconv_widen_bits(u, &hi, &lo);
    const float f = bitsf(u);
    const uint64_t got = ((uint64_t)hi << 32) | lo;
    uint32_t fh, fl, sp = 0;
    fsconv_widen_fast(u, &fh, &fl, &sp);
    const uint32_t e8 = (u >> 23) & 0xffu;
    const int plain = (e8 >= 1u && e8 <= 254u) || (u << 1) == 0;
    if (sp != (uint32_t)!plain || (!sp && (fh != hi || fl != lo))) {
      printf("widen fast %08x: special %u\n", u, sp);
      return 1;
    }
    if (isnan(f)) {
      if (!isnan(bitsd(got))) { printf("widen NaN %08x\n", u); return 1; }
      continue;
    }
    if (got != dbits((double)f)) {
      printf("widen %08x: got %016llx want %016llx\n", u, (unsigned long long)got,
             (unsigned long long)dbits((double)f));
      return 1;
    }
  }
  /* narrowing: every exponent 0..2047, both signs; mantissas random, all-ones, zero,
     and the rounding boundaries (tie, tie +- 1) at every shift the subnormal path uses */
  for (int sign = 0; sign < 2; ++sign)
    for (uint64_t e = 0; e < 2048; ++e) {
      const uint64_t base = ((uint64_t)sign << 63) | (e << 52);
      const uint64_t fixed[] = {0ull, 0xfffffffffffffull, 0x10000000ull, 0x10000000ull - 1, 0x10000000ull + 1,
                                0x30000000ull, 0xfffffefffffffull, 0x8000000000000ull, 1ull};
      for (unsigned q = 0; q < sizeof(fixed) / sizeof(fixed[0]); ++q)
        if (narrow_one(base | fixed[q])) return 1;
      for (int sh = 1; sh < 53; ++sh) {
        const uint64_t half = 1ull << (sh - 1);
        for (int r = 0; r < 8; ++r) {
          const uint64_t hi = (next() & 0xfffffffffffffull) & ~((1ull << sh) - 1);
          const uint64_t ms[3] = {hi | half, hi | (half - 1), hi | (half + 1)};
          for (int t = 0; t < 3; ++t)
            if (narrow_one(base | (ms[t] & 0xfffffffffffffull))) return 1;
        }
      }
      for (int r = 0; r < 2000; ++r)
        if (narrow_one(base | (next() & 0xfffffffffffffull))) return 1;
    }
  for (long r = 0; r < 20000000; ++r)
    if (narrow_one(next())) return 1;
  printf("ok\n");
  return 0;
}
