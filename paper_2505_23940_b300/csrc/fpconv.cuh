// Exact binary32 <-> binary64 conversions done with integer field arithmetic
// (IEEE 754-2008 §3.4 encodings: sign, biased exponent, trailing significand;
// narrowing rounds to nearest, ties to even, §4.3.1).
//
// On B300 every FP64 instruction, conversions included, goes through a narrow
// FP64 pipe; the y solve of the mixed-precision pressure step is bound by it.
// Widening the FP32 spectrum to FP64 and narrowing the solution back with
// shifts, masks and adds moves two of its per-cell FP64 instructions onto the
// integer pipes, which run beside the FP64 pipe.  Results are bit-identical to
// the hardware conversions for every non-NaN input (NaN maps to a NaN).
//
// Plain C as well as CUDA, so that the host can check both functions
// exhaustively (binary32 -> binary64) and on every exponent range and rounding
// tie (binary64 -> binary32) against its own conversions.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define FSCONV_FN __host__ __device__ __forceinline__
#else
#define FSCONV_FN static inline
#endif

FSCONV_FN uint32_t fsconv_clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__clz((int)v);
#else
  return v ? (uint32_t)__builtin_clz(v) : 32u;
#endif
}

// binary32 bits -> binary64 bits (hi word, lo word)
FSCONV_FN void fsconv_widen_bits(uint32_t u, uint32_t* hi, uint32_t* lo) {
  const uint32_t sign = u & 0x80000000u, mag = u & 0x7fffffffu;
  const uint32_t e8 = mag >> 23, man = mag & 0x7fffffu;
  if (e8 - 1u < 254u) {
    // normal: rebias the exponent by 1023 - 127 = 896; the 23 fraction bits become the
    // top 23 of the 52 (20 in the high word, 3 at the top of the low word)
    *hi = sign | ((mag >> 3) + (896u << 20));
    *lo = man << 29;
  } else if (e8 == 255u) {
    *hi = sign | 0x7ff00000u | (man >> 3) | (man ? 0x80000u : 0u);   // inf; NaN made quiet
    *lo = man << 29;
  } else if (man == 0u) {
    *hi = sign;   // signed zero
    *lo = 0u;
  } else {
    // subnormal man * 2^-149: normalise the leading one to bit 23, exponent -126 - shift
    const uint32_t sh = fsconv_clz32(man) - 8u;
    const uint32_t m = man << sh;
    *hi = sign | ((897u - sh) << 20) | ((m & 0x7fffffu) >> 3);
    *lo = m << 29;
  }
}

// binary64 bits -> binary32 bits, round to nearest even
FSCONV_FN uint32_t fsconv_narrow_bits(uint32_t hi, uint32_t lo) {
  const uint32_t sign = hi & 0x80000000u, mhi = hi & 0x7fffffffu;
  const uint32_t e11 = mhi >> 20;
  if (e11 - 897u < 254u) {
    // result exponent 1..254: bits 29..60 of the magnitude hold the exponent (mod 2^9) and the
    // top 23 fraction bits; rebiasing by 896 << 23 wraps correctly modulo 2^32
    const uint32_t t = ((mhi << 3) | (lo >> 29)) - (896u << 23);
    const uint32_t rem = lo & 0x1fffffffu;
    const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & t);
    return sign | (t + up);   // a carry out of the fraction steps the exponent (to inf from 254)
  }
  if (e11 >= 1151u) {
    if (e11 == 2047u && ((mhi & 0xfffffu) | lo)) return sign | 0x7fc00000u | ((mhi & 0xfffffu) << 3);
    return sign | 0x7f800000u;   // |x| >= 2^128 and inf
  }
  if (e11 < 873u) return sign;   // |x| < 2^-150 (2^-150 itself ties to zero below)
  // subnormal result: q = M >> (926 - e11) with the 53-bit significand M, rounded to even
  const uint64_t M = ((uint64_t)((mhi & 0xfffffu) | 0x100000u) << 32) | lo;
  const uint32_t sh = 926u - e11;   // 30..53
  const uint64_t q = M >> sh;
  const uint64_t rem = M & ((1ull << sh) - 1ull);
  const uint64_t half = 1ull << (sh - 1u);
  const uint32_t up = (rem > half) || (rem == half && (q & 1ull));
  return sign | (uint32_t)(q + up);
}

// Fast paths: normal numbers and zeros, the values of the y solve; `special` is set for
// every other input (subnormal, infinite, NaN, and for narrowing also out-of-range
// magnitudes), which the caller then converts with the general routines above.
FSCONV_FN void fsconv_widen_fast(uint32_t u, uint32_t* hi, uint32_t* lo, uint32_t* special) {
  const uint32_t mag = u & 0x7fffffffu;
  *hi = mag ? (u & 0x80000000u) | ((mag >> 3) + (896u << 20)) : u;
  *lo = u << 29;
  *special |= (uint32_t)((mag - 0x00800000u) >= 0x7f000000u && mag != 0u);
}

FSCONV_FN uint32_t fsconv_narrow_fast(uint32_t hi, uint32_t lo, uint32_t* special) {
  const uint32_t sign = hi & 0x80000000u, mhi = hi & 0x7fffffffu;
  const uint32_t t = ((mhi << 3) | (lo >> 29)) - (896u << 23);
  const uint32_t rem = (lo & 0x1fffffffu) + (t & 1u);   // ties go up only from an odd fraction
  const uint32_t r = t + (uint32_t)(rem > 0x10000000u);
  const int zero = (mhi | lo) == 0u;
  *special |= (uint32_t)(mhi - (897u << 20) >= (254u << 20) && !zero);
  return zero ? sign : (sign | r);
}

// The binary64 product RN(e * f) of a binary32 value f (bits u) and a binary64 value e (words
// ehi, elo), rounded to nearest even once, from integer products of the significands (24 x 53
// bits, 77 exact bits): the multiply of the twisted y solve's scaled elimination, moved off the
// FP64 pipe.  Fast path: f and e normal or zero with a normal (or zero) result; `special` is set
// for every other input, which the caller multiplies in FP64 instead.
FSCONV_FN void fsconv_scale_fast(uint32_t u, uint32_t ehi, uint32_t elo, uint32_t* hi, uint32_t* lo,
                                 uint32_t* special) {
  const uint32_t sign = (u ^ ehi) & 0x80000000u;
  const uint32_t fm = u & 0x7fffffffu, em = ehi & 0x7fffffffu;
  const uint32_t e8 = fm >> 23, e11 = em >> 20;
  const int fz = fm == 0u, ez = (em | elo) == 0u, zero = fz || ez;
  const uint64_t mf = (uint64_t)((fm & 0x7fffffu) | 0x800000u);
  const uint64_t p_lo = mf * elo;                                              // < 2^56
  const uint64_t p_hi = mf * (uint64_t)((em & 0xfffffu) | 0x100000u) + (p_lo >> 32);   // P >> 32 < 2^45
  const uint32_t p_lw = (uint32_t)p_lo;                                        // P mod 2^32
  const uint32_t sh = 23u + (uint32_t)(p_hi >> 44);                            // 24 when P >= 2^76
  uint64_t r = (p_hi << (32u - sh)) | (uint64_t)(p_lw >> sh);                  // P >> sh, 53 bits
  const uint32_t rem = p_lw & ((1u << sh) - 1u), half = 1u << (sh - 1u);
  r += (uint64_t)((rem > half) | ((rem == half) & (uint32_t)(r & 1u)));
  // biased exponent of r / 2^52; a rounding carry to 2^53 steps it (the fraction bits are then 0)
  const int32_t eb = (int32_t)e8 + (int32_t)e11 + (int32_t)sh - 150 + (int32_t)(r >> 53);
  const uint64_t bits = ((uint64_t)(uint32_t)eb << 52) + (r & 0xfffffffffffffull);
  const int fin = (e8 - 1u < 254u || fz) && (e11 - 1u < 2046u || ez);
  *special |= (uint32_t)(!fin || (!zero && (eb < 1 || eb > 2046)));
  *hi = zero ? sign : (sign | (uint32_t)(bits >> 32));
  *lo = zero ? 0u : (uint32_t)bits;
}

#ifdef __CUDACC__
__device__ __forceinline__ double fsconv_widen(float f) {
  uint32_t hi, lo;
  fsconv_widen_bits(__float_as_uint(f), &hi, &lo);
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float fsconv_narrow(double d) {
  return __uint_as_float(fsconv_narrow_bits((uint32_t)__double2hiint(d), (uint32_t)__double2loint(d)));
}
#endif
