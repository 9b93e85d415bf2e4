// Integer-instruction helpers of the float64-accurate tensor-core kernels
// (k_ozaki.cu, k_ozgemm.cu): slicing a float64 into integer digits, and
// rounding an exact integer combination of slice-product levels back to
// float64.
//
// GB300 retires two float64 operations (and about sixteen conversions) per
// SM per clock against 128 fp32 or int32 ones, so slicing and epilogues that
// scale, round and convert in float64 are bound by those pipes.  Everything
// here works on the bits with fp32 and int32 instructions.
#pragma once

#include <cstdint>

namespace lrs {

// Biased exponent field of a float64 (0 for zero and subnormals, 0x7FF for
// infinities and NaN).
__device__ __forceinline__ int oz_exp_field(double x) {
  return (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
}

// Row scale from the largest exponent field of the row: every element has
// |x| < 2^(e - 1) with e = max(E, 1) - 1021, so x 2^-e lies in (-1/2, 1/2).
__device__ __forceinline__ int oz_row_scale(int max_exp_field) {
  return (max_exp_field > 1 ? max_exp_field : 1) - 1021;
}

// round(x 2^(56 - e)) for |x| < 2^(e - 1) (so |result| <= 2^55), rounding
// halves away from zero, from the bits of x.
__device__ __forceinline__ long long oz_fixed56(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)(b >> 52) & 0x7FF;
  const unsigned long long frac = b & 0xFFFFFFFFFFFFFull;
  const unsigned long long mx = E ? (frac | 0x10000000000000ull) : frac;   // x = mx 2^(ex)
  const int ex = E ? E - 1075 : -1074;
  const int sh = ex + 56 - e;   // <= 2 by the bound on x
  unsigned long long n;
  if (sh >= 0) n = mx << sh;
  else if (sh > -64) n = (mx + (1ull << (-sh - 1))) >> (-sh);
  else n = 0;
  return (b >> 63) ? -(long long)n : (long long)n;
}

// bf16 bit pattern of an integer |d| <= 256 (exact: at most 8 significant
// bits): the integer is placed in the mantissa of 1.5 2^23 by an integer add,
// recovered as an fp32 by one fp32 subtraction, and its top 16 bits are the
// bf16 value.
__device__ __forceinline__ uint16_t oz_int_to_bf16_bits(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return (uint16_t)(__float_as_uint(f) >> 16);
}

// An integer |S| <= 2^22 held exactly in fp32 (a level sum read from TMEM) as
// an int32: S + 1.5 2^23 lies in [2^23, 2^24], where consecutive integers are
// consecutive bit patterns.
__device__ __forceinline__ int oz_level_int(float s) {
  return __float_as_int(s + 12582912.0f) - 0x4B400000;
}

// The same without removing the bias: the bit pattern S + OZ_LEVEL_BIAS.  Combinations of
// several levels remove the bias once (below); the bias is a multiple of 2^22.
constexpr unsigned OZ_LEVEL_BIAS = 0x4B400000u;
__device__ __forceinline__ unsigned oz_level_bits(float s) { return __float_as_uint(s + 12582912.0f); }

// (S_a 2^W) + S_b from the biased bit patterns, in 32-bit arithmetic that wraps modulo 2^32:
// exact whenever the result fits in an int32.
template <int W>
__device__ __forceinline__ int oz_pair(unsigned ba, unsigned bb) {
  return (int)((ba << W) + bb - ((OZ_LEVEL_BIAS << W) + OZ_LEVEL_BIAS));
}

// floor(S / 2^W) from the biased bit pattern (W <= 22, so the bias divides exactly).
template <int W>
__device__ __forceinline__ int oz_level_shr(unsigned b) {
  return (int)(b >> W) - (int)(OZ_LEVEL_BIAS >> W);
}

// v 2^k rounded to float64 through the float64 pipe, for the results that oz_round_pow2
// does not assemble (subnormal or beyond the normal range): kept out of line so that its
// float64 instructions stay off the common path.
static __device__ __noinline__ double oz_i64_times_pow2_slow(long long v, int k) { return ldexp((double)v, k); }

// v 2^k rounded to the nearest float64 (ties to even) from the bits of v, without
// branches, for |v| < 2^63: the leading one is found on 32-bit halves (a clamped
// funnel shift normalises both cases), 53 bits are kept, the rounding bit is added
// after the exponent is assembled (a carry out of the fraction moves into the
// exponent, as it should), and v = 0 gives +0.  Where the exponent of the leading
// one leaves (-1020, 1022), `ok` is false and the result is +0; the caller then takes
// oz_i64_times_pow2_slow, which the slice scaling makes rare.
__device__ __forceinline__ double oz_round_pow2(long long v, int k, bool& ok) {
  const unsigned long long sm = (unsigned long long)(v >> 63);   // all ones when v < 0
  const unsigned long long a = ((unsigned long long)v ^ sm) - sm;
  const unsigned ah = (unsigned)(a >> 32), al = (unsigned)a;
  const bool big = ah != 0u;
  const unsigned xh = big ? ah : al, xl = big ? al : 0u;
  const unsigned s = (unsigned)__clz((int)xh);                 // 32 when a = 0
  const unsigned mh = __funnelshift_lc(xl, xh, s);             // a shifted to put its leading one at bit 63
  const unsigned ml = __funnelshift_lc(0u, xl, s);
  const unsigned nh = mh >> 11;                                // 53 bits, leading one at bit 52
  const unsigned nl = __funnelshift_r(ml, mh, 11);
  // ties to even: the 11 dropped bits plus the kept lowest bit carry out of 0x3FF + 0x400
  const unsigned up = ((ml & 0x7FFu) + (nl & 1u) + 0x3FFu) >> 11;
  const int e = (big ? 63 : 31) - (int)s + k;                  // exponent of the leading one
  const bool in_range = (unsigned)(e + 1019) <= 2040u;          // -1020 < e < 1022
  ok = in_range || xh == 0u;
  const unsigned hi = ((unsigned)(e + 1022) << 20) + nh;       // the leading one adds one to the field
  unsigned long long bits = ((((unsigned long long)hi) << 32) | nl) + up;
  bits |= sm & 0x8000000000000000ull;
  return __longlong_as_double((xh != 0u && in_range) ? (long long)bits : 0ll);
}

}  // namespace lrs
