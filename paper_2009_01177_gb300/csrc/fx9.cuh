// fx9.cuh -- fixed-point arithmetic of the 256-bit-class tier in nine 29-bit limbs.
//
// The paper's multiprecision mode (Sec. 5.1-5.2): one global scaling factor,
// products truncated to the scale, on the integer unit.  The GB300 form:
//
//   value = sum_{i=0..8} l_i 2^(29 i) * 2^-203,   l_i in [-2^28, 2^28)
//
// i.e. 261 bits of balanced ("signed-digit") limbs in nine 32-bit registers,
// 203 fraction bits (seven limbs) and a magnitude below 2^57.  A product of two
// limbs has at most 56 magnitude bits, so a column of the schoolbook product
// (at most nine limb products) and even a fused  s + a1 b1 + a2 b2  (eighteen
// products and one limb of s) sum in a signed 64-bit register with no carry:
// every limb product is one 32 x 32 -> 64-bit multiply-add (mad.wide.s32)
// into its column, with no carry chains and no sign handling, and only one
// carry pass per result.  Negation is limb by limb.
//
// Rounding: columns 0..5 of the 17 product columns are not formed (for
// balanced operands they hold at most 1.5 units of 2^-203 per product), and
// column 6 is rounded to nearest into column 7 by the balanced carry pass, so
// a product is off by at most 2 units of 2^-203 and a fused two-product
// operation by at most 3.5.  A result whose magnitude reaches 2^57 sets the
// overflow flag.
#pragma once
#include <cstdint>

namespace tor {

struct fx9 {
  int l[9];
};

constexpr int FX9_LIMBS = 9;
constexpr int FX9_BITS = 29;   // bits per limb
constexpr int FX9_FRAC = 203;  // fraction bits: 7 limbs
constexpr int FX9_ONE_LIMB = 7;  // limb of weight 2^0
constexpr int FX9_HALF = 1 << 28;
constexpr unsigned FX9_MASK = (1u << 29) - 1u;

// acc += a * b (signed 32 x 32 -> 64)
__device__ __forceinline__ void fx9_mac(long long &acc, int a, int b) {
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

__device__ __forceinline__ fx9 fx9_zero() {
  fx9 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.l[i] = 0;
  return r;
}

__device__ __forceinline__ fx9 fx9_int(int v) {  // small integer, |v| < 2^28
  fx9 r = fx9_zero();
  r.l[FX9_ONE_LIMB] = v;
  return r;
}

__device__ __forceinline__ fx9 fx9_neg(const fx9 &a) {
  fx9 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.l[i] = -a.l[i];
  return r;
}

// columns c = 6..16 of the product a b added into col[c - 6]
__device__ __forceinline__ void fx9_columns(long long (&col)[11], const fx9 &a, const fx9 &b) {
#pragma unroll
  for (int c = 6; c <= 16; ++c) {
#pragma unroll
    for (int i = (c > 8 ? c - 8 : 0); i <= (c < 8 ? c : 8); ++i) fx9_mac(col[c - 6], a.l[i], b.l[c - i]);
  }
}

// the same for a b whose b has limbs 0..JB only (the rest zero)
template <int JB>
__device__ __forceinline__ void fx9_columns_short(long long (&col)[11], const fx9 &a, const fx9 &b) {
#pragma unroll
  for (int c = 6; c <= 16; ++c) {
#pragma unroll
    for (int i = (c > 8 ? c - 8 : 0); i <= (c < 8 ? c : 8); ++i)
      if (c - i <= JB) fx9_mac(col[c - 6], a.l[i], b.l[c - i]);
  }
}

// column accumulators: column 6 starts at the rounding bias, columns 7..15 at
// the balanced-carry bias 2^28 plus the limbs of s (if any), column 16 at 0
__device__ __forceinline__ void fx9_init(long long (&col)[11]) {
#pragma unroll
  for (int c = 0; c < 10; ++c) col[c] = FX9_HALF;
  col[10] = 0;
}
__device__ __forceinline__ void fx9_init(long long (&col)[11], const fx9 &s) {
  col[0] = FX9_HALF;
#pragma unroll
  for (int m = 0; m < 9; ++m) col[m + 1] = (long long)s.l[m] + FX9_HALF;
  col[10] = 0;
}

// balanced carry pass: columns 7..15 -> limbs 0..8; ovf when the result's
// magnitude reaches 2^57 (a carry out of limb 8, or column 16 non-zero)
__device__ __forceinline__ fx9 fx9_carry(const long long (&col)[11], int &ovf) {
  fx9 r;
  long long c = col[0] >> 29;  // column 6, rounded to nearest
#pragma unroll
  for (int m = 0; m < 9; ++m) {
    const long long v = col[m + 1] + c;  // includes the bias 2^28
    r.l[m] = (int)((unsigned)v & FX9_MASK) - FX9_HALF;
    c = v >> 29;
  }
  if ((c + col[10]) != 0) ovf = 1;
  return r;
}

// a b
__device__ __forceinline__ fx9 fx9_mul(const fx9 &a, const fx9 &b, int &ovf) {
  long long col[11];
  fx9_init(col);
  fx9_columns(col, a, b);
  return fx9_carry(col, ovf);
}

// s + a b
__device__ __forceinline__ fx9 fx9_fma(const fx9 &s, const fx9 &a, const fx9 &b, int &ovf) {
  long long col[11];
  fx9_init(col, s);
  fx9_columns(col, a, b);
  return fx9_carry(col, ovf);
}

// a1 b1 + a2 b2
__device__ __forceinline__ fx9 fx9_dot2(const fx9 &a1, const fx9 &b1, const fx9 &a2, const fx9 &b2, int &ovf) {
  long long col[11];
  fx9_init(col);
  fx9_columns(col, a1, b1);
  fx9_columns(col, a2, b2);
  return fx9_carry(col, ovf);
}

// s + a1 b1 + a2 b2
__device__ __forceinline__ fx9 fx9_fma2(const fx9 &s, const fx9 &a1, const fx9 &b1, const fx9 &a2, const fx9 &b2,
                                        int &ovf) {
  long long col[11];
  fx9_init(col, s);
  fx9_columns(col, a1, b1);
  fx9_columns(col, a2, b2);
  return fx9_carry(col, ovf);
}

// a + b (limb by limb, then one carry pass so the limbs stay balanced)
__device__ __forceinline__ fx9 fx9_add(const fx9 &a, const fx9 &b, int &ovf) {
  long long col[11];
  col[0] = FX9_HALF;
#pragma unroll
  for (int m = 0; m < 9; ++m) col[m + 1] = (long long)a.l[m] + b.l[m] + FX9_HALF;
  col[10] = 0;
  return fx9_carry(col, ovf);
}

__device__ __forceinline__ fx9 fx9_sub(const fx9 &a, const fx9 &b, int &ovf) {
  long long col[11];
  col[0] = FX9_HALF;
#pragma unroll
  for (int m = 0; m < 9; ++m) col[m + 1] = (long long)a.l[m] - b.l[m] + FX9_HALF;
  col[10] = 0;
  return fx9_carry(col, ovf);
}

// a / 2 exactly when a is even in its last limb, else rounded toward -inf
// by 2^-204: each limb halved (arithmetic shift) with its low bit moved into
// the limb below as 2^28.  The limbs stay below 2^29 in magnitude, which every
// operation above accepts as an input.
__device__ __forceinline__ fx9 fx9_half(const fx9 &a) {
  fx9 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.l[i] = (a.l[i] >> 1) + (i < 8 ? ((a.l[i + 1] & 1) << 28) : 0);
  return r;
}

// nearest-ish double of a value whose magnitude is at least 2^-58 (relative
// error below 2^-56): three 58-bit limb pairs, two roundings
__device__ __forceinline__ double fx9_to_double(const fx9 &a) {
  const long long hi = ((long long)a.l[8] << 29) + a.l[7];   // weight 2^0
  const long long mid = ((long long)a.l[6] << 29) + a.l[5];  // weight 2^-58
  const long long lo = ((long long)a.l[4] << 29) + a.l[3];   // weight 2^-116
  return fma((double)mid, 0x1p-58, fma((double)lo, 0x1p-116, (double)hi));
}

// the double x as a value, exactly when 2^-150 <= |x| < 2^57 (its lowest
// mantissa bit at or above 2^-203); smaller magnitudes keep the bits at or
// above 2^-203 (toward zero), zero and subnormals give 0; |x| >= 2^57,
// infinities and NaN set ovf.  Limbs come out in [0, 2^29) for x >= 0
// (negated for x < 0): valid operands, normalised by the next operation.
__device__ __forceinline__ fx9 fx9_from_double(double x, int &ovf) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  fx9 r = fx9_zero();
  if (e == 0) return r;
  if (e >= 1023 + 57) { ovf = 1; return r; }
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  int sh = e - 1075 + FX9_FRAC;  // x = m 2^sh in units of 2^-203
  unsigned long long mm = m;
  if (sh < 0) {
    mm = (sh > -64) ? (m >> (-sh)) : 0ull;
    sh = 0;
  }
  const int q = sh / 29, b = sh - 29 * q;  // limb and bit of mm's lowest bit
  // mm 2^b spans three limbs: bits [0, 29 - b), [29 - b, 58 - b), [58 - b, 53 + b)
  const unsigned l0 = (unsigned)(mm << b) & FX9_MASK;
  const unsigned l1 = (unsigned)(mm >> (29 - b)) & FX9_MASK;
  const unsigned l2 = (unsigned)(mm >> (58 - b));
#pragma unroll
  for (int i = 0; i < 9; ++i) r.l[i] = (i == q) ? (int)l0 : (i == q + 1) ? (int)l1 : (i == q + 2) ? (int)l2 : 0;
  return (bits >> 63) ? fx9_neg(r) : r;
}

// sign of a normalised value: the sign of its highest non-zero limb
__device__ __forceinline__ int fx9_sign(const fx9 &a) {
  int s = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s = a.l[i] ? (a.l[i] > 0 ? 1 : -1) : s;
  return s;
}

}  // namespace tor
