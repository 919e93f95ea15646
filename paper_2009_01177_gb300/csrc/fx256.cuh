// fx256.cuh -- 256-bit fixed-point arithmetic for the fourth precision tier.
//
// The paper's 256-bit mode (Sec. 5.1-5.2): one global scaling factor, products
// truncated, on the integer unit.  Representation: a signed (two's complement)
// 256-bit integer X in four 64-bit limbs, value X * 2^-192.  The scale is
// limb-aligned, so the product of two values is limbs 3..6 of their 512-bit
// product and no bit shifts are needed; the 63 integer bits hold every
// intermediate of an instance with t_max = 1/sqrt(det(I - O)) <= 2^30
// (the pivot inverses 1/det2 <= t_max^2 are the largest).
//
// The product is accumulated column by column (each column is the sum of the
// low halves of the limb products a_i b_j with i + j equal to the column and
// the high halves of those one column lower): by default each column summed
// on its own in 128 bits, then one carry propagation; TOR_FX4_MUL_CHAIN=1
// uses a single PTX multiply-add carry chain through the columns instead.
// Columns 0..2 lie below the kept part: only their carries into column 3 are
// dropped, an error of a few units of 2^-192 on top of the truncation
// (Sec. 5.1 truncates too).  Overflow of the 255-bit magnitude
// range sets a flag instead of wrapping silently.
#pragma once
#include <cstdint>

namespace tor {

struct fx4 {
  unsigned long long w[4];  // little-endian limbs, value = signed int / 2^192
};

constexpr int FX256_FRAC = 192;

__device__ __forceinline__ bool fx4_neg_p(const fx4 &a) { return (long long)a.w[3] < 0; }

__device__ __forceinline__ fx4 fx4_neg(const fx4 &a) {
  fx4 r;
  asm("sub.cc.u64 %0, 0, %4;\n\t"
      "subc.cc.u64 %1, 0, %5;\n\t"
      "subc.cc.u64 %2, 0, %6;\n\t"
      "subc.u64 %3, 0, %7;"
      : "=l"(r.w[0]), "=l"(r.w[1]), "=l"(r.w[2]), "=l"(r.w[3])
      : "l"(a.w[0]), "l"(a.w[1]), "l"(a.w[2]), "l"(a.w[3]));
  return r;
}

__device__ __forceinline__ fx4 fx4_add(const fx4 &a, const fx4 &b) {
  fx4 r;
  asm("add.cc.u64 %0, %4, %8;\n\t"
      "addc.cc.u64 %1, %5, %9;\n\t"
      "addc.cc.u64 %2, %6, %10;\n\t"
      "addc.u64 %3, %7, %11;"
      : "=l"(r.w[0]), "=l"(r.w[1]), "=l"(r.w[2]), "=l"(r.w[3])
      : "l"(a.w[0]), "l"(a.w[1]), "l"(a.w[2]), "l"(a.w[3]), "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]),
        "l"(b.w[3]));
  return r;
}

__device__ __forceinline__ fx4 fx4_sub(const fx4 &a, const fx4 &b) {
  fx4 r;
  asm("sub.cc.u64 %0, %4, %8;\n\t"
      "subc.cc.u64 %1, %5, %9;\n\t"
      "subc.cc.u64 %2, %6, %10;\n\t"
      "subc.u64 %3, %7, %11;"
      : "=l"(r.w[0]), "=l"(r.w[1]), "=l"(r.w[2]), "=l"(r.w[3])
      : "l"(a.w[0]), "l"(a.w[1]), "l"(a.w[2]), "l"(a.w[3]), "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]),
        "l"(b.w[3]));
  return r;
}

// (c0, c1, c2) += low or high 64 bits of x y, with carries into c1 and c2
__device__ __forceinline__ void col_lo(unsigned long long &c0, unsigned long long &c1, unsigned long long &c2,
                                       unsigned long long x, unsigned long long y) {
  asm("mad.lo.cc.u64 %0, %3, %4, %0;\n\t"
      "addc.cc.u64 %1, %1, 0;\n\t"
      "addc.u64 %2, %2, 0;"
      : "+l"(c0), "+l"(c1), "+l"(c2)
      : "l"(x), "l"(y));
}
__device__ __forceinline__ void col_hi(unsigned long long &c0, unsigned long long &c1, unsigned long long &c2,
                                       unsigned long long x, unsigned long long y) {
  asm("mad.hi.cc.u64 %0, %3, %4, %0;\n\t"
      "addc.cc.u64 %1, %1, 0;\n\t"
      "addc.u64 %2, %2, 0;"
      : "+l"(c0), "+l"(c1), "+l"(c2)
      : "l"(x), "l"(y));
}

#ifndef TOR_FX4_MUL_CHAIN
#define TOR_FX4_MUL_CHAIN 0
#endif

// (a * b) >> 192 on magnitudes, truncated, sign restored; ovf = 1 when the
// result does not fit in 255 magnitude bits
__device__ __forceinline__ fx4 fx4_mul(const fx4 &a, const fx4 &b, int &ovf) {
  const bool na = fx4_neg_p(a), nb = fx4_neg_p(b);
  const fx4 ua = na ? fx4_neg(a) : a, ub = nb ? fx4_neg(b) : b;
  const unsigned long long *x = ua.w, *y = ub.w;
  fx4 r;
#if TOR_FX4_MUL_CHAIN
  // one carry chain through the columns in order
  unsigned long long c0 = 0ull, c1 = 0ull, c2 = 0ull;
  // column 3: low halves of i + j = 3, high halves of i + j = 2
  col_hi(c0, c1, c2, x[0], y[2]); col_hi(c0, c1, c2, x[1], y[1]); col_hi(c0, c1, c2, x[2], y[0]);
  col_lo(c0, c1, c2, x[0], y[3]); col_lo(c0, c1, c2, x[1], y[2]);
  col_lo(c0, c1, c2, x[2], y[1]); col_lo(c0, c1, c2, x[3], y[0]);
  r.w[0] = c0; c0 = c1; c1 = c2; c2 = 0ull;
  // column 4
  col_hi(c0, c1, c2, x[0], y[3]); col_hi(c0, c1, c2, x[1], y[2]);
  col_hi(c0, c1, c2, x[2], y[1]); col_hi(c0, c1, c2, x[3], y[0]);
  col_lo(c0, c1, c2, x[1], y[3]); col_lo(c0, c1, c2, x[2], y[2]); col_lo(c0, c1, c2, x[3], y[1]);
  r.w[1] = c0; c0 = c1; c1 = c2; c2 = 0ull;
  // column 5
  col_hi(c0, c1, c2, x[1], y[3]); col_hi(c0, c1, c2, x[2], y[2]); col_hi(c0, c1, c2, x[3], y[1]);
  col_lo(c0, c1, c2, x[2], y[3]); col_lo(c0, c1, c2, x[3], y[2]);
  r.w[2] = c0; c0 = c1; c1 = c2; c2 = 0ull;
  // column 6
  col_hi(c0, c1, c2, x[2], y[3]); col_hi(c0, c1, c2, x[3], y[2]);
  col_lo(c0, c1, c2, x[3], y[3]);
  r.w[3] = c0; c0 = c1; c1 = c2; c2 = 0ull;
  // column 7 and above must be empty, and the top bit of column 6 clear
  col_hi(c0, c1, c2, x[3], y[3]);
  if (c0 | c1 | c2 | (r.w[3] >> 63)) ovf = 1;
#else
  // the same columns summed independently (each fits 128 bits: at most seven
  // 64-bit terms), so the multiplies and the four column sums can overlap;
  // then one short carry propagation across the columns
  typedef unsigned __int128 u128;
  const u128 p02 = (u128)x[0] * y[2], p11 = (u128)x[1] * y[1], p20 = (u128)x[2] * y[0];
  const u128 p03 = (u128)x[0] * y[3], p12 = (u128)x[1] * y[2], p21 = (u128)x[2] * y[1], p30 = (u128)x[3] * y[0];
  const u128 p13 = (u128)x[1] * y[3], p22 = (u128)x[2] * y[2], p31 = (u128)x[3] * y[1];
  const u128 p23 = (u128)x[2] * y[3], p32 = (u128)x[3] * y[2];
  const u128 p33 = (u128)x[3] * y[3];
  const unsigned long long M = ~0ull;
  const u128 s3 = (p02 >> 64) + (p11 >> 64) + (p20 >> 64) + (u128)(unsigned long long)(p03 & M) +
                  (u128)(unsigned long long)(p12 & M) + (u128)(unsigned long long)(p21 & M) +
                  (u128)(unsigned long long)(p30 & M);
  const u128 s4 = (p03 >> 64) + (p12 >> 64) + (p21 >> 64) + (p30 >> 64) + (u128)(unsigned long long)(p13 & M) +
                  (u128)(unsigned long long)(p22 & M) + (u128)(unsigned long long)(p31 & M);
  const u128 s5 = (p13 >> 64) + (p22 >> 64) + (p31 >> 64) + (u128)(unsigned long long)(p23 & M) +
                  (u128)(unsigned long long)(p32 & M);
  const u128 s6 = (p23 >> 64) + (p32 >> 64) + (u128)(unsigned long long)(p33 & M);
  u128 t = s3;
  r.w[0] = (unsigned long long)t;
  t = s4 + (t >> 64);
  r.w[1] = (unsigned long long)t;
  t = s5 + (t >> 64);
  r.w[2] = (unsigned long long)t;
  t = s6 + (t >> 64);
  r.w[3] = (unsigned long long)t;
  t = (p33 >> 64) + (t >> 64);  // column 7 and above must be empty, and bit 255 clear
  if (t != 0 || (r.w[3] >> 63)) ovf = 1;
#endif
  return (na != nb) ? fx4_neg(r) : r;
}

}  // namespace tor
