// fx128.cuh -- 128-bit fixed-point arithmetic for the third precision tier.
//
// The paper's own answer to the Torontonian's cancellation is fixed point with
// ONE global scaling factor on the integer unit (Sec. 5.1-5.3: a 128-bit and a
// 256-bit mode, the scale set from the upper bound of all intermediates).  On
// GB300 the same choice pays for a different reason: FP64 runs at 2 FMA per
// clock per SM while the integer pipe does about 60 IMAD per clock, so a
// 128 x 128-bit fixed-point product (seven 64 x 64-bit partial products) costs
// about what one DFMA does, against ~20 FP64 operations for a double-double
// FMA.
//
// Representation: a signed (two's complement) 128-bit integer X, value
// X * 2^-F, with F fraction bits fixed per instance (kernel argument).  The
// caller picks F so that every intermediate (Schur entries, pivot inverses,
// the running term t_Z <= t_max) stays below 2^(126 - F).
//
// Products are truncated toward zero on the magnitude (the paper truncates,
// Sec. 5.1); overflow of the 128-bit range sets a flag instead of wrapping
// silently.
#pragma once
#include <cstdint>

// the product's words as independent 128-bit column sums (default; 3-7 % faster
// walks than one PTX carry chain, TOR_FX_MUL_U128=0, with the same bits)
#ifndef TOR_FX_MUL_U128
#define TOR_FX_MUL_U128 1
#endif

namespace tor {

struct fx {
  unsigned long long lo;
  long long hi;
};

__device__ __forceinline__ bool fx_neg_p(const fx &a) { return a.hi < 0; }

__device__ __forceinline__ fx fx_neg(const fx &a) {
  fx r;
  asm("sub.cc.u64 %0, 0, %2;\n\tsubc.u64 %1, 0, %3;" : "=l"(r.lo), "=l"(r.hi) : "l"(a.lo), "l"(a.hi));
  return r;
}

__device__ __forceinline__ fx fx_add(const fx &a, const fx &b) {
  fx r;
  asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;" : "=l"(r.lo), "=l"(r.hi)
      : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}

__device__ __forceinline__ fx fx_sub(const fx &a, const fx &b) {
  fx r;
  asm("sub.cc.u64 %0, %2, %4;\n\tsubc.u64 %1, %3, %5;" : "=l"(r.lo), "=l"(r.hi)
      : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}

// (a * b) >> F on magnitudes, sign restored; F in [64, 126].  ovf |= 1 when the
// result does not fit in 127 magnitude bits.
__device__ __forceinline__ fx fx_mul(const fx &a, const fx &b, int F, int &ovf) {
  const bool na = fx_neg_p(a), nb = fx_neg_p(b);
  const fx ua = na ? fx_neg(a) : a, ub = nb ? fx_neg(b) : b;
  const unsigned long long a0 = ua.lo, a1 = (unsigned long long)ua.hi;
  const unsigned long long b0 = ub.lo, b1 = (unsigned long long)ub.hi;
  // P = a1 b1 2^128 + (a1 b0 + a0 b1) 2^64 + a0 b0.  With each 64 x 64 product
  // split as h 2^64 + l, the low word l00 of a0 b0 lies wholly below 2^64, so
  // Q = P >> 64 = h11 2^128 + (l11 + h10 + h01) 2^64 + (l10 + l01 + h00) exactly.
#if TOR_FX_MUL_U128
  // the three words of Q as independent 128-bit column sums, then one carry pass
  typedef unsigned __int128 u128;
  const u128 p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
  const u128 c0 = (u128)__umul64hi(a0, b0) + (unsigned long long)p01 + (unsigned long long)p10;
  const u128 c1 = (p01 >> 64) + (p10 >> 64) + (unsigned long long)p11 + (c0 >> 64);
  const unsigned long long q0 = (unsigned long long)c0, q1 = (unsigned long long)c1;
  const unsigned long long q2 = (unsigned long long)(p11 >> 64) + (unsigned long long)(c1 >> 64);
#else
  const unsigned long long h00 = __umul64hi(a0, b0);
  const unsigned long long l10 = a1 * b0, h10 = __umul64hi(a1, b0);
  const unsigned long long l01 = a0 * b1, h01 = __umul64hi(a0, b1);
  const unsigned long long l11 = a1 * b1, h11 = __umul64hi(a1, b1);
  unsigned long long q0, q1, q2;
  asm("add.cc.u64  %0, %3, %4;\n\t"   // q0 = l10 + l01
      "addc.cc.u64 %1, %5, %6;\n\t"   // q1 = h10 + h01 + carry
      "addc.u64    %2, %7, 0;\n\t"    // q2 = h11 + carry
      "add.cc.u64  %0, %0, %8;\n\t"   // q0 += h00
      "addc.cc.u64 %1, %1, %9;\n\t"   // q1 += l11 + carry
      "addc.u64    %2, %2, 0;"          // q2 += carry
      : "=&l"(q0), "=&l"(q1), "=&l"(q2)
      : "l"(l10), "l"(l01), "l"(h10), "l"(h01), "l"(h11), "l"(h00), "l"(l11));
#endif
  const int s = F - 64;  // 0..62
  fx r;
  if (s == 0) {
    r.lo = q0;
    r.hi = (long long)q1;
    if (q2 | (q1 >> 63)) ovf = 1;
  } else {
    r.lo = (q0 >> s) | (q1 << (64 - s));
    const unsigned long long rhi = (q1 >> s) | (q2 << (64 - s));
    r.hi = (long long)rhi;
    if ((q2 >> s) | (rhi >> 63)) ovf = 1;
  }
  return (na != nb) ? fx_neg(r) : r;
}

}  // namespace tor
