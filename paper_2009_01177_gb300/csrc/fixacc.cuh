// fixacc.cuh -- exact 256-bit fixed-point accumulation of positive doubles.
//
// The paper sums its subset terms in fixed point with one global scaling
// factor (Sec. 5.1-5.2).  Here the same idea runs on the GPU's integer pipe:
// every term t_Z >= 2^-75 is a double whose lowest mantissa bit weighs at
// least 2^-128, so a two's-complement integer with 128 fractional bits holds
// it, and any sum of such terms, EXACTLY.  The 128 integer bits bound the sum
// by 2^127.  Positive and negative terms of Eq. 2 go to two accumulators,
// so that sum_abs = pos + neg and Tor = pos - neg are both exact.
//
// Integer adds with carry cost nothing next to the FP64 pipe on sm_103a
// (about 60 integer ops per clock per SM against 2 DFMA), which is why the
// alternating sum is kept off the FP64 pipe entirely.
#pragma once
#include <cstdint>

namespace tor {

struct Fx256 {
  unsigned long long w[4];  // little-endian limbs, value = signed int / 2^128
};

__host__ __device__ __forceinline__ void fx_zero(Fx256 &a) { a.w[0] = a.w[1] = a.w[2] = a.w[3] = 0ull; }

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ void fx_add(Fx256 &a, const Fx256 &b) {
  asm("add.cc.u64 %0, %0, %4;\n\t"
      "addc.cc.u64 %1, %1, %5;\n\t"
      "addc.cc.u64 %2, %2, %6;\n\t"
      "addc.u64 %3, %3, %7;"
      : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3])
      : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]), "l"(b.w[3]));
}
__device__ __forceinline__ void fx_sub(Fx256 &a, const Fx256 &b) {
  asm("sub.cc.u64 %0, %0, %4;\n\t"
      "subc.cc.u64 %1, %1, %5;\n\t"
      "subc.cc.u64 %2, %2, %6;\n\t"
      "subc.u64 %3, %3, %7;"
      : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3])
      : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]), "l"(b.w[3]));
}
#else
inline void fx_add(Fx256 &a, const Fx256 &b) {
  unsigned long long c = 0;
  for (int i = 0; i < 4; ++i) {
    unsigned long long s = a.w[i] + b.w[i];
    unsigned long long c1 = s < a.w[i];
    unsigned long long s2 = s + c;
    unsigned long long c2 = s2 < s;
    a.w[i] = s2;
    c = c1 | c2;
  }
}
inline void fx_sub(Fx256 &a, const Fx256 &b) {
  unsigned long long br = 0;
  for (int i = 0; i < 4; ++i) {
    unsigned long long d = a.w[i] - b.w[i];
    unsigned long long b1 = a.w[i] < b.w[i];
    unsigned long long d2 = d - br;
    unsigned long long b2 = d < br;
    a.w[i] = d2;
    br = b1 | b2;
  }
}
#endif

// Place a positive double x exactly as a 256-bit fixed-point number.
// Returns false (and a zero X) when x is not a finite positive double with
// 2^-75 <= x < 2^75; such a term cannot come from a positive definite input
// of the sizes the library accepts, and the caller flags it.
__host__ __device__ __forceinline__ bool fx_from_pos_double(double x, Fx256 &X) {
#if defined(__CUDA_ARCH__)
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long bits;
  __builtin_memcpy(&bits, &x, 8);
#endif
  const int e = (int)((bits >> 52) & 0x7FFull);
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = e - 947;  // weight of m's lowest bit, 2^(e-1075), in units of 2^-128
  const bool ok = ((bits >> 63) == 0ull) && (e != 0) && (sh >= 0) && (sh <= 202);
  const int shc = ok ? sh : 0;
  const int q = shc >> 6, s = shc & 63;
  const unsigned long long lo = ok ? (m << s) : 0ull;
  const unsigned long long hi = ok ? ((m >> 1) >> (63 - s)) : 0ull;  // m >> (64 - s), 0 when s == 0
  X.w[0] = (q == 0) ? lo : 0ull;
  X.w[1] = (q == 1) ? lo : ((q == 0) ? hi : 0ull);
  X.w[2] = (q == 2) ? lo : ((q == 1) ? hi : 0ull);
  X.w[3] = (q == 3) ? lo : ((q == 2) ? hi : 0ull);
  return ok;
}

// Nearest-ish double of a signed 256-bit fixed-point value (top 64 bits,
// rounded to nearest by the integer-to-double conversion).
__host__ __device__ inline double fx_to_double(const Fx256 &a) {
  const bool neg = (a.w[3] >> 63) != 0ull;
  Fx256 m = a;
  if (neg) {
    Fx256 z;
    fx_zero(z);
    fx_sub(z, a);
    m = z;
  }
  int top = -1;
  for (int i = 3; i >= 0 && top < 0; --i) {
    if (m.w[i]) {
#if defined(__CUDA_ARCH__)
      top = 64 * i + 63 - __clzll((long long)m.w[i]);
#else
      top = 64 * i + 63 - __builtin_clzll(m.w[i]);
#endif
    }
  }
  if (top < 0) return 0.0;
  int lo = top - 63;
  if (lo < 0) lo = 0;
  const int q = lo >> 6, s = lo & 63;
  unsigned long long bits = m.w[q] >> s;
  if (s && q + 1 < 4) bits |= m.w[q + 1] << (64 - s);
  double d = (double)bits;  // one rounding to nearest
#if defined(__CUDA_ARCH__)
  d = scalbn(d, lo - 128);
#else
  d = __builtin_scalbn(d, lo - 128);
#endif
  return neg ? -d : d;
}

// Value as hi + lo (lo = rounded remainder after removing hi exactly).
__host__ __device__ inline void fx_to_dd(const Fx256 &a, double &hi, double &lo) {
  hi = fx_to_double(a);
  Fx256 r = a, h;
  const double ah = hi < 0 ? -hi : hi;
  if (ah != 0.0 && fx_from_pos_double(ah, h)) {
    if (hi > 0) fx_sub(r, h); else fx_add(r, h);
    lo = fx_to_double(r);
  } else {
    lo = 0.0;
  }
}

}  // namespace tor
