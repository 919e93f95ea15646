// fixacc.cuh -- exact fixed-point accumulation of the subset terms.
//
// The paper sums its subset terms in fixed point with one global scaling
// factor (Sec. 5.1-5.2).  Here the same idea runs on the GPU's integer pipe:
// every term t_Z >= 2^-75 is a double whose lowest mantissa bit weighs at
// least 2^-128, so a two's-complement integer with 128 fractional bits holds
// it, and any sum of such terms, EXACTLY.  The 128 integer bits bound the sum
// by 2^127.  Positive and negative terms of Eq. 2 go to two accumulators,
// so that sum_abs = pos + neg and Tor = pos - neg are both exact.
//
// The accumulators are L 64-bit limbs with L/2 of them fraction: 256 bits
// (128 fraction bits) for the FP64, double-double and 128-bit fixed-point
// tiers, whose terms have no bits below 2^-128, and 512 bits (256 fraction
// bits) for the partial sums of the 256-bit-class tier, whose terms carry 203
// fraction bits (tor_fx9.cuh).
//
// Integer adds with carry cost nothing next to the FP64 pipe on sm_103a
// (about 60 integer ops per clock per SM against 2 DFMA), which is why the
// alternating sum is kept off the FP64 pipe entirely.
#pragma once
#include <cstdint>

namespace tor {

template <int L>
struct alignas(16) FxW {
  unsigned long long w[L];  // little-endian limbs, value = signed int / 2^(32 L)
};
using Fx256 = FxW<4>;  // 128 fraction bits
using Fx512 = FxW<8>;  // 256 fraction bits

template <int L>
__host__ __device__ __forceinline__ void fx_zero(FxW<L> &a) {
#pragma unroll
  for (int i = 0; i < L; ++i) a.w[i] = 0ull;
}

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
__device__ __forceinline__ void fx_add(Fx512 &a, const Fx512 &b) {
  asm("add.cc.u64 %0, %0, %8;\n\t"
      "addc.cc.u64 %1, %1, %9;\n\t"
      "addc.cc.u64 %2, %2, %10;\n\t"
      "addc.cc.u64 %3, %3, %11;\n\t"
      "addc.cc.u64 %4, %4, %12;\n\t"
      "addc.cc.u64 %5, %5, %13;\n\t"
      "addc.cc.u64 %6, %6, %14;\n\t"
      "addc.u64 %7, %7, %15;"
      : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3]), "+l"(a.w[4]), "+l"(a.w[5]), "+l"(a.w[6]),
        "+l"(a.w[7])
      : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]), "l"(b.w[3]), "l"(b.w[4]), "l"(b.w[5]), "l"(b.w[6]), "l"(b.w[7]));
}
__device__ __forceinline__ void fx_sub(Fx512 &a, const Fx512 &b) {
  asm("sub.cc.u64 %0, %0, %8;\n\t"
      "subc.cc.u64 %1, %1, %9;\n\t"
      "subc.cc.u64 %2, %2, %10;\n\t"
      "subc.cc.u64 %3, %3, %11;\n\t"
      "subc.cc.u64 %4, %4, %12;\n\t"
      "subc.cc.u64 %5, %5, %13;\n\t"
      "subc.cc.u64 %6, %6, %14;\n\t"
      "subc.u64 %7, %7, %15;"
      : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3]), "+l"(a.w[4]), "+l"(a.w[5]), "+l"(a.w[6]),
        "+l"(a.w[7])
      : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]), "l"(b.w[3]), "l"(b.w[4]), "l"(b.w[5]), "l"(b.w[6]), "l"(b.w[7]));
}
#else
template <int L>
inline void fx_add(FxW<L> &a, const FxW<L> &b) {
  unsigned long long c = 0;
  for (int i = 0; i < L; ++i) {
    unsigned long long s = a.w[i] + b.w[i];
    unsigned long long c1 = s < a.w[i];
    unsigned long long s2 = s + c;
    unsigned long long c2 = s2 < s;
    a.w[i] = s2;
    c = c1 | c2;
  }
}
template <int L>
inline void fx_sub(FxW<L> &a, const FxW<L> &b) {
  unsigned long long br = 0;
  for (int i = 0; i < L; ++i) {
    unsigned long long d = a.w[i] - b.w[i];
    unsigned long long b1 = a.w[i] < b.w[i];
    unsigned long long d2 = d - br;
    unsigned long long b2 = d < br;
    a.w[i] = d2;
    br = b1 | b2;
  }
}
#endif

// Place a positive double x exactly as an L-limb fixed-point number (32 L
// fraction bits).  Returns false (and a zero X) when x is not a finite
// positive double whose lowest mantissa bit is at least 2^-(32 L) and whose
// value stays below 2^(32 L - 2); such a term cannot come from a positive
// definite input of the sizes the library accepts, and the caller flags it.
template <int L>
__host__ __device__ __forceinline__ bool fx_from_pos_double(double x, FxW<L> &X) {
#if defined(__CUDA_ARCH__)
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long bits;
  __builtin_memcpy(&bits, &x, 8);
#endif
  const int e = (int)((bits >> 52) & 0x7FFull);
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = e - 1075 + 32 * L;  // weight of m's lowest bit, 2^(e-1075), in units of 2^-(32 L)
  const bool ok = ((bits >> 63) == 0ull) && (e != 0) && (sh >= 0) && (sh <= 64 * L - 54);
  const int shc = ok ? sh : 0;
  const int q = shc >> 6, s = shc & 63;
  const unsigned long long lo = ok ? (m << s) : 0ull;
  const unsigned long long hi = ok ? ((m >> 1) >> (63 - s)) : 0ull;  // m >> (64 - s), 0 when s == 0
#pragma unroll
  for (int i = 0; i < L; ++i) X.w[i] = (q == i) ? lo : ((q + 1 == i) ? hi : 0ull);
  return ok;
}

// Nearest-ish double of a signed fixed-point value (top 64 bits, rounded to
// nearest by the integer-to-double conversion).
template <int L>
__host__ __device__ inline double fx_to_double(const FxW<L> &a) {
  const bool neg = (a.w[L - 1] >> 63) != 0ull;
  FxW<L> m = a;
  if (neg) {
    FxW<L> z;
    fx_zero(z);
    fx_sub(z, a);
    m = z;
  }
  int top = -1;
  for (int i = L - 1; i >= 0 && top < 0; --i) {
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
  if (s && q + 1 < L) bits |= m.w[q + 1] << (64 - s);
  double d = (double)bits;  // one rounding to nearest
#if defined(__CUDA_ARCH__)
  d = scalbn(d, lo - 32 * L);
#else
  d = __builtin_scalbn(d, lo - 32 * L);
#endif
  return neg ? -d : d;
}

// Value as hi + lo (lo = rounded remainder after removing hi exactly).
template <int L>
__host__ __device__ inline void fx_to_dd(const FxW<L> &a, double &hi, double &lo) {
  hi = fx_to_double(a);
  FxW<L> r = a, h;
  const double ah = hi < 0 ? -hi : hi;
  if (ah != 0.0 && fx_from_pos_double(ah, h)) {
    if (hi > 0) fx_sub(r, h); else fx_add(r, h);
    lo = fx_to_double(r);
  } else {
    lo = 0.0;
  }
}

}  // namespace tor
