// tor_dfs.cuh -- depth-first subset walk for the Torontonian (Eq. 2).
//
// Work split (Algorithm 1's balanced partition, GB300 form): the 2^k subset
// masks are cut into 2^d equal chunks; chunk c fixes the membership of the
// high modes r1..k-1 (r1 = k - d) by the bits of c and enumerates every subset
// of the low modes 0..r1-1, i.e. the masks [c 2^r1, (c+1) 2^r1).  One thread
// owns one chunk at a time, so all lanes of a warp walk trees of the same
// shape in lock step.
//
// Per chunk:
//  1. Chunk root (the GENAZ step of the paper's kernel list, Sec. 7.1): gather
//     B = I - O over the chunk's fixed modes P0 followed by the low modes and
//     eliminate the P0 modes; what remains is the Schur complement
//     S_P0 = B_RR - B_RP0 B_P0^-1 B_P0R over the low modes, and
//     t_P0 = 1/sqrt(det B_P0) (product of the 2x2 pivot-block factors).
//  2. Depth-first walk over the prefix tree of subsets of the low modes.  A
//     node Q holds the Schur complement of B_Q over the modes after max(Q).
//     Its child Q+{c} needs only the 2x2 block of mode c:
//        det B_{Q+c} = det B_Q * det S_Q[c,c],   t_{Q+c} = t_Q / sqrt(det S_Q[c,c]),
//     and the grandchildren need the rank-2 update
//        S_{Q+c} = S_Q[>c,>c] - S_Q[>c,c] S_Q[c,c]^-1 S_Q[c,>c].
//     So each subset's factor extends its parent's by one appended block row
//     (the elimination of Sec. 4.2, done once per tree edge instead of once
//     per subset), costing about 20 FMA per subset on average instead of
//     O(k^3).
//
// Storage: a symmetric 2r x 2r matrix is kept as its lower triangle in
// REVERSED packed order: with reversed indices p = 2r-1-i, q = 2r-1-j and
// p >= q, entry (i, j) lives at p(p+1)/2 + q.  Mode m (0-based, of r) owns
// rows 2m (x) and 2m+1 (p), i.e. reversed rows 2(r-1-m)+1 and 2(r-1-m).  The
// trailing block after dropping or eliminating the first modes is then a
// PREFIX of the storage with the same formula, and every offset an update
// touches depends only on the child's size rp (number of modes after c):
//   pivot block   a = (2rp+1, 2rp+1)  b = (2rp+1, 2rp)  d = (2rp, 2rp)
//   pivot columns u_x[i] = (2rp+1, i), u_p[i] = (2rp, i),  i < 2rp
//   child entries (i, j), j <= i < 2rp  -> offsets [0, rp(2rp+1))
// The last child (rp = r-1) therefore overwrites its parent in place.
//
// Three storage tiers: subtrees of at most RREG modes are fully unrolled in
// registers; larger nodes live in a per-thread stack in global memory laid
// out entry-major ([entry][thread]) so that a warp's accesses coalesce.
//
// Accumulation: each t_Z goes exactly into 256-bit fixed point (fixacc.cuh),
// so the alternating sum adds no rounding error and no FP64 work.
#pragma once
#include <cstdint>
#include "fixacc.cuh"
#include "dd.cuh"
#include "fx128.cuh"

namespace tor {

__host__ __device__ constexpr int sz(int r) { return r * (2 * r + 1); }
__host__ __device__ constexpr int ix(int hi, int lo) { return hi * (hi + 1) / 2 + lo; }

// status bits written by the kernels
enum : int { ST_NOTPD = 1, ST_RANGE = 2 };  // ST_RANGE also marks fixed-point overflow

// ----------------------------------------------------------- accumulators
template <class A>
struct SumsOf {
  A tor;   // sum of (-1)^(k-|Z|) t_Z
  A sabs;  // sum of t_Z
  int flags;
};
using Sums = SumsOf<Fx256>;

// acc += (neg ? -|x| : |x|); tiny magnitudes (< 2^-75) are dropped (their
// contribution is far below any result's resolution); x must be finite.
__device__ __forceinline__ void fx_add_signed(Fx256 &acc, double x, bool neg, int &flags) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const bool xneg = (bits >> 63) != 0ull;
  bits &= 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(bits >> 52);
  if (e < 947) return;                      // zero or below 2^-75
  Fx256 X;
  if (!fx_from_pos_double(__longlong_as_double((long long)bits), X)) { flags |= ST_RANGE; return; }
  if (neg != xneg) fx_sub(acc, X); else fx_add(acc, X);
}

// ------------------------------------------------------- FP64 primitives
// Tuning switches (compile time).  Defaults are the fastest measured on GB300
// for the k = 32 workload: larger register subtrees, unrolled memory-tier
// updates and the FP32-seeded reciprocal square root each cut FP64 instructions
// but lengthen dependency chains or code; with the FP64 pipe about 2/3 busy,
// the added latency costs more than the saved issue slots.
#ifndef TOR_F64_RREG
#define TOR_F64_RREG 3
#endif
#ifndef TOR_F64_RUNROLL
#define TOR_F64_RUNROLL 0
#endif
#ifndef TOR_RSQRT_DF
#define TOR_RSQRT_DF 0
#endif
#ifndef TOR_RSQRT_CUBIC
#define TOR_RSQRT_CUBIC 1
#endif
// the seed of the reciprocal square root: 2 = the FP64 approximation
// instruction (measured max relative error 2^-20.05 over [2^-60, 2^60)),
// 1 = the FP32 one with x and the seed moved between FP64 and FP32 by exponent
// rebias on the bit patterns, 0 = the FP32 one with conversion instructions.
// Taking the FP64<->FP32 conversions out of the pivot's dependency chain pays
// on GB300: 0 measured 291.9 ms for the k = 32 FP64 walk, 1 275.2 ms and
// 2 273.9 ms.
#ifndef TOR_RSQRT_SEED
#define TOR_RSQRT_SEED 2
#endif
// Nodes of at most RSMEM modes live in one shared-memory slot per thread.  A
// node of r <= RREG + 2 modes has only register-resident children and its
// last child, which it overwrites in place, so one slot is enough.
#ifndef TOR_F64_RSMEM
#define TOR_F64_RSMEM 5
#endif
#ifndef TOR_DD_RSMEM
#define TOR_DD_RSMEM 3
#endif
#ifndef TOR_F64_MINB
#define TOR_F64_MINB 1
#endif
// double-double: one-mode register subtrees and three resident blocks (168
// registers) beat two-mode subtrees at two blocks (186) by 23-29 % at k = 28-30
#ifndef TOR_DD_MINB
#define TOR_DD_MINB 3
#endif
#ifndef TOR_DD_RREG
#define TOR_DD_RREG 1
#endif
// The fixed-point tier: 128-bit products are register-hungry (254 registers
// with two-mode register subtrees, so two resident blocks), so its register
// subtrees hold one mode and the kernel is compiled for four resident blocks
// (128 registers): 2.5x faster at k = 28..32 on GB300.
#ifndef TOR_FX_RREG
#define TOR_FX_RREG 1
#endif
#ifndef TOR_FX_RSMEM
#define TOR_FX_RSMEM 3
#endif
#ifndef TOR_FX_MINB
#define TOR_FX_MINB 4
#endif
__device__ __forceinline__ double dmul(double a, double b) { return a * b; }

// Which FP64 multiplies of the FP64 walk run on the integer pipes (dmul_i,
// below) instead of the FP64 pipe, as a bit mask: 1 = the two products of each
// pivot row v = S_cc^-1 u, 2 = the pivot coefficients S_cc^-1, 4 = the term
// t y.  GB300 issues 2 FP64 operations per clock per SM but 64 integer ones,
// so a multiply in about 40 integer instructions takes the SM about as long
// as the native one, on pipes the walk otherwise leaves idle.  Measured on the
// k = 32 walk, with bit-identical results: 0 (default) 273.2 ms, 1 336.0 ms,
// 2 314.1 ms, 3 437.8 ms, 7 521.9 ms.  The walk has few warps per SM, and the
// longer dependency chains cost more than the FP64 issue slots they free.
#ifndef TOR_F64_IMUL
#define TOR_F64_IMUL 0
#endif

// a * b rounded to nearest even, computed with integer instructions: IEEE 754
// binary64 multiplication of the significands (53 x 53 -> 106 bits from four
// 32 x 32 -> 64-bit products), normalised by one place and rounded on the
// dropped bits.  Operands or results outside the normal range (zero,
// subnormal, infinite, NaN, or an exponent that could overflow or underflow)
// take the FP64 multiply, so the result is bit-identical to a * b everywhere.
__device__ __forceinline__ double dmul_i(double a, double b) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const int ea = (int)(ua >> 52) & 0x7FF, eb = (int)(ub >> 52) & 0x7FF;
  const int e0 = ea + eb - 1023;  // the result's biased exponent, before normalisation
  if ((unsigned)(ea - 1) >= 2046u || (unsigned)(eb - 1) >= 2046u || (unsigned)(e0 - 1) >= 2044u) return a * b;
  const unsigned long long ma = (ua & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long mb = (ub & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned a0 = (unsigned)ma, a1 = (unsigned)(ma >> 32), b0 = (unsigned)mb, b1 = (unsigned)(mb >> 32);
  const unsigned long long p00 = (unsigned long long)a0 * b0;
  const unsigned long long mid = (unsigned long long)a0 * b1 + (unsigned long long)a1 * b0;  // < 2^54
  const unsigned long long lo = p00 + (mid << 32);
  const unsigned long long hi = (unsigned long long)a1 * b1 + (mid >> 32) + (lo < p00 ? 1ull : 0ull);
  // P = hi 2^64 + lo in [2^104, 2^106): keep its top 53 bits
  const int top = (int)(hi >> 41);  // 1 when P >= 2^105
  const int s = 52 + top;
  const unsigned long long m = (hi << (64 - s)) | (lo >> s);  // in [2^52, 2^53)
  const unsigned long long rem = lo & ((1ull << s) - 1ull), half = 1ull << (s - 1);
  const unsigned long long up = (rem + (m & 1ull) > half) ? 1ull : 0ull;  // nearest, ties to even
  // the implicit bit of m adds one to the exponent field, and a rounding carry
  // out of m (m + up = 2^53) moves on into it
  const unsigned long long r = ((unsigned long long)(e0 + top - 1) << 52) + m + up;
  return __longlong_as_double((long long)(r | ((ua ^ ub) & 0x8000000000000000ull)));
}

// 1/sqrt(x) for a positive double x, accurate to about one ulp.
// Default: a seed of at least 20 bits (TOR_RSQRT_SEED) and one third-order
// FP64 step (two FP64 multiplies and three FMAs, against two and four for two
// Newton steps y <- y + y (1/2 - (x/2) y^2), the TOR_RSQRT_CUBIC=0
// alternative; 3% faster walk at k = 32).  From a seed with relative error
// 2^-20 the step's truncation error (5/16) e^3, e = 1 - x y^2 < 2^-18.9, stays
// below 2^-58.  With TOR_RSQRT_DF, the seed comes instead
// from a double-float step: x is split EXACTLY into two floats by integer operations on its bit
// pattern, x = xh + xl (xh = the top 24 mantissa bits); one Newton step
// y1 = y0 + y0 e / 2, e = 1 - x y0^2, is taken in FP32 arithmetic with the
// products kept exact by FMA (TwoProd), giving ~45 correct bits as y0 + c.
// Then one FP64 Newton step y <- y + y (1/2 - (x/2) y^2) doubles that past
// 53 bits.  FP64 pipe cost: one add and three FMA-type operations, against
// six for two FP64 Newton steps from a 23-bit seed.  Inputs outside
// [2^-74, 2^100) take two FP64 Newton steps from the FP64 approximation.
__device__ __forceinline__ double rsqrt_fp64(double x) {
  const long long bx = __double_as_longlong(x);
  const int ex = (int)(bx >> 52);  // biased exponent, x > 0
  const double hx = __longlong_as_double(bx - (1ll << 52));  // x / 2, exact for normal x
  double y;
  if (TOR_RSQRT_DF && ex >= 949 && ex < 1123) {  // x in [2^-74, 2^100): both halves are normal floats
    const unsigned long long m = ((unsigned long long)bx & 0xFFFFFFFFFFFFFull);  // 52 fraction bits
    const float xh = __int_as_float(((ex - 1023 + 127) << 23) | (int)(m >> 29));
    const float xl = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull)) *
                     __int_as_float((ex - 1075 + 127) << 23);
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(xh));
    const float ph = y0 * y0, pl = fmaf(y0, y0, -ph);      // y0^2 = ph + pl exactly
    const float q = xh * ph, ql = fmaf(xh, ph, -q);        // xh ph = q + ql exactly
    const float e = (1.0f - q) - (ql + fmaf(xh, pl, xl * ph));
    const float c = (0.5f * y0) * e;
    y = (double)y0 + (double)c;
    const double r = fma(-dmul(hx, y), y, 0.5);
    y = fma(y, r, y);
  } else {  // the seed (out of float range: the FP64 approximation), then the FP64 step(s)
    if (TOR_RSQRT_SEED == 2) {
      asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    } else if (TOR_RSQRT_SEED == 1 && ex >= 1023 - 99 && ex <= 1023 + 99) {
      // x -> float and the float seed -> double by exponent rebias on the bit
      // patterns (x's mantissa truncated to 23 bits), integer operations only
      const float xf = __int_as_float((int)(((unsigned long long)bx >> 29) - (896ull << 23)));
      float yf;
      asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
      y = __longlong_as_double(((long long)(unsigned)__float_as_int(yf) << 29) + (896ll << 52));
    } else if (TOR_RSQRT_SEED == 0 && __double2float_rn(x) > 1e-30f && __double2float_rn(x) < 1e30f) {
      const float xf = __double2float_rn(x);
      float yf;
      asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
      y = (double)yf;
    } else {
      asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    }
    if (TOR_RSQRT_CUBIC) {
      // one third-order step: with e = 1 - x y^2, x^-1/2 = y (1 - e)^-1/2 =
      // y (1 + e/2 + 3 e^2/8 + O(e^3)) by the binomial series; from a seed of
      // relative error d <= 2^-20, |e| <= 2d + d^2 < 2^-18.9 and the truncation
      // error is about (5/16) |e|^3 < 2^-58, below FP64 rounding
      const double e = fma(-dmul(x, y), y, 1.0);
      const double p = fma(e, 0.375, 0.5);
      y = fma(dmul(y, e), p, y);
    } else {
      double r = fma(-dmul(hx, y), y, 0.5);
      y = fma(y, r, y);
      r = fma(-dmul(hx, y), y, 0.5);
      y = fma(y, r, y);
    }
  }
  return y;
}

// ------------------------------------------------------------ FP64 tier
struct TierF64 {
  using T = double;
  static constexpr int W = 1;      // doubles per stored entry
  static constexpr int RREG = TOR_F64_RREG;       // register-resident subtree size (modes)
  static constexpr int RUNROLL = TOR_F64_RUNROLL; // memory-tier updates unrolled up to this child size
  static constexpr int RSMEM = TOR_F64_RSMEM;     // shared-memory node size (modes), <= RREG + 2
  static constexpr int MINB = TOR_F64_MINB;       // __launch_bounds__ minimum blocks per SM
  static constexpr int PREC = 1;                  // TOR_PREC_FP64
  using Acc = Fx256;                              // exact accumulator of the terms

  __device__ static __forceinline__ T ld(const double *P, int e, size_t st) { return P[(size_t)e * st]; }
  __device__ static __forceinline__ void stv(double *P, int e, size_t st, T v) { P[(size_t)e * st] = v; }
  __device__ static __forceinline__ T one() { return 1.0; }
  __device__ static __forceinline__ T det2(T a, T b, T d, int &) { return fma(a, d, -dmul(b, b)); }
  // not (0 < x < inf): integer test on the bit pattern, no FP64 compare
  __device__ static __forceinline__ bool bad(T x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u - 1ull) >= 0x7FEFFFFFFFFFFFFFull;
  }
  __device__ static __forceinline__ T rsqrt(T x, int &) { return rsqrt_fp64(x); }
  __device__ static __forceinline__ T mul(T a, T b, int &) { return (TOR_F64_IMUL & 4) ? dmul_i(a, b) : dmul(a, b); }
  // pivot coefficients: S_cc^-1 = [[al, -be], [-be, de]] with inv = y^2 = 1/det2
  __device__ static __forceinline__ void coef(T a, T b, T d, T y, T &al, T &be, T &de, int &) {
    if (TOR_F64_IMUL & 2) {
      const T inv = dmul_i(y, y);
      al = dmul_i(d, inv); be = dmul_i(b, inv); de = dmul_i(a, inv);
    } else {
      const T inv = dmul(y, y);
      al = dmul(d, inv); be = dmul(b, inv); de = dmul(a, inv);
    }
  }
  // v = S_cc^-1 u
  __device__ static __forceinline__ void vrow(T al, T be, T de, T ux, T up, T &vx, T &vp, int &) {
    if (TOR_F64_IMUL & 1) {
      vx = fma(al, ux, -dmul_i(be, up));
      vp = fma(de, up, -dmul_i(be, ux));
    } else {
      vx = fma(al, ux, -dmul(be, up));
      vp = fma(de, up, -dmul(be, ux));
    }
  }
  __device__ static __forceinline__ T upd(T s, T vx, T ux, T vp, T up, int &) {
    return fma(-vp, up, fma(-vx, ux, s));
  }
  // entries of B = I - O: from the prepped (rounded 1 - o, exact low part) pair, or from o
  __device__ static __forceinline__ T from_hilo(double h, double) { return h; }
  __device__ static __forceinline__ T from_o(double o, bool diag) { return diag ? 1.0 - o : -o; }
  __device__ static __forceinline__ void acc(Sums &S, T t, bool neg) {
    fx_add_signed(S.tor, t, neg, S.flags);
    fx_add_signed(S.sabs, t, false, S.flags);
  }
};

// ------------------------------------------------------ double-double tier
struct TierDD {
  using T = dd;
  static constexpr int W = 2;
  static constexpr int RREG = TOR_DD_RREG;
  static constexpr int RUNROLL = 4;
  static constexpr int RSMEM = TOR_DD_RSMEM;
  static constexpr int MINB = TOR_DD_MINB;
  static constexpr int PREC = 2;  // TOR_PREC_DD
  using Acc = Fx256;

  __device__ static __forceinline__ T ld(const double *P, int e, size_t st) {
    return {P[(size_t)(2 * e) * st], P[(size_t)(2 * e + 1) * st]};
  }
  __device__ static __forceinline__ void stv(double *P, int e, size_t st, T v) {
    P[(size_t)(2 * e) * st] = v.hi;
    P[(size_t)(2 * e + 1) * st] = v.lo;
  }
  __device__ static __forceinline__ T one() { return {1.0, 0.0}; }
  __device__ static __forceinline__ T det2(T a, T b, T d, int &) { return dd_det2(a, b, d); }
  __device__ static __forceinline__ bool bad(T x) { return TierF64::bad(x.hi); }
  __device__ static __forceinline__ T rsqrt(T x, int &) { return dd_rsqrt(x, rsqrt_fp64(x.hi)); }
  __device__ static __forceinline__ T mul(T a, T b, int &) { return dd_mul(a, b); }
  __device__ static __forceinline__ void coef(T a, T b, T d, T y, T &al, T &be, T &de, int &) {
    const T inv = dd_mul(y, y);
    al = dd_mul(d, inv); be = dd_mul(b, inv); de = dd_mul(a, inv);
  }
  __device__ static __forceinline__ void vrow(T al, T be, T de, T ux, T up, T &vx, T &vp, int &) {
    vx = dd_add(dd_mul(al, ux), dd_neg(dd_mul(be, up)));
    vp = dd_add(dd_mul(de, up), dd_neg(dd_mul(be, ux)));
  }
  __device__ static __forceinline__ T upd(T s, T vx, T ux, T vp, T up, int &) {
    return dd_rank2_update(s, vx, ux, vp, up);
  }
  __device__ static __forceinline__ T from_hilo(double h, double l) { return {h, l}; }
  __device__ static __forceinline__ T from_o(double o, bool diag) { return diag ? two_sum(1.0, -o) : dd{-o, 0.0}; }
  __device__ static __forceinline__ void acc(Sums &S, T t, bool neg) {
    fx_add_signed(S.tor, t.hi, neg, S.flags);
    fx_add_signed(S.tor, t.lo, neg, S.flags);
    fx_add_signed(S.sabs, t.hi, false, S.flags);
    fx_add_signed(S.sabs, t.lo, false, S.flags);
  }
};

// ------------------------------------------------- 128-bit fixed-point tier
// Values are 128-bit two's-complement integers with F fraction bits (one
// scale for the whole instance, Sec. 5.1-5.2), stored as two 64-bit words in
// the same 16-byte entries as the double-double tier.  The caller picks F so
// that every intermediate stays below 2^(126-F).  Products are the only
// rounding (toward zero, Sec. 5.1) and set ST_RANGE if they overflow.
template <int F>
struct TierFx {
  using T = fx;
  static constexpr int W = 2;
  static constexpr int RREG = TOR_FX_RREG;
  static constexpr int RUNROLL = 0;
  static constexpr int RSMEM = TOR_FX_RSMEM;
  static constexpr int MINB = TOR_FX_MINB;
  static constexpr int PREC = 3;  // TOR_PREC_FX128
  using Acc = Fx256;
  static constexpr int FRAC = F;
  static_assert(F >= 64 && F <= 124, "fraction bits");

  __device__ static __forceinline__ T ld(const double *P, int e, size_t st) {
    return {(unsigned long long)__double_as_longlong(P[(size_t)(2 * e) * st]),
            __double_as_longlong(P[(size_t)(2 * e + 1) * st])};
  }
  __device__ static __forceinline__ void stv(double *P, int e, size_t st, T v) {
    P[(size_t)(2 * e) * st] = __longlong_as_double((long long)v.lo);
    P[(size_t)(2 * e + 1) * st] = __longlong_as_double(v.hi);
  }
  __device__ static __forceinline__ T one() { return {0ull, 1ll << (F - 64)}; }
  // exact for 2^(53-F) <= |x| < 2^(126-F); smaller magnitudes lose their low bits
  __device__ static __forceinline__ T from_double(double x, int &fl) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return {0ull, 0ll};
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = e - 1075 + F;  // value = m 2^sh in units of 2^-F
    T r;
    if (sh >= 64) {
      if (sh + 53 > 127) fl |= ST_RANGE;
      r = {0ull, (long long)(m << (sh - 64))};
    } else if (sh > 0) {
      r = {m << sh, (long long)(m >> (64 - sh))};
    } else if (sh > -64) {
      r = {m >> (-sh), 0ll};
    } else {
      r = {0ull, 0ll};
    }
    return (bits >> 63) ? fx_neg(r) : r;
  }
  __device__ static __forceinline__ double to_double(const T &x) {
    const bool neg = x.hi < 0;
    const T m = neg ? fx_neg(x) : x;
    const double d = ((double)(unsigned long long)m.hi * 18446744073709551616.0 + (double)m.lo) *
                     __longlong_as_double((long long)(1023 - F) << 52);  // * 2^-F
    return neg ? -d : d;
  }
  __device__ static __forceinline__ T from_hilo(double h, double l) {
    int fl = 0;
    return fx_add(from_double(h, fl), from_double(l, fl));
  }
  __device__ static __forceinline__ T from_o(double o, bool diag) {
    int fl = 0;
    const T v = from_double(o, fl);
    return diag ? fx_sub(one(), v) : fx_neg(v);
  }
  __device__ static __forceinline__ T mul(T a, T b, int &fl) {
    int o = 0;
    const T r = fx_mul(a, b, F, o);
    if (o) fl |= ST_RANGE;
    return r;
  }
  __device__ static __forceinline__ T det2(T a, T b, T d, int &fl) { return fx_sub(mul(a, d, fl), mul(b, b, fl)); }
  __device__ static __forceinline__ bool bad(T x) { return x.hi < 0 || (x.hi == 0 && x.lo == 0ull); }
  // 1/sqrt(x): the FP64 pipe (idle in this tier) gives a ~53-bit seed, two fixed-point
  // Newton steps y <- y (3 - x y^2) / 2 take it to the full fraction width
  __device__ static __forceinline__ T rsqrt(T x, int &fl) {
    const double xd = to_double(x);
    T y = from_double(xd > 0.0 ? rsqrt_fp64(xd) : 0.0, fl);
    const T three = {0ull, 3ll << (F - 64)};
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const T e = fx_sub(three, mul(x, mul(y, y, fl), fl));
      const T p = mul(y, e, fl);
      y = {(p.lo >> 1) | ((unsigned long long)p.hi << 63), p.hi >> 1};  // / 2 (arithmetic shift)
    }
    return y;
  }
  __device__ static __forceinline__ void coef(T a, T b, T d, T y, T &al, T &be, T &de, int &fl) {
    const T inv = mul(y, y, fl);
    al = mul(d, inv, fl); be = mul(b, inv, fl); de = mul(a, inv, fl);
  }
  __device__ static __forceinline__ void vrow(T al, T be, T de, T ux, T up, T &vx, T &vp, int &fl) {
    vx = fx_sub(mul(al, ux, fl), mul(be, up, fl));
    vp = fx_sub(mul(de, up, fl), mul(be, ux, fl));
  }
  __device__ static __forceinline__ T upd(T s, T vx, T ux, T vp, T up, int &fl) {
    return fx_sub(fx_sub(s, mul(vx, ux, fl)), mul(vp, up, fl));
  }
  // t (F fraction bits, positive) into the 128-fraction-bit accumulators, exactly
  __device__ static __forceinline__ void acc(Sums &S, T t, bool neg) {
    if (t.hi < 0) { S.flags |= ST_RANGE; return; }
    const int sh = 128 - F;  // 4..64
    Fx256 X;
    const unsigned long long hi = (unsigned long long)t.hi;
    X.w[0] = (sh == 64) ? 0ull : (t.lo << sh);
    X.w[1] = (sh == 64) ? t.lo : ((hi << sh) | (t.lo >> (64 - sh)));
    X.w[2] = (sh == 64) ? hi : (hi >> (64 - sh));
    X.w[3] = 0ull;
    if (neg) fx_sub(S.tor, X); else fx_add(S.tor, X);
    fx_add(S.sabs, X);
  }
};

// ------------------------------------------------------ register subtrees
template <class Tier, int R>
struct RegNode;

// child of size RP (modes after the pivot) computed from a parent accessor
template <class Tier, int RP, class Get>
__device__ __forceinline__ void reg_child(const Get &get, typename Tier::T a, typename Tier::T b,
                                          typename Tier::T d, typename Tier::T y,
                                          typename Tier::T tc, int parc, int k, SumsOf<typename Tier::Acc> &S) {
  using T = typename Tier::T;
  int &FL = S.flags;
  T al, be, de;
  Tier::coef(a, b, d, y, al, be, de, FL);
  T ux[2 * RP], up[2 * RP];
#pragma unroll
  for (int i = 0; i < 2 * RP; ++i) {
    ux[i] = get(ix(2 * RP + 1, i));
    up[i] = get(ix(2 * RP, i));
  }
  T C[sz(RP)];
#pragma unroll
  for (int i = 0; i < 2 * RP; ++i) {
    T vx, vp;
    Tier::vrow(al, be, de, ux[i], up[i], vx, vp, FL);
#pragma unroll
    for (int j = 0; j <= i; ++j) C[ix(i, j)] = Tier::upd(get(ix(i, j)), vx, ux[j], vp, up[j], FL);
  }
  RegNode<Tier, RP>::visit(C, tc, parc, k, S);
}

template <class Tier, int R, int RP>
struct RegChildren {
  using T = typename Tier::T;
  __device__ static __forceinline__ void run(const T (&M)[sz(R)], T t, int par, int k, SumsOf<typename Tier::Acc> &S) {
    int &FL = S.flags;
    const T a = M[ix(2 * RP + 1, 2 * RP + 1)], b = M[ix(2 * RP + 1, 2 * RP)], d = M[ix(2 * RP, 2 * RP)];
    const T det2 = Tier::det2(a, b, d, FL);
    if (Tier::bad(det2) || Tier::bad(a)) S.flags |= ST_NOTPD;  // 2x2 block PD iff a > 0 and det > 0
    const T y = Tier::rsqrt(det2, FL);
    const T tc = Tier::mul(t, y, FL);
    Tier::acc(S, tc, ((k ^ (par + 1)) & 1) != 0);
    if constexpr (RP > 0) {
      auto get = [&](int e) { return M[e]; };
      reg_child<Tier, RP>(get, a, b, d, y, tc, par + 1, k, S);
    }
    RegChildren<Tier, R, RP + 1>::run(M, t, par, k, S);
  }
};
template <class Tier, int R>
struct RegChildren<Tier, R, R> {
  using T = typename Tier::T;
  __device__ static __forceinline__ void run(const T (&)[sz(R)], T, int, int, SumsOf<typename Tier::Acc> &) {}
};

template <class Tier, int R>
struct RegNode {
  using T = typename Tier::T;
  __device__ static __forceinline__ void visit(const T (&M)[sz(R)], T t, int par, int k, SumsOf<typename Tier::Acc> &S) {
    RegChildren<Tier, R, 0>::run(M, t, par, k, S);
  }
};

// memory parent -> register child of size rp (1..RREG)
template <class Tier>
__device__ __forceinline__ void mem_to_reg_child(int rp, const double *P, size_t st,
                                                 typename Tier::T a, typename Tier::T b,
                                                 typename Tier::T d, typename Tier::T y,
                                                 typename Tier::T tc, int parc, int k, SumsOf<typename Tier::Acc> &S) {
  auto get = [&](int e) { return Tier::ld(P, e, st); };
  if constexpr (Tier::RREG >= 1) { if (rp == 1) { reg_child<Tier, 1>(get, a, b, d, y, tc, parc, k, S); return; } }
  if constexpr (Tier::RREG >= 2) { if (rp == 2) { reg_child<Tier, 2>(get, a, b, d, y, tc, parc, k, S); return; } }
  if constexpr (Tier::RREG >= 3) { if (rp == 3) { reg_child<Tier, 3>(get, a, b, d, y, tc, parc, k, S); return; } }
  if constexpr (Tier::RREG >= 4) { if (rp == 4) { reg_child<Tier, 4>(get, a, b, d, y, tc, parc, k, S); return; } }
}

// ------------------------------------------------------- memory-tier update
// child C (size rp) = parent P's trailing block minus the rank-2 term; C may equal P.
// Looped form, for children larger than Tier::RUNROLL modes (rare).
template <class Tier>
__device__ __noinline__ void schur_mem_loop(const double *P, size_t sp, double *C, size_t sc, int rp,
                                            typename Tier::T a, typename Tier::T b,
                                            typename Tier::T d, typename Tier::T y, int &FL) {
  using T = typename Tier::T;
  T al, be, de;
  Tier::coef(a, b, d, y, al, be, de, FL);
  const int n2 = 2 * rp;
  const int cx = ix(2 * rp + 1, 0), cp = ix(2 * rp, 0);
  for (int i = 0; i < n2; ++i) {
    const T uxi = Tier::ld(P, cx + i, sp), upi = Tier::ld(P, cp + i, sp);
    T vx, vp;
    Tier::vrow(al, be, de, uxi, upi, vx, vp, FL);
    const int row = ix(i, 0);
#pragma unroll 4
    for (int j = 0; j <= i; ++j) {
      const T s = Tier::ld(P, row + j, sp);
      Tier::stv(C, row + j, sc, Tier::upd(s, vx, Tier::ld(P, cx + j, sp), vp, Tier::ld(P, cp + j, sp), FL));
    }
  }
}

// Unrolled form for a compile-time child size RP: the pivot columns stay in
// registers, so each child entry costs one load and one store.  P and C may
// be the same storage (the in-place last child); every entry is read before it
// is written and never read again, so no reordering of independent accesses
// can change the result, which is what the restrict qualifiers allow.
template <class Tier, int RP>
__device__ __forceinline__ void schur_mem_fixed(const double *__restrict__ P, size_t sp, double *__restrict__ C,
                                                size_t sc, typename Tier::T a, typename Tier::T b,
                                                typename Tier::T d, typename Tier::T y, int &FL) {
  using T = typename Tier::T;
  T al, be, de;
  Tier::coef(a, b, d, y, al, be, de, FL);
  T ux[2 * RP], up[2 * RP];
#pragma unroll
  for (int i = 0; i < 2 * RP; ++i) {
    ux[i] = Tier::ld(P, ix(2 * RP + 1, i), sp);
    up[i] = Tier::ld(P, ix(2 * RP, i), sp);
  }
#pragma unroll
  for (int i = 0; i < 2 * RP; ++i) {
    T vx, vp;
    Tier::vrow(al, be, de, ux[i], up[i], vx, vp, FL);
#pragma unroll
    for (int j = 0; j <= i; ++j)
      Tier::stv(C, ix(i, j), sc, Tier::upd(Tier::ld(P, ix(i, j), sp), vx, ux[j], vp, up[j], FL));
  }
}

template <class Tier, int RP>
__device__ __forceinline__ bool schur_try(int rp, const double *P, size_t sp, double *C, size_t sc,
                                          typename Tier::T a, typename Tier::T b,
                                          typename Tier::T d, typename Tier::T y, int &FL) {
  if constexpr (RP > Tier::RUNROLL) {
    return false;
  } else {
    if (rp == RP) { schur_mem_fixed<Tier, RP>(P, sp, C, sc, a, b, d, y, FL); return true; }
    return schur_try<Tier, RP + 1>(rp, P, sp, C, sc, a, b, d, y, FL);
  }
}

// one out-of-line copy of the dispatch, so the unrolled bodies exist once in
// the binary however many call sites there are (instruction-cache footprint)
template <class Tier>
__device__ __noinline__ void schur_mem(const double *P, size_t sp, double *C, size_t sc, int rp,
                                       typename Tier::T a, typename Tier::T b,
                                       typename Tier::T d, typename Tier::T y, int &FL) {
  if (!schur_try<Tier, Tier::RREG + 1>(rp, P, sp, C, sc, a, b, d, y, FL))
    schur_mem_loop<Tier>(P, sp, C, sc, rp, a, b, d, y, FL);
}

// per-thread stack extent (in entries) of a walk over r modes
__host__ __device__ constexpr int stack_entries(int r, int rreg) {
  int e = 0;
  for (int j = r; j > rreg; j -= 2) e += sz(j);
  return e;
}

// ------------------------------------------------------------ the walk
// Visit every non-empty extension of the node stored at S (r modes, term t,
// |Z| = par) in depth-first order; the node's own term is added by the caller.
// Q/sq: this thread's shared-memory slot (Tier::RSMEM nodes; may be null to
// keep every node in global memory).
template <class Tier>
__device__ void dfs_walk(double *S, size_t st, int r, typename Tier::T t, int par, int k, SumsOf<typename Tier::Acc> &Sm,
                         double *Q = nullptr, size_t sq = 0) {
  using T = typename Tier::T;
  // a shared-memory node's only child above RREG is its last one, written in place
  static_assert(Tier::RSMEM <= Tier::RREG + 2, "one shared-memory slot needs RSMEM <= RREG + 2");
  struct Frame { int off, r, rp, par; T t; };
  Frame stk[33];
  int sp = 0;
  int off = 0, rp = 0;
  int &FL = Sm.flags;
  bool insm = false;  // the current node lives in the shared-memory slot
  while (true) {
    if (rp < r) {
      const int cur = rp++;
      const double *P = insm ? Q : S + (size_t)(off * Tier::W) * st;
      const size_t ps = insm ? sq : st;
      const T a = Tier::ld(P, ix(2 * cur + 1, 2 * cur + 1), ps);
      const T b = Tier::ld(P, ix(2 * cur + 1, 2 * cur), ps);
      const T d = Tier::ld(P, ix(2 * cur, 2 * cur), ps);
      const T det2 = Tier::det2(a, b, d, FL);
      if (Tier::bad(det2) || Tier::bad(a)) Sm.flags |= ST_NOTPD;
      const T y = Tier::rsqrt(det2, FL);
      const T tc = Tier::mul(t, y, FL);
      Tier::acc(Sm, tc, ((k ^ (par + 1)) & 1) != 0);
      if (cur == 0) continue;
      if (cur <= Tier::RREG) {
        mem_to_reg_child<Tier>(cur, P, ps, a, b, d, y, tc, par + 1, k, Sm);
        continue;
      }
      if (Q && cur <= Tier::RSMEM) {  // into the shared-memory slot (in place when already there)
        schur_mem<Tier>(P, ps, Q, sq, cur, a, b, d, y, FL);
        if (!insm && cur != r - 1) stk[sp++] = Frame{off, r, rp, par, t};
        insm = true; r = cur; rp = 0; t = tc; par = par + 1;
        continue;
      }
      if (cur == r - 1) {  // last child: in place, the node is finished afterwards
        schur_mem<Tier>(P, st, const_cast<double *>(P), st, cur, a, b, d, y, FL);
        r = cur; rp = 0; t = tc; par = par + 1;
        continue;
      }
      const int coff = off + sz(r);
      schur_mem<Tier>(P, st, S + (size_t)(coff * Tier::W) * st, st, cur, a, b, d, y, FL);
      stk[sp++] = Frame{off, r, rp, par, t};
      off = coff; r = cur; rp = 0; t = tc; par = par + 1;
    } else {
      if (sp == 0) break;
      --sp;
      off = stk[sp].off; r = stk[sp].r; rp = stk[sp].rp; par = stk[sp].par; t = stk[sp].t;
      insm = false;
    }
  }
}

// shared-memory bytes a walk kernel needs per block: the per-thread slots, and
// at least the two accumulators per thread of the block's partial-sum reduction
template <class Tier>
__host__ __device__ constexpr size_t walk_smem_bytes(int threads) {
  const size_t slot = (size_t)sz(Tier::RSMEM) * Tier::W * sizeof(double);
  const size_t red = 2 * sizeof(typename Tier::Acc);
  return (slot > red ? slot : red) * (size_t)threads;
}

}  // namespace tor
