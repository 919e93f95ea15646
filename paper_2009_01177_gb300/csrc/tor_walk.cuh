// tor_walk.cuh -- per-chunk walk and result conversion shared by the single,
// sharded and batched kernels.
#pragma once
#include "tor_dfs.cuh"
#include "tor_internal.h"

namespace tor {

// B = I - O entries as the tier's type, from the prepped mode-interleaved matrix
// (diagonal rounded in B, its exact remainder in Blo)
struct SrcPrepped {
  const double *__restrict__ B;
  const double *__restrict__ Blo;
  int n2k;
  template <class Tier>
  __device__ __forceinline__ typename Tier::T get(int row, int col) const {
    return Tier::from_hilo(B[(size_t)row * n2k + col], (row == col) ? Blo[row] : 0.0);
  }
};

// B = I - O entries straight from the caller's O (xxpp or xpxp, leading dim ld)
struct SrcDirect {
  const double *__restrict__ O;
  int k, ld, layout;
  __device__ __forceinline__ double o(int row, int col) const {
    const int ri = layout == 0 ? ((row & 1) * k + (row >> 1)) : row;
    const int rj = layout == 0 ? ((col & 1) * k + (col >> 1)) : col;
    return O[(size_t)ri * ld + rj];
  }
  template <class Tier>
  __device__ __forceinline__ typename Tier::T get(int row, int col) const {
    return Tier::from_o(o(row, col), row == col);
  }
};

// B = I - O_S entries for a click pattern S of the full M-mode matrix O (xxpp,
// leading dim ld): local mode m is the m-th clicked mode gm[m], whose x and p
// rows are gm[m] and M + gm[m] (the selection rule under Eq. 1)
struct SrcPattern {
  const double *__restrict__ O;
  int M, ld;
  const unsigned char *gm;
  __device__ __forceinline__ double o(int row, int col) const {
    const int gr = (row & 1) * M + gm[row >> 1];
    const int gc = (col & 1) * M + gm[col >> 1];
    return O[(size_t)gr * ld + gc];
  }
  template <class Tier>
  __device__ __forceinline__ typename Tier::T get(int row, int col) const {
    return Tier::from_o(o(row, col), row == col);
  }
};

// One chunk: the subsets whose high modes r1..k-1 are fixed by the bits of c.
// Root: gather B over the fixed modes then the low modes into the thread's
// stack S and eliminate the fixed modes in place; then the depth-first walk.
template <class Tier, class Src>
__device__ __forceinline__ void walk_chunk(const Src &src, int k, int r1, unsigned long long c, double *S,
                                           size_t st, SumsOf<typename Tier::Acc> &Sm, double *Q, size_t sq) {
  using T = typename Tier::T;
  unsigned char pm[64];
  int np = 0;
  for (unsigned long long m = c; m; m &= m - 1) pm[np++] = (unsigned char)(r1 + __ffsll((long long)m) - 1);
  const int n = np + r1;
  for (int hi = 0; hi < 2 * n; ++hi) {
    const int ph = n - 1 - (hi >> 1), qh = 1 - (hi & 1);
    const int mh = (ph < np) ? pm[ph] : (ph - np);
    for (int lo = 0; lo <= hi; ++lo) {
      const int pl = n - 1 - (lo >> 1), ql = 1 - (lo & 1);
      const int ml = (pl < np) ? pm[pl] : (pl - np);
      Tier::stv(S, ix(hi, lo), st, src.template get<Tier>(2 * mh + qh, 2 * ml + ql));
    }
  }
  T t = Tier::one();
  for (int s = 0; s < np; ++s) {
    const int rp = n - 1 - s;
    const T a = Tier::ld(S, ix(2 * rp + 1, 2 * rp + 1), st);
    const T b = Tier::ld(S, ix(2 * rp + 1, 2 * rp), st);
    const T d = Tier::ld(S, ix(2 * rp, 2 * rp), st);
    const T det2 = Tier::det2(a, b, d, Sm.flags);
    if (Tier::bad(det2) || Tier::bad(a)) Sm.flags |= ST_NOTPD;
    const T y = Tier::rsqrt(det2, Sm.flags);
    t = Tier::mul(t, y, Sm.flags);
    if (rp > 0) schur_mem<Tier>(S, st, S, st, rp, a, b, d, y, Sm.flags);
  }
  Tier::acc(Sm, t, ((k ^ np) & 1) != 0);
  dfs_walk<Tier>(S, st, r1, t, np, k, Sm, Q, sq);
}

// Two L-limb fixed-point sums (signed sum, sum_abs; L/2 fraction limbs) ->
// tor_result with the tier's error model
template <int L>
__host__ __device__ inline void fixed_to_result_w(const unsigned long long *w, int k, int tier, int status,
                                                  tor_result *out) {
  FxW<L> a, b;
  for (int i = 0; i < L; ++i) { a.w[i] = w[i]; b.w[i] = w[L + i]; }
  double hi, lo;
  fx_to_dd(a, hi, lo);
  out->hi = hi;
  out->lo = lo;
  out->sum_abs = fx_to_double(b);
  out->err_est = err_gamma(k) * unit_roundoff(tier) * out->sum_abs;
  out->tier = tier;
  out->status = (status & ST_NOTPD) ? TOR_ENOTPD : ((status & ST_RANGE) ? TOR_EINVAL : TOR_OK);
}

// limbs of one partial (signed sum and sum_abs) for a tier: 8 (256-bit sums,
// 128 fraction bits), or 16 for the 256-bit-class tier (512-bit sums, 256)
__host__ __device__ inline int partial_limbs(int tier) { return tier == TOR_PREC_FX256 ? 16 : 8; }

__host__ __device__ inline void fixed_to_result(const unsigned long long *w, int k, int tier, int status,
                                                tor_result *out) {
  if (tier == TOR_PREC_FX256) fixed_to_result_w<8>(w, k, tier, status, out);
  else fixed_to_result_w<4>(w, k, tier, status, out);
}

}  // namespace tor
