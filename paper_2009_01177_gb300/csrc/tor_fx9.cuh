// tor_fx9.cuh -- the 256-bit-class fixed-point walk (TOR_PREC_FX256).
//
// The same prefix-chunk depth-first walk as tor_dfs.cuh (Eq. 2 by incremental
// Schur complements along the prefix tree; the chunk root is the GENAZ step
// and each tree edge one elimination step of Sec. 4.2), in the paper's
// multiprecision fixed point (Sec. 5.1-5.2) with the fx9 arithmetic: nine
// 29-bit balanced limbs, 203 fraction bits.
//
// Written for the instruction cache: every multiprecision operation is one
// inlined copy in one loop (the chunk root's eliminations and the walk share
// the pivot step and the Schur update), so the hot code stays a few tens of
// KB; an earlier template-unrolled 256-bit walk was 290 KB of code and spent
// most of its cycles waiting for instructions.
//
// Node storage: a node of r modes is r(2r+1) entries in the reversed packed
// order of tor_dfs.cuh.  An entry is nine 32-bit limbs stored planar for
// 128-bit accesses: limbs 0-3 | limbs 4-7 | limb 8, each plane contiguous over
// the threads that share the layout ([entry][plane][thread]).  Nodes of at
// most FX9_RSMEM modes live in a per-thread stack in shared memory, larger
// ones in a per-thread stack in global memory.
//
// Accumulation: the signed terms go limb by limb into nine 64-bit column
// sums, the terms' top four limbs (2^-58 and up) into four more for the sum of
// terms; both fold exactly into 512-bit fixed point (256 fraction bits) at the
// end of a chunk.
#pragma once
#include <cstdint>
#include "fx9.cuh"
#include "fixacc.cuh"
#include "tor_dfs.cuh"
#include "tor_walk.cuh"

namespace tor {

#ifndef FX9_RSMEM
#define FX9_RSMEM 2
#endif
#ifndef FX9_MINB
#define FX9_MINB 3
#endif
// 1: the three coefficient products and the two pivot-row products each
// share one inlined copy (operands selected per pass): about 75 KB of code
// against 81 KB, 1853.8 against 1862.5 ms for the k = 32 walk; 0: one copy
// per product
#ifndef FX9_COMPACT
#define FX9_COMPACT 1
#endif
// the reciprocal square root's seed: 1 = double-double (about 100 bits) and
// one fixed-point Newton step (2.28 G subset-dets/s at k = 32), 0 = FP64 and
// two steps (2.20)
#ifndef FX9_DDSEED
#define FX9_DDSEED 1
#endif
// 1: the walk kernels keep each chunk's column sums in shared memory
// (Fx9SumsShared) instead of 26 registers: spills 176 -> 20 bytes, the k = 32
// walk 1808.0 -> 1759.3 ms and an fx256 batch 2.35 -> 2.41 G subset-dets/s,
// same bits; 0: in registers (Fx9Sums)
#ifndef FX9_SUMS_SMEM
#define FX9_SUMS_SMEM 1
#endif

// entries of the shared-memory mini-stack: a node of RSMEM modes and the chain
// of its largest non-last descendants (RSMEM - 2, RSMEM - 4, ...)
__host__ __device__ constexpr int fx9_smem_entries(int rs) {
  int e = 0;
  for (int j = rs; j > 0; j -= 2) e += sz(j);
  return e;
}

// planar node storage shared by `st` threads (st a multiple of 4)
struct Fx9Mem {
  char *base;
  unsigned st, tid;
  __device__ __forceinline__ char *at(int e) const { return base + (size_t)e * 36u * st; }
  __device__ __forceinline__ fx9 ld(int e) const {
    const char *p = at(e);
    const int4 a = *reinterpret_cast<const int4 *>(p + 16u * tid);
    const int4 b = *reinterpret_cast<const int4 *>(p + 16u * st + 16u * tid);
    const int c = *reinterpret_cast<const int *>(p + 32u * st + 4u * tid);
    return fx9{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c}};
  }
  __device__ __forceinline__ void stv(int e, const fx9 &v) const {
    char *p = at(e);
    *reinterpret_cast<int4 *>(p + 16u * tid) = make_int4(v.l[0], v.l[1], v.l[2], v.l[3]);
    *reinterpret_cast<int4 *>(p + 16u * st + 16u * tid) = make_int4(v.l[4], v.l[5], v.l[6], v.l[7]);
    *reinterpret_cast<int *>(p + 32u * st + 4u * tid) = v.l[8];
  }
};

// per-thread sums of the walk: signed terms in nine column sums (2^(29 m - 203)),
// the sum of terms in four (limbs 5..8 of each term)
struct Fx9Sums {
  long long tor[9];
  long long sabs[4];
  int flags;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int m = 0; m < 9; ++m) tor[m] = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) sabs[m] = 0;
    flags = 0;
  }
  __device__ __forceinline__ void add(const fx9 &t, bool neg) {
#pragma unroll
    for (int m = 0; m < 9; ++m) tor[m] += neg ? -(long long)t.l[m] : (long long)t.l[m];
#pragma unroll
    for (int m = 0; m < 4; ++m) sabs[m] += t.l[m + 5];
  }
  __device__ __forceinline__ long long tor_col(int m) const { return tor[m]; }
  __device__ __forceinline__ long long sabs_col(int m) const { return sabs[m]; }
};

// The same column sums in shared memory, [column][thread] with stride st.
// Each thread owns its columns (plain loads and stores), and the 26 registers
// the sums would hold stay free for the walk.
struct Fx9SumsShared {
  long long *s;  // this thread's column 0
  unsigned st;
  int flags;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int m = 0; m < 13; ++m) s[m * st] = 0;
    flags = 0;
  }
  __device__ __forceinline__ void add(const fx9 &t, bool neg) {
#pragma unroll
    for (int m = 0; m < 9; ++m) s[m * st] += neg ? -(long long)t.l[m] : (long long)t.l[m];
#pragma unroll
    for (int m = 0; m < 4; ++m) s[(9 + m) * st] += t.l[m + 5];
  }
  __device__ __forceinline__ long long tor_col(int m) const { return s[m * st]; }
  __device__ __forceinline__ long long sabs_col(int m) const { return s[(9 + m) * st]; }
};

// column sums -> 512-bit two's complement with 256 fraction bits, exactly:
// the column of weight 2^(29 m - 203) is the 64-bit signed value shifted left
// by 29 m + 53 bits
__device__ __forceinline__ void fx9_fold_col(Fx512 &x, long long v, int shift) {
  Fx512 y;
  const int q = shift >> 6, s = shift & 63;
  const unsigned long long u = (unsigned long long)v, sx = (v < 0) ? ~0ull : 0ull;
  const unsigned long long lo = u << s, hi = s ? ((u >> (64 - s)) | (sx << s)) : sx;
#pragma unroll
  for (int i = 0; i < 8; ++i) y.w[i] = (i < q) ? 0ull : (i == q) ? lo : (i == q + 1) ? hi : sx;
  fx_add(x, y);
}

template <class Sums>
static __device__ __noinline__ void fx9_fold(const Sums &S, Fx512 &tor_out, Fx512 &sabs_out) {
  fx_zero(tor_out);
  fx_zero(sabs_out);
#pragma unroll 1
  for (int m = 0; m < 9; ++m) fx9_fold_col(tor_out, S.tor_col(m), 29 * m + 53);
#pragma unroll 1
  for (int m = 0; m < 4; ++m) fx9_fold_col(sabs_out, S.sabs_col(m), 29 * (m + 5) + 53);
}

// B = I - O entries as normalised fx9, exactly (up to bits below 2^-203): from
// the prepped matrix (rounded value plus exact diagonal remainder), or from o
__device__ __forceinline__ fx9 fx9_entry(const SrcPrepped &src, int row, int col, int &ovf) {
  const double h = src.B[(size_t)row * src.n2k + col], l = (row == col) ? src.Blo[row] : 0.0;
  return fx9_add(fx9_from_double(h, ovf), fx9_from_double(l, ovf), ovf);
}
template <class Src>
__device__ __forceinline__ fx9 fx9_entry(const Src &src, int row, int col, int &ovf) {
  const double o = src.o(row, col);
  const fx9 v = fx9_from_double(o, ovf);
  return (row == col) ? fx9_sub(fx9_int(1), v, ovf) : fx9_sub(fx9_zero(), v, ovf);
}

// One chunk: the subsets whose high modes r1..k-1 are fixed by the bits of c.
// G: this thread's global stack (root and large nodes); Q: its shared-memory
// mini-stack.  Adds the chunk's terms to A (Fx9Sums or Fx9SumsShared).
template <class Src, class Sums>
__device__ void fx9_walk_chunk(const Src &src, int k, int r1, unsigned long long c, const Fx9Mem &G,
                               const Fx9Mem &Q, Sums &A) {
  int ovf = 0;
  // ---- gather B over the fixed modes P0 (in Z) followed by the low modes
  // the lanes that walk a chunk of the same depth r1 now (the same number of
  // loop iterations once padded below), and their largest number of fixed modes
  const unsigned lanes = __match_any_sync(__activemask(), r1);
  const int np_max = __reduce_max_sync(lanes, (unsigned)__popcll((long long)c));
  unsigned char pm[64];
  int np = 0;
  for (unsigned long long m = c; m; m &= m - 1) pm[np++] = (unsigned char)(r1 + __ffsll((long long)m) - 1);
  const int n = np + r1;
#pragma unroll 1
  for (int hi = 0; hi < 2 * n; ++hi) {
    const int ph = n - 1 - (hi >> 1), qh = 1 - (hi & 1);
    const int mh = (ph < np) ? pm[ph] : (ph - np);
#pragma unroll 1
    for (int lo = 0; lo <= hi; ++lo) {
      const int pl = n - 1 - (lo >> 1), ql = 1 - (lo & 1);
      const int ml = (pl < np) ? pm[pl] : (pl - np);
      G.stv(ix(hi, lo), fx9_entry(src, 2 * mh + qh, 2 * ml + ql, ovf));
    }
  }

  // ---- the walk; the first np steps eliminate the fixed modes in place
  struct Frame {
    int off, r, rp, par, insm;
    fx9 t;
  };
  Frame stk[33];
  int sp = 0;
  int off = 0, r = n, par = 0, skip = np;
  int rp = (np > 0) ? n - 1 : 0;  // while skip > 0 only the last child (the next fixed mode) is taken
  bool insm = false;
  fx9 t = fx9_int(1);
  if (np == 0) A.add(t, (k & 1) != 0);  // the empty subset
  const fx9 one = fx9_int(1);
  // Lanes of a warp walk trees of the same shape, but their chunks fix
  // different numbers of modes.  Each lane first idles for the difference to
  // the warp's largest count, so that every lane runs the same number of loop
  // iterations and the same tree position on each of them; the warp
  // synchronisation at the top of every iteration keeps the lanes together
  // (independent thread scheduling would otherwise let the idle lanes run
  // ahead, and a warp whose lanes sit at different tree positions executes
  // them one after the other: 10 of 32 lanes active on average, measured).
  int idle = np_max - np;
#pragma unroll 1
  while (true) {
    __syncwarp(lanes);
    if (idle > 0) {
      --idle;
      continue;
    }
    if (rp < r) {
      const int cur = rp++;  // the child keeps the cur modes after the pivot
      const Fx9Mem P = insm ? Fx9Mem{Q.at(off), Q.st, Q.tid} : Fx9Mem{G.at(off), G.st, G.tid};
      // pivot block of the child's mode and its determinant
      const fx9 a = P.ld(ix(2 * cur + 1, 2 * cur + 1));
      const fx9 b = P.ld(ix(2 * cur + 1, 2 * cur));
      const fx9 d = P.ld(ix(2 * cur, 2 * cur));
      const fx9 det2 = fx9_dot2(a, d, fx9_neg(b), b, ovf);
      const double xd = fx9_to_double(det2);
      if (!(xd > 0.0) || fx9_sign(a) <= 0) A.flags |= ST_NOTPD;  // 2x2 block PD iff a > 0, det > 0
#if FX9_DDSEED
      // y = det2^-1/2: a double-double seed of about 100 bits on the FP64 pipe
      // (det2 = xd + xl exactly to 2^-100, one double-double Newton step from
      // the FP64 reciprocal square root), then one fixed-point Newton step
      // y += (y/2)(1 - det2 y^2), whose error term has limbs 0..3 only
      fx9 y;
      {
        const double xl = fx9_to_double(fx9_sub(det2, fx9_from_double(xd, ovf), ovf));
        const double y0 = xd > 0.0 ? rsqrt_fp64(xd) : 0.0;
        const double ph = y0 * y0, pl = fma(y0, y0, -ph);
        const double qh = xd * ph, ql = fma(xd, ph, -qh);
        const double e0 = (1.0 - qh) - fma(xl, ph, fma(xd, pl, ql));
        y = fx9_add(fx9_from_double(y0, ovf), fx9_from_double((0.5 * y0) * e0, ovf), ovf);
        const fx9 y2 = fx9_mul(y, y, ovf);
        const fx9 e = fx9_fma(one, fx9_neg(det2), y2, ovf);
        if (e.l[4] | e.l[5] | e.l[6] | e.l[7] | e.l[8]) ovf = 1;  // the seed missed 2^-115: not a PD block
        long long col[11];
        fx9_init(col, y);
        fx9_columns_short<3>(col, fx9_half(y), e);
        y = fx9_carry(col, ovf);
      }
#else
      // y = det2^-1/2: FP64 seed, two Newton steps y += (y/2)(1 - det2 y^2)
      fx9 y = fx9_from_double(xd > 0.0 ? rsqrt_fp64(xd) : 0.0, ovf);
      const fx9 nx = fx9_neg(det2);
#pragma unroll 1
      for (int it = 0; it < 2; ++it) {
        const fx9 y2 = fx9_mul(y, y, ovf);
        const fx9 e = fx9_fma(one, nx, y2, ovf);
        y = fx9_fma(y, fx9_half(y), e, ovf);
      }
#endif
      const fx9 tc = fx9_mul(t, y, ovf);
      if (skip <= 1) A.add(tc, ((k ^ (par + 1)) & 1) != 0);
      if (cur > 0) {
        // S_child = S[<c] - u D^-1 u^T with D^-1 = inv [[d, -b], [-b, a]], inv = y^2
        const fx9 inv = fx9_mul(y, y, ovf);
        const fx9 ninv = fx9_neg(inv);
#if FX9_COMPACT
        // one inlined product for the three coefficients (operands chosen per pass)
        fx9 nal, nde, be;
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {
          fx9 x, w;
#pragma unroll
          for (int l = 0; l < 9; ++l) {
            x.l[l] = (q == 0) ? d.l[l] : (q == 1) ? a.l[l] : b.l[l];
            w.l[l] = (q == 2) ? inv.l[l] : ninv.l[l];
          }
          const fx9 pr = fx9_mul(x, w, ovf);
#pragma unroll
          for (int l = 0; l < 9; ++l) {
            nal.l[l] = (q == 0) ? pr.l[l] : nal.l[l];
            nde.l[l] = (q == 1) ? pr.l[l] : nde.l[l];
            be.l[l] = (q == 2) ? pr.l[l] : be.l[l];
          }
        }
#else
        const fx9 nal = fx9_mul(d, ninv, ovf), nde = fx9_mul(a, ninv, ovf), be = fx9_mul(b, inv, ovf);
#endif
        const bool last = (cur == r - 1) || skip > 0;
        Fx9Mem C;
        int coff, cins;
        if (insm) {  // shared-memory parent: last child in place, others above it
          coff = last ? off : off + sz(r);
          cins = 1;
        } else if (cur <= FX9_RSMEM && skip == 0) {  // into the shared-memory mini-stack
          coff = 0;
          cins = 1;
        } else {  // global parent: last child in place, others above it
          coff = last ? off : off + sz(r);
          cins = 0;
        }
        C = cins ? Fx9Mem{Q.at(coff), Q.st, Q.tid} : Fx9Mem{G.at(coff), G.st, G.tid};
        const int cx = ix(2 * cur + 1, 0), cp = ix(2 * cur, 0);
#pragma unroll 1
        for (int i = 0; i < 2 * cur; ++i) {
          const fx9 uxi = P.ld(cx + i), upi = P.ld(cp + i);
          // -v_i = -(D^-1 u_i): x part be up - al ux, p part be ux - de up
#if FX9_COMPACT
          fx9 nvx, nvp;
#pragma unroll 1
          for (int q = 0; q < 2; ++q) {
            fx9 u1, c2, u2;
#pragma unroll
            for (int l = 0; l < 9; ++l) {
              u1.l[l] = q ? uxi.l[l] : upi.l[l];
              c2.l[l] = q ? nde.l[l] : nal.l[l];
              u2.l[l] = q ? upi.l[l] : uxi.l[l];
            }
            const fx9 v = fx9_dot2(be, u1, c2, u2, ovf);
#pragma unroll
            for (int l = 0; l < 9; ++l) {
              nvx.l[l] = q ? nvx.l[l] : v.l[l];
              nvp.l[l] = q ? v.l[l] : nvp.l[l];
            }
          }
#else
          const fx9 nvx = fx9_dot2(be, upi, nal, uxi, ovf);
          const fx9 nvp = fx9_dot2(be, uxi, nde, upi, ovf);
#endif
          const int row = ix(i, 0);
#pragma unroll 1
          for (int j = 0; j <= i; ++j)
            C.stv(row + j, fx9_fma2(P.ld(row + j), nvx, P.ld(cx + j), nvp, P.ld(cp + j), ovf));
        }
        if (!last) stk[sp++] = Frame{off, r, rp, par, insm ? 1 : 0, t};
        off = coff;
        insm = cins != 0;
        r = cur;
        t = tc;
        par = par + 1;
        if (skip > 0) --skip;
        rp = (skip > 0) ? r - 1 : 0;
      } else if (skip > 0) {  // the last fixed mode leaves no low mode (r1 = 0)
        skip = 0;
        r = 0;
        rp = 0;
      }
    } else {
      if (sp == 0) break;
      --sp;
      off = stk[sp].off;
      r = stk[sp].r;
      rp = stk[sp].rp;
      par = stk[sp].par;
      insm = stk[sp].insm != 0;
      t = stk[sp].t;
    }
  }
  if (ovf) A.flags |= ST_RANGE;
}

// per-thread global stack extent in entries for chunks of r1 walked modes of a
// k-mode instance: the gathered root (up to k modes) or the chain of non-last
// children above FX9_RSMEM modes
__host__ __device__ constexpr int fx9_stack_entries(int k, int r1) {
  int e = 0;
  for (int j = r1; j > FX9_RSMEM; j -= 2) e += sz(j);
  return sz(k) > e ? sz(k) : e;
}

}  // namespace tor
