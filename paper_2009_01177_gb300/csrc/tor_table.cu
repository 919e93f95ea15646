// tor_table.cu -- the Torontonian of EVERY click pattern of one state.
//
// For the full M-mode matrix O (Eq. 1), the submatrix of a pattern's
// submatrix is the submatrix of O: (O_S)_Z = O_Z for Z inside S.  So the
// terms t_Z = 1/sqrt(det(I - O_Z)) of Eq. 2 are shared by all patterns, and
//   Tor(O_S) = sum over Z inside S of (-1)^(|S| - |Z|) t_Z
// is the Moebius transform of the table t over the subset lattice.  One walk
// over the 2^M subsets of the full state (the same prefix-chunk depth-first
// walk as a single Torontonian, tor_dfs.cuh) stores every t_Z exactly in
// 256-bit fixed point; an in-place transform then turns the table into all
// 2^M Torontonians with integer arithmetic, so each result is as accurate as
// its terms.  Cost: 2^M subset determinants and M passes of additions,
// against sum_S 2^|S| = 3^M determinants for the patterns one by one.
//
//  k_dfs_table<Tier>   the walk, with an accumulator that stores each term at
//                      its subset's index instead of summing.  Every chunk is
//                      walked in the same order, so the n-th term of chunk c
//                      belongs to the mask (c << r1) | order[n], with the
//                      order table generated on the host from the walk's rule.
//  k_mobius_pass       a tile of 1024 entries in shared memory takes the
//                      signed differences (t) and plain sums (sum of t, for
//                      the error bounds) over B of the mask bits; ceil
//                      passes over the table cover all M bits.
//  k_table_finalize    entry -> tor_result (hi + lo, sum_abs, err_est).
#include <cuda_runtime.h>
#include <cstdint>
#include "tor_dfs.cuh"
#include "tor_internal.h"
#include "tor_walk.cuh"

namespace tor {

// where a table walk puts its terms
struct TableAcc {
  Fx256 *table;                  // 2^M exact terms, index = subset mask
  const unsigned int *order;     // low-mode mask of the n-th term of a chunk
  unsigned long long base;       // chunk index << r1
  unsigned int seq;              // terms stored so far in this chunk
};

// A tier whose accumulation stores the term at its subset's index
template <class Base>
struct TableTier : Base {
  using Acc = TableAcc;
  using T = typename Base::T;
  __device__ static __forceinline__ void acc(SumsOf<TableAcc> &S, T t, bool) {
    SumsOf<Fx256> one;  // the base tier's exact conversion of +t
    fx_zero(one.tor);
    fx_zero(one.sabs);
    one.flags = 0;
    Base::acc(one, t, false);
    S.flags |= one.flags;
    const unsigned long long m = S.tor.base | S.tor.order[S.tor.seq++];
    S.tor.table[m] = one.sabs;
  }
};

template <class Base>
__global__ void __launch_bounds__(128, Base::MINB)
k_dfs_table(const double *__restrict__ B, const double *__restrict__ Blo, int k, int r1,
            unsigned long long nchunks, double *__restrict__ scratch, const unsigned int *__restrict__ order,
            Fx256 *__restrict__ table, int *__restrict__ status) {
  using Tier = TableTier<Base>;
  extern __shared__ double smem[];
  const size_t st = (size_t)gridDim.x * blockDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double *S = scratch + gtid;
  double *Q = smem + threadIdx.x;
  const SrcPrepped src{B, Blo, 2 * k};
  int flags = 0;
  for (unsigned long long c = gtid; c < nchunks; c += st) {
    SumsOf<TableAcc> Sm;
    Sm.tor = TableAcc{table, order, c << r1, 0u};
    Sm.sabs = Sm.tor;
    Sm.flags = 0;
    walk_chunk<Tier>(src, k, r1, c, S, st, Sm, Q, blockDim.x);
    flags |= Sm.flags;
  }
  if (flags) atomicOr(status, flags);
}

// One pass of the transforms over mask bits [b, b + nb): a block holds the
// 2^nb x lo_n entries whose masks share all other bits (lo_n consecutive low
// offsets, so that loads and stores coalesce), applies for each of its bits
//   t[m | bit] -= t[m],   s[m | bit] += s[m]   (m without the bit),
// and writes the tile back.  2^nb * lo_n = TILE.
constexpr int TILE = 1024;
constexpr int MOB_THREADS = 256;

// init_s: the first pass, which also starts the sums of terms (s = t, from
// the terms alone, so s is not read)
__global__ void __launch_bounds__(MOB_THREADS)
k_mobius_pass(Fx256 *__restrict__ t, double *__restrict__ s, int M, int b, int nb, int lo_n, int init_s) {
  __shared__ unsigned long long tw[4][TILE];
  __shared__ double ts[TILE];
  const unsigned long long lo_blocks = (b == 0) ? 1ull : ((1ull << b) / (unsigned long long)lo_n);
  const unsigned long long blk = blockIdx.x;
  const unsigned long long lo0 = (blk % lo_blocks) * (unsigned long long)lo_n;
  const unsigned long long hi = blk / lo_blocks;                  // the bits above b + nb
  const unsigned long long base = (hi << (b + nb)) + lo0;
  // tile entry e = i * lo_n + l  <->  mask base + (i << b) + l
  for (int e = threadIdx.x; e < TILE; e += MOB_THREADS) {
    const unsigned long long m = base + ((unsigned long long)(e / lo_n) << b) + (unsigned long long)(e % lo_n);
    const Fx256 v = t[m];
    tw[0][e] = v.w[0]; tw[1][e] = v.w[1]; tw[2][e] = v.w[2]; tw[3][e] = v.w[3];
    ts[e] = init_s ? fx_to_double(v) : s[m];
  }
  __syncthreads();
  int j = 0;
  // two bits at a time in registers: each thread takes the quad of entries that
  // differ in bits j and j + 1 of i, and writes back the three that change
  for (; j + 1 < nb; j += 2) {
    for (int q = threadIdx.x; q < TILE / 4; q += MOB_THREADS) {
      const int l = q % lo_n, r = q / lo_n;                          // r: i with bits j, j+1 removed
      const int i0 = ((r >> j) << (j + 2)) | (r & ((1 << j) - 1));
      const int e0 = i0 * lo_n + l, st = lo_n << j;
      Fx256 v[4];
      double sv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * st;
        v[u].w[0] = tw[0][e]; v[u].w[1] = tw[1][e]; v[u].w[2] = tw[2][e]; v[u].w[3] = tw[3][e];
        sv[u] = ts[e];
      }
      fx_sub(v[1], v[0]); fx_sub(v[3], v[2]); sv[1] += sv[0]; sv[3] += sv[2];   // bit j
      fx_sub(v[2], v[0]); fx_sub(v[3], v[1]); sv[2] += sv[0]; sv[3] += sv[1];   // bit j + 1
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        const int e = e0 + u * st;
        tw[0][e] = v[u].w[0]; tw[1][e] = v[u].w[1]; tw[2][e] = v[u].w[2]; tw[3][e] = v[u].w[3];
        ts[e] = sv[u];
      }
    }
    __syncthreads();
  }
  for (; j < nb; ++j) {  // an odd last bit: pairs (e, e + lo_n 2^j) with bit j of i clear
    for (int p = threadIdx.x; p < TILE / 2; p += MOB_THREADS) {
      const int l = p % lo_n, q = p / lo_n;                         // q: i with bit j removed
      const int i0 = ((q >> j) << (j + 1)) | (q & ((1 << j) - 1));
      const int e0 = i0 * lo_n + l, e1 = e0 + (lo_n << j);
      Fx256 x, y;
      x.w[0] = tw[0][e1]; x.w[1] = tw[1][e1]; x.w[2] = tw[2][e1]; x.w[3] = tw[3][e1];
      y.w[0] = tw[0][e0]; y.w[1] = tw[1][e0]; y.w[2] = tw[2][e0]; y.w[3] = tw[3][e0];
      fx_sub(x, y);
      tw[0][e1] = x.w[0]; tw[1][e1] = x.w[1]; tw[2][e1] = x.w[2]; tw[3][e1] = x.w[3];
      ts[e1] += ts[e0];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < TILE; e += MOB_THREADS) {
    const unsigned long long m = base + ((unsigned long long)(e / lo_n) << b) + (unsigned long long)(e % lo_n);
    Fx256 v;
    v.w[0] = tw[0][e]; v.w[1] = tw[1][e]; v.w[2] = tw[2][e]; v.w[3] = tw[3][e];
    t[m] = v;
    s[m] = ts[e];
  }
}

// one bit of the transforms for small tables (fewer entries than a tile)
__global__ void k_mobius_bit(Fx256 *__restrict__ t, double *__restrict__ s, int M, int j) {
  const unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (1ull << (M - 1))) return;
  const unsigned long long m0 = ((p >> j) << (j + 1)) | (p & ((1ull << j) - 1)), m1 = m0 | (1ull << j);
  Fx256 x = t[m1];
  fx_sub(x, t[m0]);
  t[m1] = x;
  s[m1] += s[m0];
}

// sum of |t| starts as the terms themselves
__global__ void k_table_sabs_init(const Fx256 *__restrict__ t, double *__restrict__ s, unsigned long long n) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) s[i] = fx_to_double(t[i]);
}

__global__ void k_table_finalize(const Fx256 *__restrict__ t, const double *__restrict__ s, unsigned long long n,
                                 int tier, const int *__restrict__ status, tor_result *__restrict__ out) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  tor_result r;
  double hi, lo;
  fx_to_dd(t[i], hi, lo);
  r.hi = hi;
  r.lo = lo;
  r.sum_abs = s[i];
  r.err_est = err_gamma(__popcll(i)) * unit_roundoff(tier) * r.sum_abs;
  r.tier = tier;
  const int st = *status;
  r.status = (st & ST_NOTPD) ? TOR_ENOTPD : ((st & ST_RANGE) ? TOR_EINVAL : TOR_OK);
  out[i] = r;
}

template <class F>
static void with_table_tier(int tier, F &&f) {
  switch (tier) {
    case TOR_PREC_DD: f(TierDD{}); break;
    case TOR_PREC_FX128: f(TierFx<FX128_FRAC>{}); break;
    default: f(TierF64{}); break;
  }
}

int table_walk_max_blocks_per_sm(int tier, int block) {
  int n = 0;
  cudaError_t e = cudaSuccess;
  with_table_tier(tier, [&](auto t) {
    using Base = decltype(t);
    const size_t sm = walk_smem_bytes<Base>(block);
    cudaFuncSetAttribute(k_dfs_table<Base>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dfs_table<Base>, block, sm);
  });
  return (e == cudaSuccess && n > 0) ? n : 1;
}

int launch_table_walk(int tier, int grid, int block, const double *B, const double *Blo, int k, int r1,
                      double *scratch, const unsigned int *order, Fx256 *table, int *status, cudaStream_t s) {
  with_table_tier(tier, [&](auto t) {
    using Base = decltype(t);
    const size_t sm = walk_smem_bytes<Base>(block);
    cudaFuncSetAttribute(k_dfs_table<Base>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_dfs_table<Base><<<grid, block, sm, s>>>(B, Blo, k, r1, 1ull << (k - r1), scratch, order, table, status);
  });
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_table_transform(Fx256 *t, double *s, int M, cudaStream_t st) {
  const unsigned long long n = 1ull << M;
  if (M < 10) {  // fewer entries than a tile: one launch per bit
    k_table_sabs_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, s, n);
    if (cudaGetLastError() != cudaSuccess) return -1;
    for (int j = 0; j < M; ++j) {
      const unsigned long long pairs = n / 2;
      k_mobius_bit<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(t, s, M, j);
      if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
  }
  int b = 0;
  while (b < M) {
    int lo_n, nb;
    if (b == 0) { lo_n = 1; nb = 10; }
    else { lo_n = (b >= 5) ? 32 : (1 << b); nb = 10 - __builtin_ctz((unsigned)lo_n); }
    if (b + nb > M) {  // the last bits: keep the tile size by taking more low offsets
      nb = M - b;
      lo_n = TILE >> nb;
      if (lo_n > (1 << b)) return -1;
    }
    const unsigned long long blocks = n / TILE;
    k_mobius_pass<<<(unsigned)blocks, MOB_THREADS, 0, st>>>(t, s, M, b, nb, lo_n, b == 0 ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return -1;
    b += nb;
  }
  return 0;
}

int launch_table_finalize(const Fx256 *t, const double *s, int M, int tier, const int *status, tor_result *out,
                          cudaStream_t st) {
  const unsigned long long n = 1ull << M;
  k_table_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, s, n, tier, status, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tor
