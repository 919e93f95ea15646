// tor_kernels.cu -- kernels of the Torontonian path (sm_103a).
//
//   k_prep        O (xxpp or xpxp, leading dim ld) -> B = I - O, mode-interleaved
//                 2k x 2k (plus the exact low parts of the diagonal for the dd
//                 tier).  Step a0: the selection of Eq. 1 is the caller's.
//   k_dfs<Tier>   one thread per prefix chunk: chunk root + depth-first walk
//                 (tor_dfs.cuh); exact fixed-point partials per block (and
//                 per chunk on request).
//   k_finalize    sums the block partials (exact) and writes a tor_result.
//   k_dfma_peak   FP64 FMA throughput probe (the roofline denominator).
#include <cuda_runtime.h>
#include <cstdint>
#include "tor_dfs.cuh"
#include "tor_internal.h"
#include "tor_walk.cuh"
#include "tor_fx9.cuh"

namespace tor {

// B[(2i+q)*2k + (2j+q')] = delta - O[row(i,q)][row(j,q')];  Blo = exact low part of the diagonal
__global__ void k_prep(const double *__restrict__ O, int k, int ld, int layout,
                       double *__restrict__ B, double *__restrict__ Blo) {
  const int n = 2 * k;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int r = idx / n, c = idx % n;
  const int mi = r >> 1, qi = r & 1, mj = c >> 1, qj = c & 1;
  const int ri = (layout == 0) ? (qi * k + mi) : r;
  const int rj = (layout == 0) ? (qj * k + mj) : c;
  const double o = O[(size_t)ri * ld + rj];
  if (r == c) {
    const dd s = two_sum(1.0, -o);  // 1 - o = s.hi + s.lo exactly
    B[idx] = s.hi;
    if (Blo) Blo[r] = s.lo;
  } else {
    B[idx] = -o;
  }
}

template <class Tier>
__global__ void __launch_bounds__(128, Tier::MINB)
k_dfs(const double *__restrict__ B, const double *__restrict__ Blo, int k, const WalkSegs seg,
      double *__restrict__ scratch, unsigned long long *__restrict__ block_part,
      unsigned long long *__restrict__ chunk_part, int *__restrict__ status) {
  extern __shared__ double smem[];
  const size_t st = (size_t)gridDim.x * blockDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double *S = scratch + gtid;
  double *Q = smem + threadIdx.x;  // this thread's shared-memory node slot (stride blockDim.x)
  const SrcPrepped src{B, Blo, 2 * k};

  using Acc = typename Tier::Acc;
  constexpr int L = sizeof(Acc) / 8;  // limbs per accumulator; partials hold 2 L
  Acc tot_tor, tot_sabs;
  fx_zero(tot_tor);
  fx_zero(tot_sabs);
  int flags = 0;

#pragma unroll 1
  for (int g = 0; g < 2; ++g) {
    const int r1 = seg.r1[g];
    for (unsigned long long c = seg.c0[g] + gtid; c < seg.c1[g]; c += st) {
      SumsOf<Acc> Sm;
      fx_zero(Sm.tor);
      fx_zero(Sm.sabs);
      Sm.flags = 0;
      walk_chunk<Tier>(src, k, r1, c, S, st, Sm, Q, blockDim.x);
      if (chunk_part && g == 0) {
        unsigned long long *o = chunk_part + (size_t)(c - seg.c0[0]) * 2 * L;
#pragma unroll
        for (int i = 0; i < L; ++i) { o[i] = Sm.tor.w[i]; o[L + i] = Sm.sabs.w[i]; }
      }
      fx_add(tot_tor, Sm.tor);
      fx_add(tot_sabs, Sm.sabs);
      flags |= Sm.flags;
    }
  }

  // block reduction (exact, so the order does not matter) in the node slots' memory
  __syncthreads();
  unsigned long long(*red)[2 * L] = reinterpret_cast<unsigned long long(*)[2 * L]>(smem);
#pragma unroll
  for (int i = 0; i < L; ++i) { red[threadIdx.x][i] = tot_tor.w[i]; red[threadIdx.x][L + i] = tot_sabs.w[i]; }
  if (flags) atomicOr(status, flags);
  __syncthreads();
  if (threadIdx.x == 0) {
    Acc a, b, x;
    fx_zero(a);
    fx_zero(b);
    for (int t2 = 0; t2 < (int)blockDim.x; ++t2) {
      for (int i = 0; i < L; ++i) x.w[i] = red[t2][i];
      fx_add(a, x);
      for (int i = 0; i < L; ++i) x.w[i] = red[t2][L + i];
      fx_add(b, x);
    }
    for (int i = 0; i < L; ++i) {
      block_part[(size_t)blockIdx.x * 2 * L + i] = a.w[i];
      block_part[(size_t)blockIdx.x * 2 * L + L + i] = b.w[i];
    }
  }
}

// The 256-bit-class tier: the fx9 walk (tor_fx9.cuh) over the same chunk
// segments; per-thread 512-bit totals, exact block sums of 16 limbs.  The
// totals (read and written once per chunk) and, with FX9_SUMS_SMEM, each
// chunk's column sums live in shared memory behind the mini-stacks
// ([word][thread]), so that the walk's registers hold only the nodes it
// updates.
__global__ void __launch_bounds__(128, FX9_MINB)
k_dfs_fx9(const double *__restrict__ B, const double *__restrict__ Blo, int k, const WalkSegs seg,
          char *__restrict__ scratch, unsigned long long *__restrict__ block_part,
          unsigned long long *__restrict__ chunk_part, int *__restrict__ status) {
  extern __shared__ int4 smem_fx9[];
  const unsigned st = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned bd = blockDim.x, tid = threadIdx.x;
  const Fx9Mem G{scratch, st, gtid};
  const Fx9Mem Q{reinterpret_cast<char *>(smem_fx9), bd, tid};
  unsigned long long *tot = reinterpret_cast<unsigned long long *>(
      reinterpret_cast<char *>(smem_fx9) + (size_t)fx9_smem_entries(FX9_RSMEM) * 36 * bd);
#if FX9_SUMS_SMEM
  long long *colsum = reinterpret_cast<long long *>(tot + 16 * bd);  // the chunk's column sums
#endif
  const SrcPrepped src{B, Blo, 2 * k};
#pragma unroll
  for (int i = 0; i < 16; ++i) tot[i * bd + tid] = 0ull;
  int flags = 0;
#pragma unroll 1
  for (int g = 0; g < 2; ++g) {
    const int r1 = seg.r1[g];
#pragma unroll 1
    for (unsigned long long c = seg.c0[g] + gtid; c < seg.c1[g]; c += st) {
#if FX9_SUMS_SMEM
      Fx9SumsShared A{colsum + tid, bd, 0};
#else
      Fx9Sums A;
#endif
      A.zero();
      fx9_walk_chunk(src, k, r1, c, G, Q, A);
      Fx512 ct, cs;
      fx9_fold(A, ct, cs);
      if (chunk_part && g == 0) {
        unsigned long long *o = chunk_part + (size_t)(c - seg.c0[0]) * 16;
#pragma unroll
        for (int i = 0; i < 8; ++i) { o[i] = ct.w[i]; o[8 + i] = cs.w[i]; }
      }
      Fx512 t;
#pragma unroll
      for (int i = 0; i < 8; ++i) t.w[i] = tot[i * bd + tid];
      fx_add(t, ct);
#pragma unroll
      for (int i = 0; i < 8; ++i) tot[i * bd + tid] = t.w[i];
#pragma unroll
      for (int i = 0; i < 8; ++i) t.w[i] = tot[(8 + i) * bd + tid];
      fx_add(t, cs);
#pragma unroll
      for (int i = 0; i < 8; ++i) tot[(8 + i) * bd + tid] = t.w[i];
      flags |= A.flags;
    }
  }
  if (flags) atomicOr(status, flags);
  __syncthreads();
  if (tid == 0) {
    Fx512 a, b, x;
    fx_zero(a);
    fx_zero(b);
    for (unsigned t2 = 0; t2 < bd; ++t2) {
      for (int i = 0; i < 8; ++i) x.w[i] = tot[i * bd + t2];
      fx_add(a, x);
      for (int i = 0; i < 8; ++i) x.w[i] = tot[(8 + i) * bd + t2];
      fx_add(b, x);
    }
    for (int i = 0; i < 8; ++i) {
      block_part[(size_t)blockIdx.x * 16 + i] = a.w[i];
      block_part[(size_t)blockIdx.x * 16 + 8 + i] = b.w[i];
    }
  }
}

// shared memory of a fx9 walk block: the per-thread mini-stacks, the
// per-thread 512-bit totals (128 bytes) and the chunk's column sums (104 bytes)
static size_t fx9_smem_bytes(int block) {
  return ((size_t)fx9_smem_entries(FX9_RSMEM) * 36 + 128 + (FX9_SUMS_SMEM ? 104 : 0)) * (size_t)block;
}

// sum of the blocks' partials (2 L limbs each) -> tor_result
template <int L>
__global__ void k_finalize(const unsigned long long *__restrict__ block_part, int nblocks, int k,
                           int tier, const int *__restrict__ status, tor_result *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  FxW<L> a, b, x;
  fx_zero(a);
  fx_zero(b);
  for (int j = 0; j < nblocks; ++j) {
    for (int i = 0; i < L; ++i) x.w[i] = block_part[(size_t)j * 2 * L + i];
    fx_add(a, x);
    for (int i = 0; i < L; ++i) x.w[i] = block_part[(size_t)j * 2 * L + L + i];
    fx_add(b, x);
  }
  unsigned long long w[2 * L];
  for (int i = 0; i < L; ++i) { w[i] = a.w[i]; w[L + i] = b.w[i]; }
  fixed_to_result_w<L>(w, k, tier, *status, out);
}

// Tor of the empty pattern (k = 0): only the empty subset, t = 1
__global__ void k_result_one(tor_result *out, int tier) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = tor_result{1.0, 0.0, 1.0, 0.0, tier, TOR_OK};
}

int launch_result_one(tor_result *out, int tier, cudaStream_t s) {
  k_result_one<<<1, 32, 0, s>>>(out, tier);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Independent DFMA chains; the result is consumed so the loop is not removed.
__global__ void k_dfma_peak(double *sink, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
  }
  const double s = x0 + x1 + x2 + x3;
  if (s == 1234.5) sink[threadIdx.x] = s;
}

// Independent mad.wide.s32 chains (32 x 32 -> 64 multiply-add, the fixed-point
// tiers' limb product); the result is consumed so the loop is not removed.
__global__ void k_imad_peak(long long *sink, int iters, int a, int b) {
  long long x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) asm volatile("mad.wide.s32 %0, %1, %2, %0;" : "+l"(x[j]) : "r"(a + j), "r"(b));
  }
  long long s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == 12345) sink[threadIdx.x] = s;
}

void launch_imad_peak(long long *sink, int grid, int block, int iters, cudaStream_t s) {
  k_imad_peak<<<grid, block, 0, s>>>(sink, iters, 3, 5);
}

// ------------------------------------------------------------ host launchers
void launch_prep(const double *O, int k, int ld, int layout, double *B, double *Blo, cudaStream_t s) {
  const int n = 4 * k * k;
  k_prep<<<(n + 255) / 256, 256, 0, s>>>(O, k, ld, layout, B, Blo);
}

// elementwise s + a1 b1 + a2 b2 in the 256-bit-class arithmetic (fx9), as the
// walk's Schur updates form them; operands of nine int32 limbs each
__global__ void k_fx256_fma2(const int *__restrict__ s, const int *__restrict__ a1, const int *__restrict__ b1,
                             const int *__restrict__ a2, const int *__restrict__ b2, int n, int *__restrict__ out,
                             int *__restrict__ ovf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  fx9 v[5];
  const int *src[5] = {s, a1, b1, a2, b2};
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int j = 0; j < 9; ++j) v[q].l[j] = src[q][9 * (size_t)i + j];
  int o = 0;
  const fx9 r = fx9_fma2(v[0], v[1], v[2], v[3], v[4], o);
#pragma unroll
  for (int j = 0; j < 9; ++j) out[9 * (size_t)i + j] = r.l[j];
  ovf[i] = o;
}

int launch_fx256_fma2(const int *s, const int *a1, const int *b1, const int *a2, const int *b2, int n, int *out,
                      int *ovf, cudaStream_t st) {
  if (n > 0) k_fx256_fma2<<<(n + 127) / 128, 128, 0, st>>>(s, a1, b1, a2, b2, n, out, ovf);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// calls f(Tier{}) with the walk tier of a TOR_PREC_* value
template <class F>
static void with_tier(int tier, F &&f) {
  switch (tier) {
    case TOR_PREC_DD: f(TierDD{}); break;
    case TOR_PREC_FX128: f(TierFx<FX128_FRAC>{}); break;
    default: f(TierF64{}); break;
  }
}

void launch_dfs(int tier, int grid, int block, const double *B, const double *Blo, int k, const WalkSegs &seg,
                double *scratch, unsigned long long *block_part, unsigned long long *chunk_part, int *status,
                cudaStream_t s) {
  if (tier == TOR_PREC_FX256) {
    const size_t sm = fx9_smem_bytes(block);
    cudaFuncSetAttribute(k_dfs_fx9, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_dfs_fx9<<<grid, block, sm, s>>>(B, Blo, k, seg, reinterpret_cast<char *>(scratch), block_part, chunk_part,
                                       status);
    return;
  }
  with_tier(tier, [&](auto t) {
    using Tier = decltype(t);
    const size_t sm = walk_smem_bytes<Tier>(block);
    cudaFuncSetAttribute(k_dfs<Tier>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_dfs<Tier><<<grid, block, sm, s>>>(B, Blo, k, seg, scratch, block_part, chunk_part, status);
  });
}

int dfs_max_blocks_per_sm(int tier, int block) {
  int n = 0;
  cudaError_t e = cudaSuccess;
  if (tier == TOR_PREC_FX256) {
    const size_t sm = fx9_smem_bytes(block);
    cudaFuncSetAttribute(k_dfs_fx9, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dfs_fx9, block, sm);
    return (e == cudaSuccess && n > 0) ? n : 1;
  }
  with_tier(tier, [&](auto t) {
    using Tier = decltype(t);
    const size_t sm = walk_smem_bytes<Tier>(block);
    cudaFuncSetAttribute(k_dfs<Tier>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dfs<Tier>, block, sm);
  });
  return (e == cudaSuccess && n > 0) ? n : 1;
}

void launch_finalize(const unsigned long long *block_part, int nblocks, int k, int tier,
                     const int *status, tor_result *out, cudaStream_t s) {
  if (tier == TOR_PREC_FX256) k_finalize<8><<<1, 32, 0, s>>>(block_part, nblocks, k, tier, status, out);
  else k_finalize<4><<<1, 32, 0, s>>>(block_part, nblocks, k, tier, status, out);
}

void launch_dfma_peak(double *sink, int grid, int block, int iters, cudaStream_t s) {
  k_dfma_peak<<<grid, block, 0, s>>>(sink, iters, 1.0000001, 1e-9);
}

int scratch_entries(int tier, int k, int r1) {
  if (tier == TOR_PREC_FX256) return (fx9_stack_entries(k, r1) * 36 + 7) / 8;  // in doubles
  int rreg = 0, w = 1;
  with_tier(tier, [&](auto t) {
    using Tier = decltype(t);
    rreg = Tier::RREG;
    w = Tier::W;
  });
  const int a = sz(k), b = stack_entries(r1, rreg);
  return w * (a > b ? a : b);
}

}  // namespace tor
