// tor_batch.cu -- many Torontonians of uneven size in one persistent launch per tier.
//
// Sampling produces thousands of click patterns whose click counts k vary
// (a 2^k spread in cost).  The batch is scheduled entirely on the device so
// that the whole sequence (bound pass, plan, walks, finalize) can be captured
// once in a CUDA graph and replayed with new inputs, with no host round trip:
//
//  k_batch_plan      one block: per instance the tier (given, or from the bound
//                    pass) and the walk depth r1 (chunks fix the top k - r1
//                    modes, Algorithm 1's balanced partition), a counting sort
//                    of instances by (tier, r1 descending), and an exclusive
//                    scan of the chunk counts that lays every (instance, chunk)
//                    pair out on one item axis per tier.  Large chunks come
//                    first so the tail of the launch is made of small items.
//  k_batch_walk<T>   persistent: each warp takes 32 consecutive items from an
//                    atomic counter, finds each item's instance by binary search
//                    over the scan, gathers I - O straight from the caller's
//                    matrix, walks the chunk (tor_dfs.cuh; tor_fx9.cuh for the
//                    256-bit-class tier), and adds the exact partial sums
//                    into the instance's accumulator with 64-bit atomics that
//                    propagate carries.  Integer addition is associative, so
//                    the result does not depend on which warp ran which item.
//  k_batch_finalize  one thread per instance: accumulator -> tor_result.
//
// Four tiers share the item axis in the order FP64, double-double, 128-bit
// fixed point, 256-bit-class fixed point (the per-instance precision choice
// of Sec. 5.4, Eq. bitlen).  In TOR_PREC_AUTO mode up to two more
// plan/walk/finalize rounds re-run every instance whose result misses the
// tolerance in the next tier with more precision whose range holds it:
// FP64 -> 128-bit -> 256-bit fixed point, double-double only for instances
// outside the fixed-point ranges.
#include <cuda_runtime.h>
#include <cstdint>
#include "tor_dfs.cuh"
#include "tor_internal.h"
#include "tor_walk.cuh"
#include "tor_fx9.cuh"

namespace tor {

constexpr int PLAN_THREADS = 1024;
constexpr int NTIER = 4;
constexpr int NKEY = NTIER * 65;  // (tier 1..4) x (64 - r1)
constexpr int ACC_LIMBS = 16;     // per instance: two sums of up to 8 limbs

__device__ __forceinline__ bool fx_in_range(const tor_bound &b) {
  return b.log_tmax <= FX128_MAX_LOG2_TMAX * 0.6931472f;
}
__device__ __forceinline__ bool fx256_in_range(const tor_bound &b) {
  return b.log_tmax <= FX256_MAX_LOG2_TMAX * 0.6931472f;
}

// acc (L limbs) += X, exactly modulo 2^(64 L), from any number of threads
template <int L>
__device__ __forceinline__ void fx_atomic_add(unsigned long long *acc, const FxW<L> &X) {
  unsigned long long carry = 0ull;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const unsigned long long v = X.w[j] + carry;
    const unsigned long long c1 = (v < carry) ? 1ull : 0ull;  // X.w[j] == 2^64-1 with a carry in
    unsigned long long c2 = 0ull;
    if (v) {
      const unsigned long long old = atomicAdd(acc + j, v);
      c2 = (old + v < old) ? 1ull : 0ull;
    }
    carry = c1 + c2;
  }
}

// mode 0: first round; mode 1: escalate the instances that missed tol to the
// next tier with more precision whose range holds them (FP64 -> 128-bit ->
// 256-bit fixed point, double-double outside the fixed-point ranges); bounds
// is needed for AUTO and for explicit fixed-point batches
__global__ void __launch_bounds__(PLAN_THREADS)
k_batch_plan(const int *__restrict__ k, const tor_bound *__restrict__ bounds, int n, int prec, int kmax,
             const unsigned char *__restrict__ r1_table /* [4][65] */, int mode, double tol,
             BatchPlan p) {
  __shared__ unsigned int hist[NKEY], cursor[NKEY];
  __shared__ unsigned long long part[PLAN_THREADS];
  const int tid = threadIdx.x;
  for (int e = tid; e < NKEY; e += blockDim.x) hist[e] = 0;
  __syncthreads();
  // phase 1: per instance tier, r1, key
  for (int i = tid; i < n; i += blockDim.x) {
    const int ki = k[i];
    int tier;
    if (mode == 0) {
      tier = (prec == TOR_PREC_AUTO) ? (bounds ? bounds[i].tier : TOR_PREC_FP64) : prec;
      if (ki < 0 || ki > kmax) tier = 0;
      if (tier == TOR_PREC_FX128 && ki > 0 && !(bounds && fx_in_range(bounds[i]))) tier = 0;
      if (tier == TOR_PREC_FX256 && ki > 0 && !(bounds && fx256_in_range(bounds[i]))) tier = 0;
      p.tier[i] = (unsigned char)tier;
      p.flags[i] = (tier == 0) ? ST_RANGE : 0;
      p.escalated[i] = 0;
    } else {
      tier = 0;
      const tor_result r = p.result[i];
      const double mag = r.hi < 0 ? -r.hi : r.hi;
      if (r.status == TOR_OK && r.err_est > tol * mag) {
        const bool f1 = bounds && ki > 0 && fx_in_range(bounds[i]);
        const bool f2 = bounds && ki > 0 && fx256_in_range(bounds[i]);
        if (p.tier[i] == TOR_PREC_FP64)
          tier = f1 ? TOR_PREC_FX128 : (f2 ? TOR_PREC_FX256 : TOR_PREC_DD);
        else if (p.tier[i] == TOR_PREC_FX128)
          tier = f2 ? TOR_PREC_FX256 : TOR_PREC_DD;
        else if (p.tier[i] == TOR_PREC_DD && f2)
          tier = TOR_PREC_FX256;
      }
      p.escalated[i] = (tier != 0) ? 1 : 0;
      if (tier != 0) {
        p.tier[i] = (unsigned char)tier;
        p.flags[i] = 0;
      }
    }
    int key = -1, r1 = 0;
    if (tier != 0) {
      r1 = r1_table[tier * 65 + ki];
      if (r1 > ki) r1 = ki;
      key = (tier - 1) * 65 + (64 - r1);
    }
    p.r1[i] = (unsigned char)r1;
    p.key[i] = key;
    if (mode == 0 || tier != 0) {
      unsigned long long *a = p.acc + (size_t)i * ACC_LIMBS;
#pragma unroll
      for (int j = 0; j < ACC_LIMBS; ++j) a[j] = 0ull;
      if (ki == 0 && tier != 0) {  // Tor = sum t = 1 (empty set only): 1 in the tier's sums
        const int L = partial_limbs(tier) / 2;
        a[L / 2] = 1ull;
        a[L + L / 2] = 1ull;
      }
    }
    if (key >= 0) atomicAdd(&hist[key], 1u);
  }
  __syncthreads();
  if (tid == 0) {
    unsigned int run = 0;
    for (int e = 0; e < NKEY; ++e) {
      cursor[e] = run;
      run += hist[e];
      if (e % 65 == 64) p.counts[e / 65] = run;  // instances of tiers <= e / 65 + 1
    }
  }
  __syncthreads();
  // phase 2: scatter into sorted order
  for (int i = tid; i < n; i += blockDim.x) {
    const int key = p.key[i];
    if (key >= 0) p.order[atomicAdd(&cursor[key], 1u)] = i;
  }
  __syncthreads();
  // phase 3: exclusive scan of chunk counts over the sorted order
  const int m = (int)p.counts[NTIER - 1];
  const int per = (m + PLAN_THREADS - 1) / PLAN_THREADS;
  const int lo = tid * per, hi = min(m, lo + per);
  unsigned long long sum = 0;
  for (int j = lo; j < hi; ++j) {
    const int i = p.order[j];
    const int ki = k[i];
    sum += (ki == 0) ? 0ull : (1ull << (ki - p.r1[i]));
  }
  part[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    unsigned long long run = 0;
    for (int t = 0; t < PLAN_THREADS; ++t) { const unsigned long long v = part[t]; part[t] = run; run += v; }
  }
  __syncthreads();
  unsigned long long run = part[tid];
  for (int j = lo; j < hi; ++j) {
    p.item_off[j] = run;
    const int i = p.order[j];
    const int ki = k[i];
    run += (ki == 0) ? 0ull : (1ull << (ki - p.r1[i]));
  }
  if (tid == PLAN_THREADS - 1) p.item_off[m] = run;
  __syncthreads();
  if (tid == 0) {  // items of tier t + 1: [range[2t], range[2t + 1])
    for (int t = 0; t < NTIER; ++t) {
      p.range[2 * t] = (t == 0) ? 0ull : p.item_off[p.counts[t - 1]];
      p.range[2 * t + 1] = p.item_off[p.counts[t]];
      p.counter[t] = p.range[2 * t];
    }
  }
}

template <class Tier, bool PAT>
__global__ void __launch_bounds__(128, Tier::MINB)
k_batch_walk(BatchInput in, BatchPlan p, double *__restrict__ scratch) {
  extern __shared__ double smem[];
  double *Q = smem + threadIdx.x;
  constexpr int t = Tier::PREC - 1;
  const size_t st = (size_t)gridDim.x * blockDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double *S = scratch + gtid;
  const int lane = threadIdx.x & 31;
  const unsigned long long end = p.range[2 * t + 1];
  const int jlo = (t == 0) ? 0 : (int)p.counts[t - 1];
  const int jhi = (int)p.counts[t];
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.counter + t, 32ull);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= end) break;
    const unsigned long long item = base + lane;
    if (item < end) {
      // last sorted position j in [jlo, jhi) with item_off[j] <= item
      int a = jlo, b = jhi - 1;
      while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (p.item_off[mid] <= item) a = mid; else b = mid - 1;
      }
      const int i = p.order[a];
      const unsigned long long c = item - p.item_off[a];
      const int ki = in.k[i], r1 = p.r1[i];
      Sums Sm;
      fx_zero(Sm.tor);
      fx_zero(Sm.sabs);
      Sm.flags = 0;
      if constexpr (PAT) {
        unsigned char gm[64];
        int m = 0;
        for (int w = 0; w < in.words; ++w)
          for (unsigned long long bits = in.patterns[(size_t)i * in.words + w]; bits && m < 64; bits &= bits - 1)
            gm[m++] = (unsigned char)(64 * w + __ffsll((long long)bits) - 1);
        const SrcPattern src{in.Ofull, in.M, in.ldfull, gm};
        walk_chunk<Tier>(src, ki, r1, c, S, st, Sm, Q, blockDim.x);
      } else {
        const SrcDirect src{in.O[i], ki, in.ld[i], in.layout};
        walk_chunk<Tier>(src, ki, r1, c, S, st, Sm, Q, blockDim.x);
      }
      fx_atomic_add(p.acc + (size_t)i * ACC_LIMBS, Sm.tor);
      fx_atomic_add(p.acc + (size_t)i * ACC_LIMBS + 4, Sm.sabs);
      if (Sm.flags) atomicOr(p.flags + i, Sm.flags);
    }
  }
}

// The 256-bit-class tier's persistent walk: the same item scheme, the fx9
// walk (tor_fx9.cuh) with its planar global stacks and shared-memory
// mini-stacks, 512-bit partial sums.
template <bool PAT>
__global__ void __launch_bounds__(128, FX9_MINB)
k_batch_walk_fx9(BatchInput in, BatchPlan p, char *__restrict__ scratch) {
  extern __shared__ int4 smem_b9[];
  constexpr int t = TOR_PREC_FX256 - 1;
  const unsigned st = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const Fx9Mem G{scratch, st, gtid};
  const Fx9Mem Q{reinterpret_cast<char *>(smem_b9), blockDim.x, threadIdx.x};
  const int lane = threadIdx.x & 31;
  const unsigned long long end = p.range[2 * t + 1];
  const int jlo = (int)p.counts[t - 1];
  const int jhi = (int)p.counts[t];
#if FX9_SUMS_SMEM
  long long *colsum = reinterpret_cast<long long *>(reinterpret_cast<char *>(smem_b9) +
                                                    (size_t)fx9_smem_entries(FX9_RSMEM) * 36 * blockDim.x);
#endif
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.counter + t, 32ull);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= end) break;
    const unsigned long long item = base + lane;
    if (item < end) {
      int a = jlo, b = jhi - 1;
      while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (p.item_off[mid] <= item) a = mid; else b = mid - 1;
      }
      const int i = p.order[a];
      const unsigned long long c = item - p.item_off[a];
      const int ki = in.k[i], r1 = p.r1[i];
#if FX9_SUMS_SMEM
      Fx9SumsShared A{colsum + threadIdx.x, blockDim.x, 0};
#else
      Fx9Sums A;
#endif
      A.zero();
      if constexpr (PAT) {
        unsigned char gm[64];
        int m = 0;
        for (int w = 0; w < in.words; ++w)
          for (unsigned long long bits = in.patterns[(size_t)i * in.words + w]; bits && m < 64; bits &= bits - 1)
            gm[m++] = (unsigned char)(64 * w + __ffsll((long long)bits) - 1);
        const SrcPattern src{in.Ofull, in.M, in.ldfull, gm};
        fx9_walk_chunk(src, ki, r1, c, G, Q, A);
      } else {
        const SrcDirect src{in.O[i], ki, in.ld[i], in.layout};
        fx9_walk_chunk(src, ki, r1, c, G, Q, A);
      }
      Fx512 ct, cs;
      fx9_fold(A, ct, cs);
      fx_atomic_add(p.acc + (size_t)i * ACC_LIMBS, ct);
      fx_atomic_add(p.acc + (size_t)i * ACC_LIMBS + 8, cs);
      if (A.flags) atomicOr(p.flags + i, A.flags);
    }
  }
}

static size_t fx9_batch_smem(int block) {
  const size_t slot = (size_t)fx9_smem_entries(FX9_RSMEM) * 36 + (FX9_SUMS_SMEM ? 104 : 0);
  return slot * (size_t)block;
}

// tol > 0: mark results whose error bound exceeds tol * |Tor| with TOR_EPREC
__global__ void k_batch_finalize(const int *__restrict__ k, int n, int only_escalated, double tol, BatchPlan p,
                                 tor_result *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (only_escalated && !p.escalated[i]) return;
  tor_result r;
  if (p.tier[i] == 0) {
    r = tor_result{0.0, 0.0, 0.0, 0.0, 0, TOR_EINVAL};
  } else {
    fixed_to_result(p.acc + (size_t)i * ACC_LIMBS, k[i], p.tier[i], p.flags[i], &r);
    const double mag = r.hi < 0 ? -r.hi : r.hi;
    if (tol > 0.0 && r.status == TOR_OK && r.err_est > tol * mag) r.status = TOR_EPREC;
  }
  out[i] = r;
  p.result[i] = r;
}

int launch_batch_plan(const int *k, const tor_bound *bounds, int n, int prec, int kmax,
                      const unsigned char *r1_table, int mode, double tol, const BatchPlan &p, cudaStream_t s) {
  k_batch_plan<<<1, PLAN_THREADS, 0, s>>>(k, bounds, n, prec, kmax, r1_table, mode, tol, p);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_batch_walk(int tier, int grid, int block, const BatchInput &in, const BatchPlan &p, double *scratch,
                      cudaStream_t s) {
  const bool pat = in.words > 0;
  if (tier == TOR_PREC_FX256) {
    const size_t sm = fx9_batch_smem(block);
    char *scr = reinterpret_cast<char *>(scratch);
    if (pat) {
      cudaFuncSetAttribute(k_batch_walk_fx9<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      k_batch_walk_fx9<true><<<grid, block, sm, s>>>(in, p, scr);
    } else {
      cudaFuncSetAttribute(k_batch_walk_fx9<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      k_batch_walk_fx9<false><<<grid, block, sm, s>>>(in, p, scr);
    }
  } else if (tier == TOR_PREC_DD) {
    const size_t sm = walk_smem_bytes<TierDD>(block);
    if (pat) k_batch_walk<TierDD, true><<<grid, block, sm, s>>>(in, p, scratch);
    else k_batch_walk<TierDD, false><<<grid, block, sm, s>>>(in, p, scratch);
  } else if (tier == TOR_PREC_FX128) {
    using TF = TierFx<FX128_FRAC>;
    const size_t sm = walk_smem_bytes<TF>(block);
    if (pat) k_batch_walk<TF, true><<<grid, block, sm, s>>>(in, p, scratch);
    else k_batch_walk<TF, false><<<grid, block, sm, s>>>(in, p, scratch);
  } else {
    const size_t sm = walk_smem_bytes<TierF64>(block);
    if (pat) k_batch_walk<TierF64, true><<<grid, block, sm, s>>>(in, p, scratch);
    else k_batch_walk<TierF64, false><<<grid, block, sm, s>>>(in, p, scratch);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void k_pattern_popcount(const unsigned long long *__restrict__ patterns, int n, int words,
                                   int *__restrict__ k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int w = 0; w < words; ++w) c += __popcll(patterns[(size_t)i * words + w]);
  k[i] = c;
}

int launch_pattern_popcount(const unsigned long long *patterns, int n, int words, int *k, cudaStream_t s) {
  k_pattern_popcount<<<(n + 255) / 256, 256, 0, s>>>(patterns, n, words, k);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_batch_finalize(const int *k, int n, int only_escalated, double tol, const BatchPlan &p,
                          tor_result *out, cudaStream_t s) {
  k_batch_finalize<<<(n + 127) / 128, 128, 0, s>>>(k, n, only_escalated, tol, p, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class K>
static int occ_of(K kern, int block, size_t sm) {
  int nb = 0;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, sm);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int batch_walk_max_blocks_per_sm(int tier, int block, bool patterns) {
  if (tier == TOR_PREC_FX256) {
    const size_t sm = fx9_batch_smem(block);
    return patterns ? occ_of(k_batch_walk_fx9<true>, block, sm) : occ_of(k_batch_walk_fx9<false>, block, sm);
  }
  if (tier == TOR_PREC_FX128) {
    using TF = TierFx<FX128_FRAC>;
    const size_t sm = walk_smem_bytes<TF>(block);
    return patterns ? occ_of(k_batch_walk<TF, true>, block, sm) : occ_of(k_batch_walk<TF, false>, block, sm);
  }
  if (tier == TOR_PREC_DD) {
    const size_t sm = walk_smem_bytes<TierDD>(block);
    return patterns ? occ_of(k_batch_walk<TierDD, true>, block, sm) : occ_of(k_batch_walk<TierDD, false>, block, sm);
  }
  const size_t sm = walk_smem_bytes<TierF64>(block);
  return patterns ? occ_of(k_batch_walk<TierF64, true>, block, sm) : occ_of(k_batch_walk<TierF64, false>, block, sm);
}

}  // namespace tor
