// tor_levels.cu -- the Torontonian by the paper's own schedule.
//
// Algorithm 1 walks the subsets level by level (all Z with the same |Z| = m
// together, so that every unit of work has a matrix of the same size), and
// Algorithm 2 gives each worker its share of a level: the r-th mask of
// popcount m (unranking from the highest bit down: a 1 at bit b leaves
// C(b, m - 1) masks to the lower bits) and then the next mask of the same
// popcount, in decreasing order.  Every subset gets a fresh elimination of
// B_Z = I - O_Z -- no reuse between subsets, the paper's arithmetic work
// -- here the chunk root of the prefix walk with no walked modes
// (walk_chunk with r1 = 0 and the mask as the chunk), summed exactly.
//
// It is an independent second evaluation of Eq. 2 on the GPU (another
// subset order, another factorization of each term) for cross-checks at
// sizes the CPU oracle cannot reach, and it lets each level use its own tier
// (the paper's per-|Z| precision and scaling choice).
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include "tor_dfs.cuh"
#include "tor_internal.h"
#include "tor_walk.cuh"

namespace tor {
namespace {

constexpr int LV_THREADS = 128;

__constant__ unsigned long long c_binom[TOR_LEVELS_MAX_K + 1][TOR_LEVELS_MAX_K + 1];

struct Binom {
  unsigned long long v[TOR_LEVELS_MAX_K + 1][TOR_LEVELS_MAX_K + 1];
  Binom() {
    memset(v, 0, sizeof(v));
    for (int n = 0; n <= TOR_LEVELS_MAX_K; ++n) {
      v[n][0] = 1ull;
      for (int r = 1; r <= n; ++r) v[n][r] = v[n - 1][r - 1] + (r <= n - 1 ? v[n - 1][r] : 0ull);
    }
  }
};
const Binom &host_binom() {
  static const Binom b;
  return b;
}

// The next smaller mask with the same popcount.  Masks of one popcount in
// decreasing order are their complements in increasing order, so the answer is
// the complement of the smallest larger word with as many ones as ~mask (the
// ones-moving identity of HAKMEM item 175, Gosper): adding the lowest set bit
// carries through the lowest block of ones, leaving one 1 just above the
// block, and the block's other ones return at the bottom.  Undefined for the
// smallest mask of a level (all its ones at the bottom: no smaller mask).
__host__ __device__ inline unsigned long long next_mask(unsigned long long mask) {
  const unsigned long long y = ~mask;
  const unsigned long long low = y & (0ull - y);  // lowest set bit of y
  const unsigned long long r = y + low;           // the block of ones carried up by one place
#if defined(__CUDA_ARCH__)
  const int p = __ffsll((long long)low) - 1;
#else
  const int p = __builtin_ctzll(low);
#endif
  const unsigned long long back = ((y ^ r) >> 2) >> p;  // block length minus one ones, at the bottom
  return ~(r | back);
}

// the r-th (0-based) mask of popcount m over k bits, in decreasing order
__host__ __device__ inline unsigned long long kth_mask(int k, int m, unsigned long long r,
                                                       const unsigned long long (*C)[TOR_LEVELS_MAX_K + 1]) {
  unsigned long long mask = 0ull;
  for (int b = k - 1; b >= 0 && m > 0; --b) {
    const unsigned long long with = C[b][m - 1];  // masks with bit b set and m - 1 ones below it
    if (r < with) {
      mask |= 1ull << b;
      --m;
    } else {
      r -= with;
    }
  }
  return mask;
}

// one level: thread g takes ranks [g per, (g + 1) per) of the C(k, m) masks
template <class Tier>
__global__ void __launch_bounds__(LV_THREADS)
k_level(const double *__restrict__ B, const double *__restrict__ Blo, int k, int m, unsigned long long count,
        unsigned long long per, double *__restrict__ scratch, unsigned long long *__restrict__ part,
        int *__restrict__ status) {
  __shared__ unsigned long long red[LV_THREADS][8];
  const size_t st = (size_t)gridDim.x * blockDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double *S = scratch + gtid;
  const SrcPrepped src{B, Blo, 2 * k};
  SumsOf<Fx256> Sm;
  fx_zero(Sm.tor);
  fx_zero(Sm.sabs);
  Sm.flags = 0;
  const unsigned long long lo = gtid * per;
  const unsigned long long hi = (lo + per < count) ? lo + per : count;
  if (lo < hi) {
    unsigned long long mask = kth_mask(k, m, lo, c_binom);
    for (unsigned long long r = lo; r < hi; ++r) {
      walk_chunk<Tier>(src, k, 0, mask, S, st, Sm, nullptr, 0);  // a fresh elimination of B_Z
      if (r + 1 < hi) mask = next_mask(mask);
    }
  }
  if (Sm.flags) atomicOr(status, Sm.flags);
#pragma unroll
  for (int i = 0; i < 4; ++i) { red[threadIdx.x][i] = Sm.tor.w[i]; red[threadIdx.x][4 + i] = Sm.sabs.w[i]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    Fx256 a, b, x;
    fx_zero(a);
    fx_zero(b);
    for (int t = 0; t < (int)blockDim.x; ++t) {
      for (int i = 0; i < 4; ++i) x.w[i] = red[t][i];
      fx_add(a, x);
      for (int i = 0; i < 4; ++i) x.w[i] = red[t][4 + i];
      fx_add(b, x);
    }
    for (int i = 0; i < 4; ++i) { part[(size_t)blockIdx.x * 8 + i] = a.w[i]; part[(size_t)blockIdx.x * 8 + 4 + i] = b.w[i]; }
  }
}

// all levels' block partials -> one result; the error bound adds each level's
// 4k u(tier) sum t, and the reported tier is the least precise one used
__global__ void k_levels_finalize(const unsigned long long *__restrict__ part, int nlevels, int grid, int k,
                                  const int *__restrict__ tiers, const int *__restrict__ status,
                                  tor_result *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Fx256 a, b, x;
  fx_zero(a);
  fx_zero(b);
  double err = 0.0;
  int worst = tiers[0];
  for (int L = 0; L < nlevels; ++L) {
    Fx256 sl;
    fx_zero(sl);
    for (int j = 0; j < grid; ++j) {
      const unsigned long long *p = part + ((size_t)L * grid + j) * 8;
      for (int i = 0; i < 4; ++i) x.w[i] = p[i];
      fx_add(a, x);
      for (int i = 0; i < 4; ++i) x.w[i] = p[4 + i];
      fx_add(b, x);
      fx_add(sl, x);
    }
    err += err_gamma(k) * unit_roundoff(tiers[L]) * fx_to_double(sl);
    if (unit_roundoff(tiers[L]) > unit_roundoff(worst)) worst = tiers[L];
  }
  unsigned long long w[8];
  for (int i = 0; i < 4; ++i) { w[i] = a.w[i]; w[4 + i] = b.w[i]; }
  fixed_to_result_w<4>(w, k, worst, *status, out);
  out->err_est = err;
}

template <class F>
void with_level_tier(int tier, F &&f) {
  switch (tier) {
    case TOR_PREC_DD: f(TierDD{}); break;
    case TOR_PREC_FX128: f(TierFx<FX128_FRAC>{}); break;
    default: f(TierF64{}); break;
  }
}

int level_grid(int device, int tier) {
  int sms = 0, occ = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  with_level_tier(tier, [&](auto t) {
    using Tier = decltype(t);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_level<Tier>, LV_THREADS, 0) != cudaSuccess) occ = 0;
  });
  if (occ < 1) occ = 1;
  if (occ > 4) occ = 4;
  return sms * occ;
}

// workspace: per-thread elimination stacks (two doubles per entry, the widest
// of the three tiers), per-level block partials, the level tiers, the status
// word and the prepped B = I - O
struct Layout {
  size_t scratch, part, tiers, status, prep, total;
};
Layout layout_of(int k, int grid) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  Layout l;
  l.scratch = al(sizeof(double) * 2 * (size_t)sz(k > 0 ? k : 1) * (size_t)grid * LV_THREADS);
  l.part = al(sizeof(unsigned long long) * 8 * (size_t)(k + 1) * (size_t)grid);
  l.tiers = al(sizeof(int) * (size_t)(k + 1));
  l.status = al(sizeof(int));
  l.prep = al(sizeof(double) * (4 * (size_t)k * k + 2 * (size_t)k + 1));
  l.total = l.scratch + l.part + l.tiers + l.status + l.prep;
  return l;
}

thread_local char g_lv_err[256] = "";
int lv_fail(int code, const char *msg) {
  snprintf(g_lv_err, sizeof(g_lv_err), "%s", msg);
  return code;
}

}  // namespace
}  // namespace tor

extern "C" {

uint64_t tor_level_next_mask(uint64_t mask) {
  if (mask == 0ull || (mask & (mask + 1ull)) == 0ull) return 0ull;  // 0 or the smallest mask: none below
  return tor::next_mask(mask);
}

int tor_level_kth_mask(int k, int m, uint64_t r, uint64_t *mask) {
  if (!mask || k < 0 || k > TOR_LEVELS_MAX_K || m < 0 || m > k) return TOR_EINVAL;
  const auto &C = tor::host_binom().v;
  if (r >= C[k][m]) return TOR_EINVAL;
  *mask = tor::kth_mask(k, m, r, C);
  return TOR_OK;
}

int tor_levels_workspace(int k, int device, size_t *bytes) {
  if (!bytes || k < 0 || k > TOR_LEVELS_MAX_K) return TOR_EINVAL;
  int grid = 0;
  for (int tier = TOR_PREC_FP64; tier <= TOR_PREC_FX128; ++tier) {
    const int g = tor::level_grid(device, tier);
    if (g > grid) grid = g;
  }
  if (grid == 0) return TOR_ECUDA;
  *bytes = tor::layout_of(k, grid).total;
  return TOR_OK;
}

int tor_levels(const double *O, int k, int ld, int layout, int prec, const int *level_prec, void *workspace,
               size_t workspace_bytes, cudaStream_t s, tor_result *out_dev) {
  using namespace tor;
  if (k < 0 || k > TOR_LEVELS_MAX_K) return lv_fail(TOR_EINVAL, "k outside [0, TOR_LEVELS_MAX_K]");
  if ((k > 0 && !O) || !out_dev || !workspace) return lv_fail(TOR_EINVAL, "null pointer");
  if (k > 0 && ld < 2 * k) return lv_fail(TOR_EINVAL, "ld < 2k");
  if (layout != TOR_LAYOUT_XXPP && layout != TOR_LAYOUT_XPXP) return lv_fail(TOR_EINVAL, "bad layout");
  int tiers[TOR_LEVELS_MAX_K + 1];
  for (int L = 0; L <= k; ++L) {
    tiers[L] = level_prec ? level_prec[L] : prec;
    if (tiers[L] != TOR_PREC_FP64 && tiers[L] != TOR_PREC_DD && tiers[L] != TOR_PREC_FX128)
      return lv_fail(TOR_EINVAL, "level tiers must be TOR_PREC_FP64, TOR_PREC_DD or TOR_PREC_FX128");
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return lv_fail(TOR_ECUDA, "cudaGetDevice failed");
  int grid = 0;
  for (int tier = TOR_PREC_FP64; tier <= TOR_PREC_FX128; ++tier) {
    const int g = level_grid(device, tier);
    if (g > grid) grid = g;
  }
  if (grid == 0) return lv_fail(TOR_ECUDA, "device query failed");
  const Layout lay = layout_of(k, grid);
  if (workspace_bytes < lay.total) return lv_fail(TOR_EINVAL, "workspace smaller than tor_levels_workspace");
  char *base = (char *)workspace;
  double *scratch = (double *)base;
  unsigned long long *part = (unsigned long long *)(base + lay.scratch);
  int *tiers_dev = (int *)(base + lay.scratch + lay.part);
  int *status = (int *)(base + lay.scratch + lay.part + lay.tiers);
  double *Bp = (double *)(base + lay.scratch + lay.part + lay.tiers + lay.status);
  double *Blo = Bp + 4 * (size_t)k * k;
  if (k == 0) {  // the empty pattern: only Z = {} with t = 1
    const tor_result one = {1.0, 0.0, 1.0, 0.0, tiers[0], TOR_OK};
    if (cudaMemcpyAsync(out_dev, &one, sizeof(one), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return lv_fail(TOR_ECUDA, "result copy failed");
    return TOR_OK;
  }
  {
    static std::mutex mu;  // the binomial table is a per-device constant, the same for every call
    std::lock_guard<std::mutex> lk(mu);
    if (cudaMemcpyToSymbolAsync(c_binom, host_binom().v, sizeof(host_binom().v), 0, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return lv_fail(TOR_ECUDA, "binomial table upload failed");
  }
  if (cudaMemcpyAsync(tiers_dev, tiers, sizeof(int) * (size_t)(k + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
    return lv_fail(TOR_ECUDA, "workspace setup failed");
  launch_prep(O, k, ld, layout, Bp, Blo, s);
  if (cudaGetLastError() != cudaSuccess) return lv_fail(TOR_ECUDA, "prep launch failed");
  const unsigned long long threads = (unsigned long long)grid * LV_THREADS;
  const auto &C = host_binom().v;
  for (int m = 0; m <= k; ++m) {  // Algorithm 1: one level |Z| = m at a time
    const unsigned long long count = C[k][m];
    const unsigned long long per = (count + threads - 1) / threads;
    unsigned long long *pl = part + (size_t)m * grid * 8;
    with_level_tier(tiers[m], [&](auto t) {
      using Tier = decltype(t);
      k_level<Tier><<<grid, LV_THREADS, 0, s>>>(Bp, Blo, k, m, count, per, scratch, pl, status);
    });
    if (cudaGetLastError() != cudaSuccess) return lv_fail(TOR_ECUDA, "level launch failed");
  }
  k_levels_finalize<<<1, 32, 0, s>>>(part, k + 1, grid, k, tiers_dev, status, out_dev);
  if (cudaGetLastError() != cudaSuccess) return lv_fail(TOR_ECUDA, "finalize launch failed");
  return TOR_OK;
}

const char *tor_levels_last_error(void) { return tor::g_lv_err; }

}  // extern "C"
