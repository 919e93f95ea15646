// capi.cu -- the C ABI (include/torontonian.h): context, workspace, entry points.
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <new>
#include <cstdlib>
#include <cmath>
#include <vector>
#include "tor_internal.h"
#include "tor_walk.cuh"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(TOR_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                   \
  } while (0)

struct Buf {
  void *p = nullptr;
  size_t cap = 0;
};

}  // namespace

int tor::record_error(int code, const char *msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
  return code;
}

struct tor_ctx {
  int device = 0;
  int sms = 0;
  int threads_per_block = 128;
  int blocks_per_sm = 4;  // clamped to the kernel's occupancy at launch
  int chunk_bits = -1;  // -1: automatic
  Buf B, Blo, scratch, block_part, status, result, total8, bound;
  bool timing = false, timed = false, transform_timed = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  // batch workspace (tor_batch_reserve)
  int batch_nmax = 0, batch_kmax = -1;
  bool batch_explicit = false;  // sized by the caller's tor_batch_reserve: never re-read k
  Buf batch, batch_scratch;
  tor::BatchPlan plan{};
  tor_bound *bounds_dev = nullptr;
  unsigned char *r1_table_dev = nullptr;
  int *k_dev = nullptr;  // pattern mode: click counts
  Buf mh;                // sampler: proposals, their log q, their Torontonians
  Buf table, table_s, order;  // all-pattern table: exact terms, sums of terms, walk order
  int order_r1 = -1;          // walked modes the order table was made for
  unsigned char r1_table[5][65];  // walked modes per chunk, by tier (TOR_PREC_*) and k
  // autotuned single-instance settings by tier and k (-1: not tuned)
  signed char tuned_d[5][65];   // by tier (TOR_PREC_FP64 .. TOR_PREC_FX256) and k
  signed char tuned_bps[5][65];
};

namespace {

int ensure(tor_ctx *c, Buf &b, size_t bytes) {
  if (b.cap >= bytes) return TOR_OK;
  if (b.p) {
    CK(cudaDeviceSynchronize());
    CK(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(TOR_ENOMEM, "workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  b.cap = bytes;
  (void)c;
  return TOR_OK;
}

// chunk bits d (chunks fix the high d modes); r1 = k - d modes are walked per chunk
int choose_chunk_bits(const tor_ctx *c, int k, int tier = TOR_PREC_FP64) {
  if (c->chunk_bits >= 0) return c->chunk_bits < k ? c->chunk_bits : k;
  if (k <= 64 && c->tuned_d[tier][k] >= 0) return c->tuned_d[tier][k];
  // 2^16 chunks fill a 152-SM grid (about 58k threads) with one to two rounds;
  // beyond k = 32 the chunks stay at 16 walked modes, where a chunk's root (the
  // elimination of its fixed modes) costs a few percent of its walk.  The
  // autotuner's choices at k = 28, 30, 32 on GB300 are d = 15, 16, 16.
  int d = k - 16;
  const int fill = (k - 8 < 16) ? k - 8 : 16;
  if (d < fill) d = fill;
  if (d > 40) d = 40;
  if (d < 0) d = 0;
  return d;
}

int check_common(tor_ctx *ctx, const void *O, int k, int ld, int layout) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (k < 0 || k > TOR_MAX_K) return fail(TOR_EINVAL, "k = %d outside [0, %d]", k, TOR_MAX_K);
  if (k > 0 && !O) return fail(TOR_EINVAL, "null matrix pointer");
  if (k > 0 && ld < 2 * k) return fail(TOR_EINVAL, "ld = %d < 2k = %d", ld, 2 * k);
  if (layout != TOR_LAYOUT_XXPP && layout != TOR_LAYOUT_XPXP) return fail(TOR_EINVAL, "bad layout %d", layout);
  return TOR_OK;
}

// threads of the walk grid: every block must be resident at once, because
// chunks are dealt out by a grid stride and a block that waited for a free SM
// would double the time
int walk_grid(tor_ctx *ctx, int tier) {
  const int occ = tor::dfs_max_blocks_per_sm(tier, ctx->threads_per_block);
  return ctx->sms * (ctx->blocks_per_sm < occ ? ctx->blocks_per_sm : occ);
}

// walked modes per chunk of an FP64 batch item (the other tiers use 12); on
// 4096 patterns with k in [8, 30]: 95.3 Tor/s at 16, 92.9 at 14, 83.7 at 12
#ifndef TOR_BATCH_R1_F64
#define TOR_BATCH_R1_F64 16
#endif

// walked modes per chunk of a 256-bit batch item: at 12 the chunk roots of a
// k = 30 instance add about 9 % to its walk, at 16 about 1 % (the
// single-instance autotuner picks 16 at k = 32)
#ifndef TOR_BATCH_R1_FX256
#define TOR_BATCH_R1_FX256 16
#endif

#ifndef TOR_TAIL_SPLIT
#define TOR_TAIL_SPLIT 1
#endif

// Segments for all 2^d chunks on T threads.  The chunks are equal in cost, so
// the grid-stride loop takes ceil(2^d / T) rounds and a partial last round
// leaves threads idle.  Only the full rounds W = floor(2^d / T) stay at d
// bits; the R leftover chunks are cut e bits finer (2^e sub-chunks each, e
// from a cost model) and walked as a second segment by the whole grid.  The
// sub-chunks cover the same subsets as their parent chunk; only the rounding
// of their terms changes, because each root eliminates e more modes before
// the walk starts.
tor::WalkSegs plan_segments(int k, int d, size_t T) {
  const int r1 = k - d;
  const unsigned long long n = 1ull << d;
  const unsigned long long W = n / T, R = n - W * T;
  if (!TOR_TAIL_SPLIT || W == 0 || R == 0 || r1 < 2) return tor::one_segment(r1, 0ull, n);
  // cost of one chunk of r low modes, in FMAs: 27.5 per walked subset plus the
  // root, about 2 m^2 for each of the k - r fixed modes (half are eliminated)
  auto cost = [k](int r) {
    double root = 0.0;
    for (int m = r; m < k; ++m) root += 2.0 * m * m;
    return 27.5 * std::ldexp(1.0, r) + root;
  };
  int best_e = 0;
  double best = cost(r1);  // e = 0: one more full-size round
  for (int e = 1; e <= 3 && e < r1; ++e) {
    const double rounds = std::ceil((double)(R << e) / (double)T);
    const double c = rounds * cost(r1 - e);
    if (c < best) { best = c; best_e = e; }
  }
  if (best_e == 0) return tor::one_segment(r1, 0ull, n);
  tor::WalkSegs g;
  g.r1[0] = r1;       g.c0[0] = 0ull;                g.c1[0] = W * T;
  g.r1[1] = r1 - best_e; g.c0[1] = (W * T) << best_e; g.c1[1] = n << best_e;
  return g;
}

// enqueue prep + walk over the segments; block partials in ctx->block_part
int enqueue_walk(tor_ctx *ctx, const double *O, int k, int ld, int layout, int tier, const tor::WalkSegs &seg,
                 unsigned long long *chunk_part, cudaStream_t s, int grid) {
  const int block = ctx->threads_per_block;
  const int r1 = seg.r1[0];  // the larger of the two
  const size_t nthreads = (size_t)grid * block;
  int rc;
  if ((rc = ensure(ctx, ctx->B, sizeof(double) * 4 * (size_t)k * k))) return rc;
  if ((rc = ensure(ctx, ctx->Blo, sizeof(double) * 2 * (size_t)k))) return rc;
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * nthreads * (size_t)tor::scratch_entries(tier, k, r1)))) return rc;
  if ((rc = ensure(ctx, ctx->block_part, sizeof(unsigned long long) * 16 * (size_t)grid))) return rc;
  if ((rc = ensure(ctx, ctx->status, sizeof(int)))) return rc;
  tor::launch_prep(O, k, ld, layout, (double *)ctx->B.p, (double *)ctx->Blo.p, s);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), s));
  if (ctx->timing) CK(cudaEventRecord(ctx->ev0, s));
  tor::launch_dfs(tier, grid, block, (const double *)ctx->B.p, (const double *)ctx->Blo.p, k, seg,
                  (double *)ctx->scratch.p, (unsigned long long *)ctx->block_part.p, chunk_part,
                  (int *)ctx->status.p, s);
  CK(cudaGetLastError());
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev1, s));
    ctx->timed = true;
  }
  return TOR_OK;
}

int pick_tier(int prec) {
  if (prec == TOR_PREC_DD) return TOR_PREC_DD;
  return TOR_PREC_FP64;
}

}  // namespace

extern "C" {

const char *tor_last_error(void) { return g_err; }

int tor_create(tor_ctx **out, int device) {
  if (!out) return fail(TOR_EINVAL, "null output pointer");
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(TOR_EINVAL, "device %d outside [0, %d)", device, ndev);
  CK(cudaSetDevice(device));
  tor_ctx *c = new (std::nothrow) tor_ctx();
  if (!c) return fail(TOR_ENOMEM, "host allocation failed");
  c->device = device;
  memset(c->tuned_d, -1, sizeof(c->tuned_d));
  memset(c->tuned_bps, -1, sizeof(c->tuned_bps));
  for (int kk = 0; kk <= 64; ++kk) {
    c->r1_table[0][kk] = 0;
    c->r1_table[TOR_PREC_FP64][kk] = (unsigned char)(kk < TOR_BATCH_R1_F64 ? kk : TOR_BATCH_R1_F64);
    c->r1_table[TOR_PREC_DD][kk] = (unsigned char)(kk < 12 ? kk : 12);
    c->r1_table[TOR_PREC_FX128][kk] = (unsigned char)(kk < 12 ? kk : 12);
    c->r1_table[TOR_PREC_FX256][kk] = (unsigned char)(kk < TOR_BATCH_R1_FX256 ? kk : TOR_BATCH_R1_FX256);
  }
  cudaError_t e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return fail(TOR_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
  }
  *out = c;
  return TOR_OK;
}

void tor_destroy(tor_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  Buf *bufs[] = {&c->B, &c->Blo, &c->scratch, &c->block_part, &c->status, &c->result, &c->total8, &c->bound,
                 &c->batch, &c->batch_scratch, &c->mh, &c->table, &c->table_s, &c->order};
  for (Buf *b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev2) cudaEventDestroy(c->ev2);
  if (c->ev3) cudaEventDestroy(c->ev3);
  delete c;
}

int tor_set_timing(tor_ctx *ctx, int on) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  CK(cudaSetDevice(ctx->device));
  if (on && !ctx->ev0) {
    CK(cudaEventCreate(&ctx->ev0));
    CK(cudaEventCreate(&ctx->ev1));
    CK(cudaEventCreate(&ctx->ev2));
    CK(cudaEventCreate(&ctx->ev3));
  }
  ctx->timing = on != 0;
  ctx->timed = false;
  ctx->transform_timed = false;
  return TOR_OK;
}

int tor_transform_time(tor_ctx *ctx, float *ms) {
  if (!ctx || !ms) return fail(TOR_EINVAL, "null pointer");
  if (!ctx->transform_timed) return fail(TOR_EINVAL, "no timed tor_all_patterns call since timing was enabled");
  CK(cudaEventSynchronize(ctx->ev3));
  CK(cudaEventElapsedTime(ms, ctx->ev2, ctx->ev3));
  return TOR_OK;
}

int tor_walk_time(tor_ctx *ctx, float *ms) {
  if (!ctx || !ms) return fail(TOR_EINVAL, "null pointer");
  if (!ctx->timed) return fail(TOR_EINVAL, "no timed call since timing was enabled");
  CK(cudaEventSynchronize(ctx->ev1));
  CK(cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
  return TOR_OK;
}

int tor_set_launch(tor_ctx *ctx, int threads_per_block, int blocks_per_sm) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (threads_per_block == 0) threads_per_block = 128;
  if (blocks_per_sm == 0) blocks_per_sm = 4;
  if (threads_per_block != 32 && threads_per_block != 64 && threads_per_block != 128)
    return fail(TOR_EINVAL, "threads_per_block must be 32, 64 or 128");
  if (blocks_per_sm < 1 || blocks_per_sm > 16) return fail(TOR_EINVAL, "blocks_per_sm outside [1, 16]");
  ctx->threads_per_block = threads_per_block;
  ctx->blocks_per_sm = blocks_per_sm;
  return TOR_OK;
}

int tor_set_chunk_bits(tor_ctx *ctx, int chunk_bits) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (chunk_bits < -1 || chunk_bits > 40) return fail(TOR_EINVAL, "chunk_bits outside [-1, 40]");
  ctx->chunk_bits = chunk_bits;
  return TOR_OK;
}

int tor_single_async(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec,
                     cudaStream_t s, tor_result *out_dev) {
  int rc = check_common(ctx, O, k, ld, layout);
  if (rc) return rc;
  if (!out_dev) return fail(TOR_EINVAL, "null result pointer");
  if (prec < TOR_PREC_FP64 || prec > TOR_PREC_FX256)
    return fail(TOR_EINVAL, "tor_single_async needs an explicit tier (TOR_PREC_FP64 .. TOR_PREC_FX256)");
  CK(cudaSetDevice(ctx->device));
  if (k == 0) {  // Tor = 1 (only the empty set), written on the stream: stays asynchronous
    if (tor::launch_result_one(out_dev, prec, s))
      return fail(TOR_ECUDA, "k = 0 result: %s", cudaGetErrorString(cudaGetLastError()));
    return TOR_OK;
  }
  const int d = choose_chunk_bits(ctx, k, prec);
  if (prec == TOR_PREC_FX256 && k - d > tor::FX256_MAX_R1)
    return fail(TOR_EINVAL, "256-bit chunks walk at most %d modes (k - chunk_bits = %d)", tor::FX256_MAX_R1, k - d);
  const int bps_saved = ctx->blocks_per_sm;
  if (ctx->chunk_bits < 0 && ctx->tuned_bps[prec][k] > 0) ctx->blocks_per_sm = ctx->tuned_bps[prec][k];
  const int grid = walk_grid(ctx, prec);
  ctx->blocks_per_sm = bps_saved;
  const tor::WalkSegs seg = plan_segments(k, d, (size_t)grid * ctx->threads_per_block);
  rc = enqueue_walk(ctx, O, k, ld, layout, prec, seg, nullptr, s, grid);
  if (rc) return rc;
  tor::launch_finalize((const unsigned long long *)ctx->block_part.p, grid, k, prec,
                       (const int *)ctx->status.p, out_dev, s);
  CK(cudaGetLastError());
  return TOR_OK;
}

// run one tier synchronously into *out
static int single_sync(tor_ctx *ctx, const double *O, int k, int ld, int layout, int tier, cudaStream_t s,
                       tor_result *out) {
  int rc;
  if ((rc = ensure(ctx, ctx->result, sizeof(tor_result)))) return rc;
  if ((rc = tor_single_async(ctx, O, k, ld, layout, tier, s, (tor_result *)ctx->result.p))) return rc;
  CK(cudaMemcpyAsync(out, ctx->result.p, sizeof(tor_result), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return TOR_OK;
}

int tor_single(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec, double tol,
               cudaStream_t s, tor_result *out) {
  int rc = check_common(ctx, O, k, ld, layout);
  if (rc) return rc;
  if (!out) return fail(TOR_EINVAL, "null result pointer");
  if (prec < TOR_PREC_AUTO || prec > TOR_PREC_FX256) return fail(TOR_EINVAL, "bad precision %d", prec);
  int tier = prec;
  if ((prec == TOR_PREC_FX128 || prec == TOR_PREC_FX256) && k > 0) {  // 1/det2 <= t_max^2 must fit
    CK(cudaSetDevice(ctx->device));
    if ((rc = ensure(ctx, ctx->bound, sizeof(tor_bound)))) return rc;
    if (tor::launch_bounds_single(O, k, ld, layout, 1e-10, (tor_bound *)ctx->bound.p, s))
      return fail(TOR_ECUDA, "bound pass launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    tor_bound bd;
    CK(cudaMemcpyAsync(&bd, ctx->bound.p, sizeof(bd), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const float lim = (prec == TOR_PREC_FX128) ? tor::FX128_MAX_LOG2_TMAX : tor::FX256_MAX_LOG2_TMAX;
    if (!(bd.log_tmax <= lim * 0.6931472f))
      return fail(TOR_EINVAL, "instance outside the %d-bit fixed-point range (log2 t_max = %.2f > %.0f)",
                  prec == TOR_PREC_FX128 ? 128 : 256, (double)bd.log_tmax / 0.6931472, (double)lim);
  }
  bool fx_ok = false, fx256_ok = false;  // t_max inside the 128-bit / 256-bit fixed-point range
  if (prec == TOR_PREC_AUTO) {
    if (!(tol > 0.0)) return fail(TOR_EINVAL, "TOR_PREC_AUTO needs a tolerance tol > 0");
    tier = TOR_PREC_FP64;
    if (k > 0) {  // FP32 bound pass picks the starting tier
      CK(cudaSetDevice(ctx->device));
      if ((rc = ensure(ctx, ctx->bound, sizeof(tor_bound)))) return rc;
      if (tor::launch_bounds_single(O, k, ld, layout, tol, (tor_bound *)ctx->bound.p, s))
        return fail(TOR_ECUDA, "bound pass launch failed: %s", cudaGetErrorString(cudaGetLastError()));
      tor_bound bd;
      CK(cudaMemcpyAsync(&bd, ctx->bound.p, sizeof(bd), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      tier = bd.tier;
      fx_ok = bd.log_tmax <= tor::FX128_MAX_LOG2_TMAX * 0.6931472f;
      fx256_ok = bd.log_tmax <= tor::FX256_MAX_LOG2_TMAX * 0.6931472f;
    }
  }
  while (true) {
    if ((rc = single_sync(ctx, O, k, ld, layout, tier, s, out))) return rc;
    if (out->status != TOR_OK)
      return fail(out->status, "instance status %d (%s)", out->status,
                  out->status == TOR_ENOTPD ? "some I - O_Z is not positive definite" : "term out of range");
    if (prec != TOR_PREC_AUTO) return TOR_OK;
    const double mag = out->hi < 0 ? -out->hi : out->hi;
    if (out->err_est <= tol * mag) return TOR_OK;
    // a-posteriori escalation to the next tier with more precision that fits:
    // FP64 (53 bits) -> 128-bit fixed point (100) or double-double (104) ->
    // 256-bit fixed point (186); double-double adds only 4 bits to the 128-bit
    // fixed point, so that step goes straight to 256 bits when it can
    int next = 0;
    if (tier == TOR_PREC_FP64) next = fx_ok ? TOR_PREC_FX128 : (fx256_ok ? TOR_PREC_FX256 : TOR_PREC_DD);
    else if (tier == TOR_PREC_FX128) next = fx256_ok ? TOR_PREC_FX256 : TOR_PREC_DD;
    else if (tier == TOR_PREC_DD) next = fx256_ok ? TOR_PREC_FX256 : 0;
    if (next == 0)
      return fail(TOR_EPREC, "error bound %.3e exceeds tol * |Tor| = %.3e in the most precise tier that fits",
                  out->err_est, tol * mag);
    tier = next;
  }
}

int tor_chunks(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec, int chunk_bits,
               uint64_t c_begin, uint64_t c_end, cudaStream_t s, uint64_t *part_dev) {
  int rc = check_common(ctx, O, k, ld, layout);
  if (rc) return rc;
  if (k == 0) return fail(TOR_EINVAL, "tor_chunks needs k >= 1");
  if (prec < TOR_PREC_FP64 || prec > TOR_PREC_FX256) return fail(TOR_EINVAL, "prec must be an explicit tier");
  if (chunk_bits < 0 || chunk_bits > k || chunk_bits > 63) return fail(TOR_EINVAL, "chunk_bits outside [0, min(k, 63)]");
  if (!part_dev) return fail(TOR_EINVAL, "null partials pointer");
  if (prec == TOR_PREC_FX256 && k - chunk_bits > tor::FX256_MAX_R1)
    return fail(TOR_EINVAL, "256-bit chunks walk at most %d modes (k - chunk_bits = %d)", tor::FX256_MAX_R1,
                k - chunk_bits);
  const uint64_t nchunks = 1ull << chunk_bits;
  if (c_begin > c_end || c_end > nchunks) return fail(TOR_EINVAL, "chunk range [%llu, %llu) outside [0, %llu)",
                                                     (unsigned long long)c_begin, (unsigned long long)c_end,
                                                     (unsigned long long)nchunks);
  if (c_begin == c_end) return TOR_OK;
  CK(cudaSetDevice(ctx->device));
  return enqueue_walk(ctx, O, k, ld, layout, prec, tor::one_segment(k - chunk_bits, c_begin, c_end),
                      (unsigned long long *)part_dev, s, walk_grid(ctx, prec));
}

int tor_fx256_fma2(const int32_t *s_dev, const int32_t *a1_dev, const int32_t *b1_dev, const int32_t *a2_dev,
                   const int32_t *b2_dev, int n, int32_t *out_dev, int *ovf_dev, cudaStream_t stream) {
  if (n < 0) return fail(TOR_EINVAL, "n = %d < 0", n);
  if (n > 0 && (!s_dev || !a1_dev || !b1_dev || !a2_dev || !b2_dev || !out_dev || !ovf_dev))
    return fail(TOR_EINVAL, "null pointer");
  if (tor::launch_fx256_fma2(s_dev, a1_dev, b1_dev, a2_dev, b2_dev, n, out_dev, ovf_dev, stream))
    return fail(TOR_ECUDA, "launch: %s", cudaGetErrorString(cudaGetLastError()));
  return TOR_OK;
}

// low-mode masks of a chunk's terms in the order the walk visits them: the
// chunk root (no low mode) first, then depth first, a node's children pivoting
// on its remaining modes from the highest down, each child's own term before
// its subtree, a child keeping the modes above its pivot
static void walk_order(unsigned int mask, int q, int r1, std::vector<unsigned int> &seq) {
  for (int cur = 0; cur < r1 - q; ++cur) {
    const int p = r1 - 1 - cur;
    const unsigned int m2 = mask | (1u << p);
    seq.push_back(m2);
    walk_order(m2, p + 1, r1, seq);
  }
}

int tor_all_patterns(tor_ctx *ctx, const double *O, int M, int ld, int prec, cudaStream_t s, tor_result *out_dev) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (M < 1 || M > TOR_TABLE_MAX_M) return fail(TOR_EINVAL, "M = %d outside [1, %d]", M, TOR_TABLE_MAX_M);
  if (!O || !out_dev) return fail(TOR_EINVAL, "null pointer");
  if (ld < 2 * M) return fail(TOR_EINVAL, "ld = %d < 2M = %d", ld, 2 * M);
  if (prec != TOR_PREC_FP64 && prec != TOR_PREC_DD && prec != TOR_PREC_FX128)
    return fail(TOR_EINVAL, "prec must be TOR_PREC_FP64, TOR_PREC_DD or TOR_PREC_FX128");
  CK(cudaSetDevice(ctx->device));
  int rc;
  const int k = M;
  if (prec == TOR_PREC_FX128) {  // every subset's t_max is at most the full state's
    if ((rc = ensure(ctx, ctx->bound, sizeof(tor_bound)))) return rc;
    if (tor::launch_bounds_single(O, k, ld, TOR_LAYOUT_XXPP, 1e-10, (tor_bound *)ctx->bound.p, s))
      return fail(TOR_ECUDA, "bound pass launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    tor_bound bd;
    CK(cudaMemcpyAsync(&bd, ctx->bound.p, sizeof(bd), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!(bd.log_tmax <= tor::FX128_MAX_LOG2_TMAX * 0.6931472f))
      return fail(TOR_EINVAL, "state outside the 128-bit fixed-point range (log2 t_max = %.2f)",
                  (double)bd.log_tmax / 0.6931472);
  }
  // walked modes per chunk: at least 2^16 chunks to fill the grid, at most 12
  // modes (a 4096-entry walk-order table)
  int r1 = k - 16;
  if (r1 > 12) r1 = 12;
  if (r1 < 0) r1 = 0;
  const int block = ctx->threads_per_block;
  const int occ = tor::table_walk_max_blocks_per_sm(prec, block);
  const int grid = ctx->sms * (ctx->blocks_per_sm < occ ? ctx->blocks_per_sm : occ);
  const size_t nthreads = (size_t)grid * block;
  const size_t n = (size_t)1 << M;
  if ((rc = ensure(ctx, ctx->B, sizeof(double) * 4 * (size_t)k * k))) return rc;
  if ((rc = ensure(ctx, ctx->Blo, sizeof(double) * 2 * (size_t)k))) return rc;
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * nthreads * (size_t)tor::scratch_entries(prec, k, r1)))) return rc;
  if ((rc = ensure(ctx, ctx->status, sizeof(int)))) return rc;
  if ((rc = ensure(ctx, ctx->table, sizeof(tor::Fx256) * n))) return rc;
  if ((rc = ensure(ctx, ctx->table_s, sizeof(double) * n))) return rc;
  if ((rc = ensure(ctx, ctx->order, sizeof(unsigned int) << r1))) return rc;
  if (ctx->order_r1 != r1) {
    std::vector<unsigned int> seq;
    seq.reserve((size_t)1 << r1);
    seq.push_back(0u);
    walk_order(0u, 0, r1, seq);
    if (seq.size() != ((size_t)1 << r1)) return fail(TOR_ECUDA, "walk order of %zu entries", seq.size());
    CK(cudaMemcpyAsync(ctx->order.p, seq.data(), sizeof(unsigned int) << r1, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // seq is a local
    ctx->order_r1 = r1;
  }
  tor::launch_prep(O, k, ld, TOR_LAYOUT_XXPP, (double *)ctx->B.p, (double *)ctx->Blo.p, s);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), s));
  if (ctx->timing) CK(cudaEventRecord(ctx->ev0, s));
  if (tor::launch_table_walk(prec, grid, block, (const double *)ctx->B.p, (const double *)ctx->Blo.p, k, r1,
                             (double *)ctx->scratch.p, (const unsigned int *)ctx->order.p,
                             (tor::Fx256 *)ctx->table.p, (int *)ctx->status.p, s))
    return fail(TOR_ECUDA, "table walk: %s", cudaGetErrorString(cudaGetLastError()));
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev1, s));
    ctx->timed = true;
  }
  if (ctx->timing) CK(cudaEventRecord(ctx->ev2, s));
  if (tor::launch_table_transform((tor::Fx256 *)ctx->table.p, (double *)ctx->table_s.p, M, s))
    return fail(TOR_ECUDA, "table transform: %s", cudaGetErrorString(cudaGetLastError()));
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev3, s));
    ctx->transform_timed = true;
  }
  if (tor::launch_table_finalize((const tor::Fx256 *)ctx->table.p, (const double *)ctx->table_s.p, M, prec,
                                 (const int *)ctx->status.p, out_dev, s))
    return fail(TOR_ECUDA, "table finalize: %s", cudaGetErrorString(cudaGetLastError()));
  return TOR_OK;
}

int tor_fixed_to_result(const uint64_t *limbs, int k, int tier, tor_result *out) {
  if (!limbs || !out) return fail(TOR_EINVAL, "null pointer");
  if (tier < TOR_PREC_FP64 || tier > TOR_PREC_FX256) return fail(TOR_EINVAL, "bad tier");
  tor::fixed_to_result((const unsigned long long *)limbs, k, tier, 0, out);
  return TOR_OK;
}

static int batch_grid(const tor_ctx *ctx, int tier, bool patterns = false) {
  const int occ = tor::batch_walk_max_blocks_per_sm(tier, ctx->threads_per_block, patterns);
  return ctx->sms * (ctx->blocks_per_sm < occ ? ctx->blocks_per_sm : occ);
}

static int batch_reserve(tor_ctx *ctx, int n_max, int k_max);

int tor_batch_reserve(tor_ctx *ctx, int n_max, int k_max) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  const int rc = batch_reserve(ctx, n_max, k_max);
  if (rc == TOR_OK) ctx->batch_explicit = true;
  return rc;
}

static int batch_reserve(tor_ctx *ctx, int n_max, int k_max) {
  if (n_max < 1) return fail(TOR_EINVAL, "n_max = %d < 1", n_max);
  if (k_max < 0 || k_max > TOR_MAX_K) return fail(TOR_EINVAL, "k_max = %d outside [0, %d]", k_max, TOR_MAX_K);
  CK(cudaSetDevice(ctx->device));
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t n = (size_t)n_max;
  const size_t sz_tier = al(n), sz_r1 = al(n), sz_esc = al(n), sz_key = al(4 * n), sz_order = al(4 * n),
               sz_flags = al(4 * n), sz_off = al(8 * (n + 1)), sz_acc = al(128 * n), sz_range = al(64),
               sz_counter = al(32), sz_counts = al(16), sz_result = al(sizeof(tor_result) * n),
               sz_bounds = al(sizeof(tor_bound) * n), sz_r1tab = al(5 * 65), sz_k = al(4 * n);
  const size_t total = sz_tier + sz_r1 + sz_esc + sz_key + sz_order + sz_flags + sz_off + sz_acc + sz_range +
                       sz_counter + sz_counts + sz_result + sz_bounds + sz_r1tab + sz_k;
  int rc;
  if ((rc = ensure(ctx, ctx->batch, total))) return rc;
  unsigned char *b = (unsigned char *)ctx->batch.p;
  tor::BatchPlan &p = ctx->plan;
  p.tier = b; b += sz_tier;
  p.r1 = b; b += sz_r1;
  p.escalated = b; b += sz_esc;
  p.key = (int *)b; b += sz_key;
  p.order = (int *)b; b += sz_order;
  p.flags = (int *)b; b += sz_flags;
  p.item_off = (unsigned long long *)b; b += sz_off;
  p.acc = (unsigned long long *)b; b += sz_acc;
  p.range = (unsigned long long *)b; b += sz_range;
  p.counter = (unsigned long long *)b; b += sz_counter;
  p.counts = (unsigned int *)b; b += sz_counts;
  p.result = (tor_result *)b; b += sz_result;
  ctx->bounds_dev = (tor_bound *)b; b += sz_bounds;
  ctx->r1_table_dev = b; b += sz_r1tab;
  ctx->k_dev = (int *)b;
  CK(cudaMemcpy(ctx->r1_table_dev, ctx->r1_table, sizeof(ctx->r1_table), cudaMemcpyHostToDevice));
  // per-thread walk stacks for the largest instance, for any tier
  size_t scratch = 0;
  for (int tier = TOR_PREC_FP64; tier <= TOR_PREC_FX256; ++tier) {
    int r1max = 0;
    for (int kk = 0; kk <= k_max; ++kk) r1max = ctx->r1_table[tier][kk] > r1max ? ctx->r1_table[tier][kk] : r1max;
    const int g0 = batch_grid(ctx, tier, false), g1 = batch_grid(ctx, tier, true);
    const size_t nth = (size_t)(g0 > g1 ? g0 : g1) * ctx->threads_per_block;
    const size_t bytes = sizeof(double) * nth * (size_t)tor::scratch_entries(tier, k_max, r1max);
    scratch = bytes > scratch ? bytes : scratch;
  }
  if ((rc = ensure(ctx, ctx->batch_scratch, scratch))) return rc;
  ctx->batch_nmax = n_max;
  ctx->batch_kmax = k_max;
  return TOR_OK;
}

// enqueue bound pass (AUTO), plan, walks, finalize, and the AUTO second round
// kcap < 0: instances up to the reserved k_max; else also refuse k > kcap (no work, TOR_EINVAL)
static int batch_enqueue(tor_ctx *ctx, const tor::BatchInput &in, int n, int prec, double tol, cudaStream_t s,
                         tor_result *out, int kcap = -1) {
  const tor::BatchPlan &p = ctx->plan;
  const bool pat = in.words > 0;
  const int block = ctx->threads_per_block;
  double *scratch = (double *)ctx->batch_scratch.p;
  const tor_bound *bd = nullptr;
  if (prec == TOR_PREC_AUTO || prec == TOR_PREC_FX128 || prec == TOR_PREC_FX256) {  // tiers, fixed-point ranges
    const int rc = pat ? tor::launch_bounds_patterns(in.Ofull, in.M, in.ldfull, in.patterns, in.words, n, tol,
                                                     ctx->bounds_dev, s)
                       : tor::launch_bounds_batch(in.O, in.k, in.ld, n, in.layout, tol, ctx->bounds_dev, s);
    if (rc) return fail(TOR_ECUDA, "bound pass: %s", cudaGetErrorString(cudaGetLastError()));
    bd = ctx->bounds_dev;
  }
  const int kmax = (kcap >= 0 && kcap < ctx->batch_kmax) ? kcap : ctx->batch_kmax;
  if (tor::launch_batch_plan(in.k, bd, n, prec, kmax, ctx->r1_table_dev, 0, tol, p, s))
    return fail(TOR_ECUDA, "plan: %s", cudaGetErrorString(cudaGetLastError()));
  for (int tier = TOR_PREC_FP64; tier <= TOR_PREC_FX256; ++tier) {
    if (prec != TOR_PREC_AUTO && prec != tier) continue;
    if (tor::launch_batch_walk(tier, batch_grid(ctx, tier, pat), block, in, p, scratch, s))
      return fail(TOR_ECUDA, "walk: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if (tor::launch_batch_finalize(in.k, n, 0, 0.0, p, out, s))
    return fail(TOR_ECUDA, "finalize: %s", cudaGetErrorString(cudaGetLastError()));
  if (prec == TOR_PREC_AUTO) {
    // results that miss tol go to the next tier with more precision whose
    // range holds them: FP64 -> 128-bit -> 256-bit fixed point (double-double
    // outside the fixed-point ranges); the last finalize marks what still
    // misses tol with TOR_EPREC.  Walks with no escalated item return at once.
    for (int round = 1; round <= 2; ++round) {
      if (tor::launch_batch_plan(in.k, bd, n, prec, kmax, ctx->r1_table_dev, 1, tol, p, s))
        return fail(TOR_ECUDA, "AUTO round %d plan: %s", round, cudaGetErrorString(cudaGetLastError()));
      for (int tier : {TOR_PREC_FX128, TOR_PREC_FX256, TOR_PREC_DD})
        if (tor::launch_batch_walk(tier, batch_grid(ctx, tier, pat), block, in, p, scratch, s))
          return fail(TOR_ECUDA, "AUTO round %d walk: %s", round, cudaGetErrorString(cudaGetLastError()));
      if (tor::launch_batch_finalize(in.k, n, round == 1 ? 1 : 0, round == 1 ? 0.0 : tol, p, out, s))
        return fail(TOR_ECUDA, "AUTO round %d finalize: %s", round, cudaGetErrorString(cudaGetLastError()));
    }
  }
  return TOR_OK;
}

// not reserved (or n grew): size the workspace from the click counts, read once
static int batch_autoreserve(tor_ctx *ctx, const int *k_dev, int n, cudaStream_t s) {
  int *hk = new (std::nothrow) int[n];
  if (!hk) return fail(TOR_ENOMEM, "host allocation failed");
  cudaError_t e = cudaMemcpyAsync(hk, k_dev, sizeof(int) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int kmax = ctx->batch_kmax > 0 ? ctx->batch_kmax : 0;
  for (int i = 0; i < n && e == cudaSuccess; ++i)
    if (hk[i] > kmax && hk[i] <= TOR_MAX_K) kmax = hk[i];
  delete[] hk;
  if (e != cudaSuccess) return fail(TOR_ECUDA, "reading k: %s", cudaGetErrorString(e));
  if (n <= ctx->batch_nmax && kmax <= ctx->batch_kmax) return TOR_OK;
  return batch_reserve(ctx, n > ctx->batch_nmax ? n : ctx->batch_nmax, kmax);
}

static int batch_check(tor_ctx *ctx, int n, int prec, double tol) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (n < 0) return fail(TOR_EINVAL, "n = %d < 0", n);
  if (prec < TOR_PREC_AUTO || prec > TOR_PREC_FX256) return fail(TOR_EINVAL, "bad precision %d", prec);
  if (prec == TOR_PREC_AUTO && !(tol > 0.0)) return fail(TOR_EINVAL, "TOR_PREC_AUTO needs tol > 0");
  return TOR_OK;
}

int tor_batch(tor_ctx *ctx, const double *const *O, const int *k, const int *ld, int n, int layout,
              int prec, double tol, cudaStream_t s, tor_result *out) {
  int rc = batch_check(ctx, n, prec, tol);
  if (rc) return rc;
  if (n == 0) return TOR_OK;
  if (!O || !k || !ld || !out) return fail(TOR_EINVAL, "null array pointer");
  if (layout != TOR_LAYOUT_XXPP && layout != TOR_LAYOUT_XPXP) return fail(TOR_EINVAL, "bad layout %d", layout);
  CK(cudaSetDevice(ctx->device));
  // without an explicit reservation every call sizes the workspace for its own
  // k (one host read), so no instance is refused for outgrowing an earlier call
  if (!ctx->batch_explicit || n > ctx->batch_nmax)
    if ((rc = batch_autoreserve(ctx, k, n, s))) return rc;
  tor::BatchInput in{O, k, ld, layout, nullptr, nullptr, 0, 0, 0};
  return batch_enqueue(ctx, in, n, prec, tol, s, out);
}

static int batch_patterns(tor_ctx *ctx, const double *O, int M, int ld, const uint64_t *patterns, int n, int prec,
                          double tol, cudaStream_t s, tor_result *out, int kcap) {
  int rc = batch_check(ctx, n, prec, tol);
  if (rc) return rc;
  if (n == 0) return TOR_OK;
  if (M < 1 || M > 128) return fail(TOR_EINVAL, "M = %d outside [1, 128]", M);
  if (!O || !patterns || !out) return fail(TOR_EINVAL, "null array pointer");
  if (ld < 2 * M) return fail(TOR_EINVAL, "ld = %d < 2M = %d", ld, 2 * M);
  CK(cudaSetDevice(ctx->device));
  const int words = (M + 63) / 64;
  // patterns of this state can have up to min(M, TOR_MAX_K) clicks: size for that
  // once, so that no later pattern is refused for outgrowing an earlier batch
  const int kstate = M < TOR_MAX_K ? M : TOR_MAX_K;
  if (n > ctx->batch_nmax || ctx->batch_kmax < kstate)
    if ((rc = batch_reserve(ctx, n > ctx->batch_nmax ? n : ctx->batch_nmax,
                            kstate > ctx->batch_kmax ? kstate : ctx->batch_kmax)))
      return rc;
  if (tor::launch_pattern_popcount((const unsigned long long *)patterns, n, words, ctx->k_dev, s))
    return fail(TOR_ECUDA, "popcount: %s", cudaGetErrorString(cudaGetLastError()));
  tor::BatchInput in{nullptr, ctx->k_dev, nullptr, TOR_LAYOUT_XXPP, O, (const unsigned long long *)patterns, M, ld,
                     words};
  return batch_enqueue(ctx, in, n, prec, tol, s, out, kcap);
}

int tor_batch_patterns(tor_ctx *ctx, const double *O, int M, int ld, const uint64_t *patterns, int n, int prec,
                       double tol, cudaStream_t s, tor_result *out) {
  return batch_patterns(ctx, O, M, ld, patterns, n, prec, tol, s, out, -1);
}

int gbs_sample_step(tor_ctx *ctx, const double *O, int M, int ld, double logdet_sigma, const double *marg_p,
                    tor_mlp *proposal, int C, uint64_t *patterns, double *logp, double *logq, int *accepted,
                    uint64_t seed, uint64_t step, int prec, double tol, int k_cap, cudaStream_t s) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (M < 1 || M > 128) return fail(TOR_EINVAL, "M = %d outside [1, 128]", M);
  if (C < 0) return fail(TOR_EINVAL, "C = %d < 0", C);
  if (C == 0) return TOR_OK;
  if (!O || !patterns || !logp || !logq || !accepted) return fail(TOR_EINVAL, "null array pointer");
  if (!proposal && !marg_p) return fail(TOR_EINVAL, "plain proposal needs the marginals marg_p");
  if (proposal && tor::mlp_modes(proposal) != M) return fail(TOR_EINVAL, "proposal network has a different M");
  CK(cudaSetDevice(ctx->device));
  const int words = (M + 63) / 64;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_prop = al(sizeof(uint64_t) * words * (size_t)C), b_lq = al(sizeof(double) * (size_t)C),
               b_res = al(sizeof(tor_result) * (size_t)C);
  int rc;
  if ((rc = ensure(ctx, ctx->mh, b_prop + b_lq + b_res))) return rc;
  unsigned char *base = (unsigned char *)ctx->mh.p;
  unsigned long long *prop = (unsigned long long *)base;
  double *lq_prop = (double *)(base + b_prop);
  tor_result *res = (tor_result *)(base + b_prop + b_lq);
  if (proposal) {
    if ((rc = tor_mlp_sample(proposal, C, seed, step, (uint64_t *)prop, lq_prop, s))) return rc;
  } else if (tor::launch_propose_plain(marg_p, M, C, words, seed, step, prop, lq_prop, s)) {
    return fail(TOR_ECUDA, "proposal: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if ((rc = batch_patterns(ctx, O, M, ld, (const uint64_t *)prop, C, prec, tol, s, res, k_cap > 0 ? k_cap : -1)))
    return rc;
  if (tor::launch_accept(C, M, words, k_cap, logdet_sigma, res, prop, lq_prop, (unsigned long long *)patterns, logp, logq,
                         accepted, seed, step, s))
    return fail(TOR_ECUDA, "accept: %s", cudaGetErrorString(cudaGetLastError()));
  return TOR_OK;
}

int gbs_sample_step_da(tor_ctx *ctx, const double *O, int M, int ld, double logdet_sigma, const double *marg_p,
                       tor_mlp *surrogate, int C, uint64_t *patterns, double *logp, double *logq, double *logs,
                       int *accepted, uint64_t seed, uint64_t step, int prec, double tol, int k_cap, cudaStream_t s) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (M < 1 || M > 128) return fail(TOR_EINVAL, "M = %d outside [1, 128]", M);
  if (C < 0) return fail(TOR_EINVAL, "C = %d < 0", C);
  if (C == 0) return TOR_OK;
  if (!O || !marg_p || !surrogate || !patterns || !logp || !logq || !logs || !accepted)
    return fail(TOR_EINVAL, "null pointer");
  if (tor::mlp_modes(surrogate) != M) return fail(TOR_EINVAL, "surrogate network has a different M");
  CK(cudaSetDevice(ctx->device));
  const int words = (M + 63) / 64;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_prop = al(sizeof(uint64_t) * words * (size_t)C), b_d = al(sizeof(double) * (size_t)C),
               b_res = al(sizeof(tor_result) * (size_t)C);
  int rc;
  if ((rc = ensure(ctx, ctx->mh, 2 * b_prop + 2 * b_d + b_res))) return rc;
  unsigned char *base = (unsigned char *)ctx->mh.p;
  unsigned long long *prop = (unsigned long long *)base;
  unsigned long long *eval = (unsigned long long *)(base + b_prop);
  double *lq_prop = (double *)(base + 2 * b_prop);
  double *ls_prop = (double *)(base + 2 * b_prop + b_d);
  tor_result *res = (tor_result *)(base + 2 * b_prop + 2 * b_d);
  if (tor::launch_propose_plain(marg_p, M, C, words, seed, step, prop, lq_prop, s))
    return fail(TOR_ECUDA, "proposal: %s", cudaGetErrorString(cudaGetLastError()));
  if ((rc = tor_mlp_logq(surrogate, (const uint64_t *)prop, C, ls_prop, s))) return rc;
  if (tor::launch_screen(C, M, words, k_cap, prop, lq_prop, ls_prop, logp, logq, logs, eval, accepted, seed, step, s))
    return fail(TOR_ECUDA, "screen: %s", cudaGetErrorString(cudaGetLastError()));
  if ((rc = batch_patterns(ctx, O, M, ld, (const uint64_t *)eval, C, prec, tol, s, res, k_cap > 0 ? k_cap : -1)))
    return rc;
  if (tor::launch_accept_da(C, M, words, logdet_sigma, res, prop, lq_prop, ls_prop, (unsigned long long *)patterns,
                            logp, logq, logs, accepted, seed, step, s))
    return fail(TOR_ECUDA, "accept: %s", cudaGetErrorString(cudaGetLastError()));
  return TOR_OK;
}

int tor_bounds(tor_ctx *ctx, const double *const *O, const int *k, const int *ld, int n, int layout,
               double tol, cudaStream_t s, tor_bound *out) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (n < 0) return fail(TOR_EINVAL, "n = %d < 0", n);
  if (n == 0) return TOR_OK;
  if (!O || !k || !ld || !out) return fail(TOR_EINVAL, "null array pointer");
  if (layout != TOR_LAYOUT_XXPP && layout != TOR_LAYOUT_XPXP) return fail(TOR_EINVAL, "bad layout %d", layout);
  if (!(tol > 0.0)) return fail(TOR_EINVAL, "tol must be > 0");
  CK(cudaSetDevice(ctx->device));
  if (tor::launch_bounds_batch(O, k, ld, n, layout, tol, out, s))
    return fail(TOR_ECUDA, "bound pass launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  return TOR_OK;
}

// ------------------------------------------------------------------ autotuner
namespace {

struct TuneEntry {
  char gpu[128];
  int k, tier, d, bps;
  double ms;
};

bool parse_line(const char *line, TuneEntry &e) {
  // {"gpu": "...", "k": K, "tier": T, "chunk_bits": D, "blocks_per_sm": B, "ms": X}
  const char *g = strstr(line, "\"gpu\": \"");
  if (!g) return false;
  g += 8;
  const char *ge = strchr(g, '"');
  if (!ge || ge - g >= (long)sizeof(e.gpu)) return false;
  memcpy(e.gpu, g, ge - g);
  e.gpu[ge - g] = 0;
  const char *kk = strstr(line, "\"k\": "), *t = strstr(line, "\"tier\": "),
             *d = strstr(line, "\"chunk_bits\": "), *b = strstr(line, "\"blocks_per_sm\": "),
             *m = strstr(line, "\"ms\": ");
  if (!kk || !t || !d || !b || !m) return false;
  e.k = atoi(kk + 5);
  e.tier = atoi(t + 8);
  e.d = atoi(d + 14);
  e.bps = atoi(b + 17);
  e.ms = atof(m + 6);
  return e.k >= 0 && e.k <= 64 && e.tier >= TOR_PREC_FP64 && e.tier <= TOR_PREC_FX256 && e.d >= 0 && e.d <= e.k &&
         e.bps >= 1 && e.bps <= 16;
}

}  // namespace

int tor_autotune(tor_ctx *ctx, int k, int prec, const char *cache_path, int *chunk_bits_out,
                 int *blocks_per_sm_out) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  if (k < 1 || k > 40) return fail(TOR_EINVAL, "autotune k = %d outside [1, 40]", k);
  if (prec < TOR_PREC_FP64 || prec > TOR_PREC_FX256) return fail(TOR_EINVAL, "prec must be an explicit tier");
  CK(cudaSetDevice(ctx->device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, ctx->device));
  // 1. a cached result for this GPU, k and tier
  if (cache_path) {
    FILE *f = fopen(cache_path, "r");
    if (f) {
      char line[512];
      TuneEntry e, best{};
      bool found = false;
      while (fgets(line, sizeof(line), f))
        if (parse_line(line, e) && e.k == k && e.tier == prec && strcmp(e.gpu, prop.name) == 0) {
          best = e;
          found = true;
        }
      fclose(f);
      if (found) {
        ctx->tuned_d[prec][k] = (signed char)best.d;
        ctx->tuned_bps[prec][k] = (signed char)best.bps;
        ctx->r1_table[prec][k] = (unsigned char)(k - best.d);
        if (ctx->r1_table_dev)  // the batch plan reads the device copy
          CK(cudaMemcpy(ctx->r1_table_dev, ctx->r1_table, sizeof(ctx->r1_table), cudaMemcpyHostToDevice));
        if (chunk_bits_out) *chunk_bits_out = best.d;
        if (blocks_per_sm_out) *blocks_per_sm_out = best.bps;
        return TOR_OK;
      }
    }
  }
  // 2. time the candidates on a synthetic instance (O = I/4: same work as any
  //    positive definite input of this size, which is all the walk's cost depends on)
  const int n = 2 * k;
  double *O = nullptr;
  tor_result *res = nullptr;
  if (cudaMalloc(&O, sizeof(double) * n * n) != cudaSuccess || cudaMalloc(&res, sizeof(tor_result)) != cudaSuccess) {
    cudaFree(O);
    return fail(TOR_ENOMEM, "autotune allocation failed");
  }
  double *h = new (std::nothrow) double[(size_t)n * n];
  if (!h) { cudaFree(O); cudaFree(res); return fail(TOR_ENOMEM, "host allocation failed"); }
  for (int i = 0; i < n * n; ++i) h[i] = (i / n == i % n) ? 0.25 : 0.0;
  cudaMemcpy(O, h, sizeof(double) * n * n, cudaMemcpyHostToDevice);
  delete[] h;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int saved_d = ctx->chunk_bits, saved_bps = ctx->blocks_per_sm;
  double best_ms = 1e30;
  int best_d = choose_chunk_bits(ctx, k), best_bps = saved_bps;
  const int r1s[] = {8, 10, 12, 13, 14, 15, 16};
  const int bpss[] = {2, 3, 4};
  int rc = TOR_OK;
  for (int r1 : r1s) {
    if (r1 > k) continue;
    const int d = k - r1;
    if (d > 24) continue;
    for (int bps : bpss) {
      ctx->chunk_bits = d;
      ctx->blocks_per_sm = bps;
      // Chunks cost the same walk; their roots differ with the number of fixed
      // modes.  So each candidate walks a sample of two waves of chunks (all of
      // them when there are fewer) whose high chunk bits are half set, a
      // typical root cost, and the time is scaled to all 2^d chunks.
      const int grid = walk_grid(ctx, prec);
      const unsigned long long nch = 1ull << d, T = (unsigned long long)grid * ctx->threads_per_block;
      unsigned long long cnt = 2 * T, c0 = 0;
      if (cnt >= nch) {
        cnt = nch;
      } else {
        unsigned long long pow2 = 1;
        while (pow2 < cnt) pow2 <<= 1;
        cnt = pow2;                                          // a power of two: all low-bit patterns
        c0 = (0x5555555555555555ull & (nch - 1)) & ~(cnt - 1);
      }
      const tor::WalkSegs seg = plan_segments(k, d, (size_t)T);
      const tor::WalkSegs sub = (cnt == nch) ? seg : tor::one_segment(r1, c0, c0 + cnt);
      for (int r = 0; r < 3 && rc == TOR_OK; ++r) {  // warm-up (sizes the workspace), then two timed
        if (r == 1) cudaEventRecord(e0, 0);
        rc = enqueue_walk(ctx, O, k, n, TOR_LAYOUT_XXPP, prec, sub, nullptr, 0, grid);
      }
      cudaEventRecord(e1, 0);
      if (rc) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double full_ms = 0.5 * ms * (double)nch / (double)cnt;
      if (full_ms < best_ms) {
        best_ms = full_ms;
        best_d = d;
        best_bps = bps;
      }
    }
    if (rc) break;
  }
  ctx->chunk_bits = saved_d;
  ctx->blocks_per_sm = saved_bps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(O);
  cudaFree(res);
  if (rc) return rc;
  ctx->tuned_d[prec][k] = (signed char)best_d;
  ctx->tuned_bps[prec][k] = (signed char)best_bps;
  ctx->r1_table[prec][k] = (unsigned char)(k - best_d);
  if (ctx->r1_table_dev)
    CK(cudaMemcpy(ctx->r1_table_dev, ctx->r1_table, sizeof(ctx->r1_table), cudaMemcpyHostToDevice));
  if (cache_path) {
    FILE *f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "{\"gpu\": \"%s\", \"k\": %d, \"tier\": %d, \"chunk_bits\": %d, \"blocks_per_sm\": %d, \"ms\": %.4f}\n",
              prop.name, k, prec, best_d, best_bps, best_ms);
      fclose(f);
    }
  }
  if (chunk_bits_out) *chunk_bits_out = best_d;
  if (blocks_per_sm_out) *blocks_per_sm_out = best_bps;
  return TOR_OK;
}

int tor_fp64_peak(tor_ctx *ctx, double *dfma_per_s, double *sm_clock_hz) {
  if (!ctx || !dfma_per_s) return fail(TOR_EINVAL, "null pointer");
  CK(cudaSetDevice(ctx->device));
  int rc;
  if ((rc = ensure(ctx, ctx->total8, 4096))) return rc;
  const int grid = ctx->sms * 2, block = 256, iters = 1 << 14;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  tor::launch_dfma_peak((double *)ctx->total8.p, grid, block, iters, 0);  // warm-up
  CK(cudaEventRecord(e0, 0));
  for (int r = 0; r < 5; ++r) tor::launch_dfma_peak((double *)ctx->total8.p, grid, block, iters, 0);
  CK(cudaEventRecord(e1, 0));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *dfma_per_s = 5.0 * grid * block * (double)iters * 4.0 / (ms * 1e-3);
  if (sm_clock_hz) {
    int khz = 0;
    CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device));
    *sm_clock_hz = khz * 1e3;
  }
  return TOR_OK;
}

int tor_int_peak(tor_ctx *ctx, double *mad_per_s) {
  if (!ctx || !mad_per_s) return fail(TOR_EINVAL, "null pointer");
  CK(cudaSetDevice(ctx->device));
  int rc;
  if ((rc = ensure(ctx, ctx->total8, 4096))) return rc;
  const int grid = ctx->sms * 8, block = 256, iters = 1 << 14;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  tor::launch_imad_peak((long long *)ctx->total8.p, grid, block, iters, 0);  // warm-up
  CK(cudaEventRecord(e0, 0));
  for (int r = 0; r < 5; ++r) tor::launch_imad_peak((long long *)ctx->total8.p, grid, block, iters, 0);
  CK(cudaEventRecord(e1, 0));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *mad_per_s = 5.0 * grid * block * (double)iters * 8.0 / (ms * 1e-3);
  return TOR_OK;
}

}  // extern "C"
