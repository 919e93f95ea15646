// capi.cu -- the C ABI (include/torontonian.h): context, workspace, entry points.
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <new>
#include "tor_internal.h"

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
  Buf B, Blo, scratch, block_part, status, result, total8;
  bool timing = false, timed = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
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
int choose_chunk_bits(const tor_ctx *c, int k) {
  if (c->chunk_bits >= 0) return c->chunk_bits < k ? c->chunk_bits : k;
  int d = k - 10;
  const int cap = (k >= 36) ? 20 : 18;
  if (d > cap) d = cap;
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

// enqueue prep + walk over chunks [c0, c1); block partials in ctx->block_part
int enqueue_walk(tor_ctx *ctx, const double *O, int k, int ld, int layout, int tier, int d,
                 unsigned long long c0, unsigned long long c1, unsigned long long *chunk_part,
                 cudaStream_t s, int *grid_out) {
  const int r1 = k - d;
  const int block = ctx->threads_per_block;
  // every block of the grid must be resident at once: chunks are dealt out by
  // a grid stride, so a block that waited for a free SM would double the time
  const int occ = tor::dfs_max_blocks_per_sm(tier, block);
  const int grid = ctx->sms * (ctx->blocks_per_sm < occ ? ctx->blocks_per_sm : occ);
  const size_t nthreads = (size_t)grid * block;
  int rc;
  if ((rc = ensure(ctx, ctx->B, sizeof(double) * 4 * (size_t)k * k))) return rc;
  if ((rc = ensure(ctx, ctx->Blo, sizeof(double) * 2 * (size_t)k))) return rc;
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * nthreads * (size_t)tor::scratch_entries(tier, k, r1)))) return rc;
  if ((rc = ensure(ctx, ctx->block_part, sizeof(unsigned long long) * 8 * (size_t)grid))) return rc;
  if ((rc = ensure(ctx, ctx->status, sizeof(int)))) return rc;
  tor::launch_prep(O, k, ld, layout, (double *)ctx->B.p, (double *)ctx->Blo.p, s);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), s));
  if (ctx->timing) CK(cudaEventRecord(ctx->ev0, s));
  tor::launch_dfs(tier, grid, block, (const double *)ctx->B.p, (const double *)ctx->Blo.p, k, r1, c0, c1,
                  (double *)ctx->scratch.p, (unsigned long long *)ctx->block_part.p, chunk_part,
                  (int *)ctx->status.p, s);
  CK(cudaGetLastError());
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev1, s));
    ctx->timed = true;
  }
  *grid_out = grid;
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
  Buf *bufs[] = {&c->B, &c->Blo, &c->scratch, &c->block_part, &c->status, &c->result, &c->total8};
  for (Buf *b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

int tor_set_timing(tor_ctx *ctx, int on) {
  if (!ctx) return fail(TOR_EINVAL, "null context");
  CK(cudaSetDevice(ctx->device));
  if (on && !ctx->ev0) {
    CK(cudaEventCreate(&ctx->ev0));
    CK(cudaEventCreate(&ctx->ev1));
  }
  ctx->timing = on != 0;
  ctx->timed = false;
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
  if (prec != TOR_PREC_FP64 && prec != TOR_PREC_DD)
    return fail(TOR_EINVAL, "tor_single_async needs TOR_PREC_FP64 or TOR_PREC_DD");
  CK(cudaSetDevice(ctx->device));
  if (k == 0) {
    tor_result one = {1.0, 0.0, 1.0, 0.0, prec, TOR_OK};
    CK(cudaMemcpyAsync(out_dev, &one, sizeof(one), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // `one` lives on this stack frame
    return TOR_OK;
  }
  const int d = choose_chunk_bits(ctx, k);
  int grid = 0;
  if ((rc = enqueue_walk(ctx, O, k, ld, layout, prec, d, 0ull, 1ull << d, nullptr, s, &grid))) return rc;
  tor::launch_finalize((const unsigned long long *)ctx->block_part.p, grid, k, prec,
                       (const int *)ctx->status.p, out_dev, nullptr, s);
  CK(cudaGetLastError());
  return TOR_OK;
}

int tor_single(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec, double tol,
               cudaStream_t s, tor_result *out) {
  int rc = check_common(ctx, O, k, ld, layout);
  if (rc) return rc;
  if (!out) return fail(TOR_EINVAL, "null result pointer");
  if (prec != TOR_PREC_AUTO && prec != TOR_PREC_FP64 && prec != TOR_PREC_DD)
    return fail(TOR_EINVAL, "bad precision %d", prec);
  (void)tol;
  const int tier = pick_tier(prec);
  if ((rc = ensure(ctx, ctx->result, sizeof(tor_result)))) return rc;
  if ((rc = tor_single_async(ctx, O, k, ld, layout, tier, s, (tor_result *)ctx->result.p))) return rc;
  CK(cudaMemcpyAsync(out, ctx->result.p, sizeof(tor_result), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (out->status != TOR_OK)
    return fail(out->status, "instance status %d (%s)", out->status,
                out->status == TOR_ENOTPD ? "some I - O_Z is not positive definite" : "term out of range");
  return TOR_OK;
}

int tor_chunks(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec, int chunk_bits,
               uint64_t c_begin, uint64_t c_end, cudaStream_t s, uint64_t *part_dev) {
  int rc = check_common(ctx, O, k, ld, layout);
  if (rc) return rc;
  if (k == 0) return fail(TOR_EINVAL, "tor_chunks needs k >= 1");
  if (prec != TOR_PREC_FP64 && prec != TOR_PREC_DD) return fail(TOR_EINVAL, "prec must be FP64 or DD");
  if (chunk_bits < 0 || chunk_bits > k || chunk_bits > 40) return fail(TOR_EINVAL, "chunk_bits outside [0, min(k, 40)]");
  if (!part_dev) return fail(TOR_EINVAL, "null partials pointer");
  const uint64_t nchunks = 1ull << chunk_bits;
  if (c_begin > c_end || c_end > nchunks) return fail(TOR_EINVAL, "chunk range [%llu, %llu) outside [0, %llu)",
                                                     (unsigned long long)c_begin, (unsigned long long)c_end,
                                                     (unsigned long long)nchunks);
  if (c_begin == c_end) return TOR_OK;
  CK(cudaSetDevice(ctx->device));
  int grid = 0;
  return enqueue_walk(ctx, O, k, ld, layout, prec, chunk_bits, c_begin, c_end,
                      (unsigned long long *)part_dev, s, &grid);
}

int tor_fixed_to_result(const uint64_t *limbs8, int k, int tier, tor_result *out) {
  if (!limbs8 || !out) return fail(TOR_EINVAL, "null pointer");
  if (tier != TOR_PREC_FP64 && tier != TOR_PREC_DD) return fail(TOR_EINVAL, "bad tier");
  tor::fixed_to_result((const unsigned long long *)limbs8, k, tier, 0, out);
  return TOR_OK;
}

int tor_batch(tor_ctx *ctx, const double *const *O, const int *k, const int *ld, int n, int layout,
              int prec, double tol, cudaStream_t s, tor_result *out) {
  (void)ctx; (void)O; (void)k; (void)ld; (void)n; (void)layout; (void)prec; (void)tol; (void)s; (void)out;
  return fail(TOR_EINVAL, "tor_batch: not built yet");
}

int tor_bounds(tor_ctx *ctx, const double *const *O, const int *k, const int *ld, int n, int layout,
               double tol, cudaStream_t s, tor_bound *out) {
  (void)ctx; (void)O; (void)k; (void)ld; (void)n; (void)layout; (void)tol; (void)s; (void)out;
  return fail(TOR_EINVAL, "tor_bounds: not built yet");
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

}  // extern "C"
