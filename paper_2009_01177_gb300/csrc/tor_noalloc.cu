// tor_noalloc.cu -- tor_single_noalloc: the Torontonian without any allocation.
//
// Who needs this: code that must not call cudaMalloc -- for example a caller
// that runs inside a memory pool it does not own, a plugin that is handed a
// stream but no allocator, or a process that has to keep its device
// footprint fixed after start-up.  tor_single allocates its workspace inside
// a context; this entry point instead carves every scratch buffer (the
// I - O matrix, the per-thread depth-first stacks, the block partial sums and
// the status word) out of one file-scope device array of fixed size, so a
// call performs no device allocation at all.  The caller still provides the
// input matrix and the output record.
//
// Limits and sharing:
//   * The array holds NOALLOC_SCRATCH_BYTES (48 MiB); the driver reserves it
//     on every GPU where the library is loaded, until the process exits.
//     Instances whose workspace does not fit are rejected with TOR_EINVAL
//     (on a 152-SM GB300: FP64 up to k = 25, double-double up to k = 17).
//   * All calls on a device share the one array and it keeps the previous
//     call's contents; the status word is cleared at the start of every call
//     and every other buffer is fully written before it is read.  Calls whose
//     work overlaps on the GPU (two streams, or two host threads) race on the
//     array and give wrong results: serialise them.
//   * The first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it; make
//     that first call before any stream capture begins.
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include "tor_dfs.cuh"
#include "tor_internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 48ull << 20;
constexpr int NOALLOC_THREADS = 32;  // one warp per SM keeps the stacks small
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_base[NOALLOC_MAX_DEVICES] = {};

int nfail(int code, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  return tor::record_error(code, msg);  // readable through tor_last_error()
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" {

int tor_single_noalloc(const double *O, int k, int ld, int layout, int prec, cudaStream_t stream,
                       tor_result *out_dev) {
  if (k < 0 || k > TOR_MAX_K) return nfail(TOR_EINVAL, "k = %d outside [0, %d]", k, TOR_MAX_K);
  if (k > 0 && !O) return nfail(TOR_EINVAL, "null matrix pointer");
  if (k > 0 && ld < 2 * k) return nfail(TOR_EINVAL, "ld = %d < 2k = %d", ld, 2 * k);
  if (layout != TOR_LAYOUT_XXPP && layout != TOR_LAYOUT_XPXP) return nfail(TOR_EINVAL, "bad layout %d", layout);
  if (prec != TOR_PREC_FP64 && prec != TOR_PREC_DD)
    return nfail(TOR_EINVAL, "tor_single_noalloc needs TOR_PREC_FP64 or TOR_PREC_DD");
  if (!out_dev) return nfail(TOR_EINVAL, "null result pointer");

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(TOR_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return nfail(TOR_EINVAL, "device %d beyond %d", dev, NOALLOC_MAX_DEVICES);
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return nfail(TOR_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));

  // one-time set-up per device: the array's device address, looked up with that device current
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return nfail(TOR_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      g_noalloc_base[dev] = p;
    }
    base = (unsigned char *)g_noalloc_base[dev];
  }

  if (k == 0) {  // Tor = 1 (only the empty set), written by a one-thread kernel: stays asynchronous
    if (tor::launch_result_one(out_dev, prec, stream))
      return nfail(TOR_ECUDA, "k = 0 result: %s", cudaGetErrorString(cudaGetLastError()));
    return TOR_OK;
  }

  // chunks of at most 10 walked modes (up to 2^18 chunks): short per-thread
  // stacks, so that the fixed array covers the largest k (the grid here is one
  // 32-thread block per SM, so 2^k-10 chunks fill it long before 2^16)
  int d = k - 10;
  if (d > 18) d = 18;
  if (d < 0) d = 0;
  const int r1 = k - d;
  const int grid = sms;
  const size_t nthreads = (size_t)grid * NOALLOC_THREADS;
  const size_t bytes_B = align256(sizeof(double) * 4 * (size_t)k * k);
  const size_t bytes_Blo = align256(sizeof(double) * 2 * (size_t)k);
  const size_t bytes_status = align256(sizeof(int));
  const size_t bytes_part = align256(sizeof(unsigned long long) * 8 * (size_t)grid);
  const size_t bytes_stack = sizeof(double) * nthreads * (size_t)tor::scratch_entries(prec, k, r1);
  const size_t need = bytes_B + bytes_Blo + bytes_status + bytes_part + bytes_stack;
  if (need > NOALLOC_SCRATCH_BYTES)
    return nfail(TOR_EINVAL,
                 "k = %d (%s) needs %zu bytes of scratch on this %d-SM device; the fixed array holds %zu",
                 k, prec == TOR_PREC_DD ? "double-double" : "FP64", need, sms, NOALLOC_SCRATCH_BYTES);

  double *B = (double *)base;
  double *Blo = (double *)(base + bytes_B);
  int *status = (int *)(base + bytes_B + bytes_Blo);
  unsigned long long *part = (unsigned long long *)(base + bytes_B + bytes_Blo + bytes_status);
  double *stack = (double *)(base + bytes_B + bytes_Blo + bytes_status + bytes_part);

  tor::launch_prep(O, k, ld, layout, B, Blo, stream);
  e = cudaMemsetAsync(status, 0, sizeof(int), stream);  // the only buffer that must start at zero
  if (e != cudaSuccess) return nfail(TOR_ECUDA, "status clear: %s", cudaGetErrorString(e));
  tor::launch_dfs(prec, grid, NOALLOC_THREADS, B, Blo, k, tor::one_segment(r1, 0ull, 1ull << d), stack, part,
                  nullptr, status, stream);
  tor::launch_finalize(part, grid, k, prec, status, out_dev, stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(TOR_ECUDA, "launch: %s", cudaGetErrorString(e));
  return TOR_OK;
}

}  // extern "C"
