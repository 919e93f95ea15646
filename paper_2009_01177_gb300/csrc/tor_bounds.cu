// tor_bounds.cu -- the cheap FP32 bound pass that routes an instance to a tier.
//
// The paper sizes its fixed-point type from an upper bound on the
// intermediate values (Sec. 5.1: every term is at most 1/sqrt(det(I - A)),
// the largest term t_max, because det(I - A) is below all its principal
// minors), a lower-bound estimate of the result (Sec. 5.1, Eq. lowbound:
// a product over modes), and an accumulated-error allowance (Sec. 5.4,
// Eq. bitlen).  Here the same three ingredients decide between FP64 and
// double-double factorisation:
//
//   tau_j      = 1/sqrt(det B_jj), B = I - O, for each mode's 2x2 block
//   Tor_est    = prod_j (tau_j - 1)     (the mode-product estimate; it is the
//                paper's Eq. lowbound with the correction factor at zero,
//                and it is exact for O = a I)
//   sumt_est   = prod_j (tau_j + 1)     (estimate of sum_Z t_Z)
//   kappa_est  = sumt_est / Tor_est     (condition number of Eq. 2's sum)
//   t_max      = 1/sqrt(det B)          (FP32 Cholesky, in the log domain)
//   bits_needed = log2 kappa_est + log2(4k) + log2(1/tol)
//
// kappa_est is pessimistic on Haar-mixed lossy GBS states: single-mode click
// probabilities are small while the multi-mode correlations make Tor much
// larger than the mode product (measured kappa_est / kappa from 10^2 to 10^13
// for k = 4..16).  An FP64 attempt costs about a tenth of a double-double one
// and every result carries an a-posteriori bound computed from the exact
// sum_Z t_Z, which the AUTO callers check before escalating to double-double.
// So the routing is optimistic: tier = FP64 if bits_needed <= 52 + 20 (the
// estimate may overshoot by 2^20); else the 128-bit fixed-point tier if the
// instance fits its range (t_max <= 2^11) and bits_needed <= 100 + 20; else
// double-double if bits_needed <= 104 + 20; else the 256-bit fixed-point tier
// if it fits (t_max <= 2^30); else double-double (the result then carries a
// bound above the tolerance).  The 128-bit fixed point runs about 3x faster
// than double-double at a 16x looser error bound (u = 2^-100 against 2^-104).
//
// One block of 64 threads per instance; B is held in FP32 in shared memory.
#include <cuda_runtime.h>
#include <cstdint>
#include <math.h>
#include "tor_internal.h"

namespace tor {

constexpr int BOUNDS_THREADS = 64;
constexpr float FP64_ROUTE_BITS = 52.f + 20.f;   // optimistic FP64 attempt, see above
constexpr float FX128_ROUTE_BITS = 100.f + 20.f; // the same slack over the fixed-point unit
constexpr float DD_ROUTE_BITS = 104.f + 20.f;

// O entries of one instance in mode-interleaved local coordinates (row = 2m + q)
struct OInstance {
  const double *O;
  int k, ld, layout;
  __device__ double operator()(int r, int c) const {
    const int ri = (layout == 0) ? ((r & 1) * k + (r >> 1)) : r;
    const int rj = (layout == 0) ? ((c & 1) * k + (c >> 1)) : c;
    return O[(size_t)ri * ld + rj];
  }
};
struct OPattern {  // O_S of a click pattern: local mode m is global mode gm[m] (rows gm[m], M + gm[m])
  const double *O;
  int M, ld;
  const unsigned char *gm;
  __device__ double operator()(int r, int c) const {
    return O[(size_t)((r & 1) * M + gm[r >> 1]) * ld + (c & 1) * M + gm[c >> 1]];
  }
};

template <class Get>
__device__ void bounds_one(const Get &getO, bool valid, int k, double tol, float *sB, tor_bound *out) {
  const int tid = threadIdx.x;
  if (k < 0 || k > TOR_MAX_K || !valid) {  // invalid instance: tier 0, bits_needed NaN
    if (tid == 0) *out = tor_bound{NAN, NAN, NAN, NAN, 0};
    return;
  }
  const int n = 2 * k;
  // B = I - O in FP32, mode-interleaved, full square in shared memory
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e % n;
    sB[e] = (float)((r == c ? 1.0 : 0.0) - getO(r, c));
  }
  __syncthreads();
  // per-mode factors tau_j (warp 0 reduces the logs)
  __shared__ float s_logm[BOUNDS_THREADS], s_logp[BOUNDS_THREADS];
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  float lm = 0.f, lp = 0.f;
  for (int j = tid; j < k; j += blockDim.x) {
    const float a = sB[(2 * j) * n + 2 * j], b = sB[(2 * j + 1) * n + 2 * j], d = sB[(2 * j + 1) * n + 2 * j + 1];
    const float det2 = a * d - b * b;
    const float tau = rsqrtf(fmaxf(det2, 1e-30f));
    lm += logf(fmaxf(tau - 1.f, 1e-30f));  // a mode with tau <= 1 cannot click
    lp += logf(tau + 1.f);
  }
  s_logm[tid] = lm;
  s_logp[tid] = lp;
  __syncthreads();
  // FP32 Cholesky of B in place (right-looking), log det = 2 sum log L_ii
  float logdet = 0.f;
  for (int j = 0; j < n; ++j) {
    const float p = sB[j * n + j];
    if (p <= 0.f || !isfinite(p)) {
      if (tid == 0) s_bad = 1;
      break;
    }
    const float l = sqrtf(p);
    logdet += 2.f * logf(l);
    __syncthreads();
    for (int i = j + 1 + tid; i < n; i += blockDim.x) sB[i * n + j] /= l;
    __syncthreads();
    for (int e = tid; e < (n - j - 1) * (n - j - 1); e += blockDim.x) {
      const int i = j + 1 + e / (n - j - 1), c = j + 1 + e % (n - j - 1);
      if (c <= i) sB[i * n + c] -= sB[i * n + j] * sB[c * n + j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    float sm = 0.f, sp = 0.f;
    for (int t = 0; t < (int)blockDim.x; ++t) { sm += s_logm[t]; sp += s_logp[t]; }
    tor_bound bd;
    bd.log_tmax = s_bad ? INFINITY : -0.5f * logdet;
    bd.log_tor_est = sm;
    bd.log_kappa_est = sp - sm;
    const float bits = (float)((sp - sm) / 0.6931471805599453) + log2f(4.f * (float)(k > 1 ? k : 1)) +
                       (float)log2(1.0 / (tol > 0 ? tol : 1e-300));
    bd.bits_needed = s_bad ? INFINITY : bits;
    const bool fx_ok = !s_bad && bd.log_tmax <= FX128_MAX_LOG2_TMAX * 0.6931472f;
    const bool fx256_ok = !s_bad && bd.log_tmax <= FX256_MAX_LOG2_TMAX * 0.6931472f;
    bd.tier = (!s_bad && bits <= FP64_ROUTE_BITS)            ? TOR_PREC_FP64
              : (fx_ok && bits <= FX128_ROUTE_BITS)           ? TOR_PREC_FX128
              : (!s_bad && bits <= DD_ROUTE_BITS)             ? TOR_PREC_DD
              : fx256_ok                                        ? TOR_PREC_FX256
                                                              : TOR_PREC_DD;
    *out = bd;
  }
}

__global__ void __launch_bounds__(BOUNDS_THREADS)
k_bounds_batch(const double *const *__restrict__ O, const int *__restrict__ k, const int *__restrict__ ld,
               int layout, double tol, tor_bound *__restrict__ out) {
  extern __shared__ float sB[];
  const int i = blockIdx.x;
  bounds_one(OInstance{O[i], k[i], ld[i], layout}, O[i] != nullptr, k[i], tol, sB, out + i);
}

__global__ void __launch_bounds__(BOUNDS_THREADS)
k_bounds_single(const double *__restrict__ O, int k, int ld, int layout, double tol, tor_bound *__restrict__ out) {
  extern __shared__ float sB[];
  bounds_one(OInstance{O, k, ld, layout}, O != nullptr, k, tol, sB, out);
}

__global__ void __launch_bounds__(BOUNDS_THREADS)
k_bounds_patterns(const double *__restrict__ Ofull, int M, int ld, const unsigned long long *__restrict__ patterns,
                  int words, double tol, tor_bound *__restrict__ out) {
  extern __shared__ float sB[];
  __shared__ unsigned char gm[TOR_MAX_K];
  __shared__ int s_k;
  const int i = blockIdx.x;
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < words; ++w)
      for (unsigned long long bits = patterns[(size_t)i * words + w]; bits; bits &= bits - 1) {
        if (m < TOR_MAX_K) gm[m] = (unsigned char)(64 * w + __ffsll((long long)bits) - 1);
        ++m;
      }
    s_k = m;
  }
  __syncthreads();
  const int k = s_k;
  bounds_one(OPattern{Ofull, M, ld, gm}, k <= TOR_MAX_K, k, tol, sB, out + i);
}

int launch_bounds_batch(const double *const *O, const int *k, const int *ld, int n, int layout, double tol,
                        tor_bound *out, cudaStream_t s) {
  const size_t smem = sizeof(float) * (2 * TOR_MAX_K) * (2 * TOR_MAX_K);
  cudaFuncSetAttribute(k_bounds_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_bounds_batch<<<n, BOUNDS_THREADS, smem, s>>>(O, k, ld, layout, tol, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_bounds_patterns(const double *Ofull, int M, int ld, const unsigned long long *patterns, int words,
                           int n, double tol, tor_bound *out, cudaStream_t s) {
  const size_t smem = sizeof(float) * (2 * TOR_MAX_K) * (2 * TOR_MAX_K);
  cudaFuncSetAttribute(k_bounds_patterns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_bounds_patterns<<<n, BOUNDS_THREADS, smem, s>>>(Ofull, M, ld, patterns, words, tol, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_bounds_single(const double *O, int k, int ld, int layout, double tol, tor_bound *out,
                         cudaStream_t s) {
  const size_t smem = sizeof(float) * (2 * k) * (2 * k);
  cudaFuncSetAttribute(k_bounds_single, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(float) * (2 * TOR_MAX_K) * (2 * TOR_MAX_K)));
  k_bounds_single<<<1, BOUNDS_THREADS, smem, s>>>(O, k, ld, layout, tol, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tor
