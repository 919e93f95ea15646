// tor_mh.cu -- one independence Metropolis-Hastings step for C chains of
// threshold GBS click patterns (the paper's MCMC use of the Torontonian,
// Sec. 7.1.1: about 100 probabilities per sample).
//
//   1. propose S'_c for every chain: plain = independent Bernoulli per mode
//      with the caller's single-mode click probabilities; learned = ancestral
//      sampling of the MADE network (tor_mlp.cu);
//   2. exact log p(S') = log Tor(O_S') - 1/2 log det Sigma (Eq. 1), all C
//      Torontonians in one tor_batch_patterns launch sequence;
//   3. accept with probability min(1, p(S') q(S) / (p(S) q(S'))).
//
// Every random draw is Philox4x32-10 at (seed; step, chain, j): j < M are
// the proposal's mode draws, j = M the acceptance draw.  A chain whose
// current log p is -inf (not yet initialised) accepts any proposal with
// p(S') > 0.  A proposal whose p(S') is not known to the requested tolerance
// is rejected and says why in `accepted` (negative codes), so that callers
// can count every such rejection: -1 more clicks than the cap (not
// evaluated), -2 the Torontonian missed the tolerance in the most precise tier
// that holds it (TOR_EPREC), -3 any other failed evaluation or Tor <= 0.
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>
#include "tor_internal.h"
#include "philox.cuh"

namespace tor {

__global__ void k_propose_plain(const double *__restrict__ marg, int M, int C, int words, unsigned long long seed,
                                unsigned long long step, unsigned long long *__restrict__ prop,
                                double *__restrict__ logq_prop) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double lq = 0.0;
  unsigned long long w[2] = {0ull, 0ull};
  for (int j = 0; j < M; ++j) {
    const double pj = marg[j];
    const double u = philox_uniform(seed, step, (uint32_t)c, (uint32_t)j);
    const bool x = u < pj;
    if (x) w[j >> 6] |= 1ull << (j & 63);
    lq += x ? log(pj) : log1p(-pj);
  }
  for (int i = 0; i < words; ++i) prop[(size_t)c * words + i] = w[i];
  logq_prop[c] = lq;
}

__global__ void k_accept(int C, int M, int words, int k_cap, double logdet_sigma, const tor_result *__restrict__ tr,
                         const unsigned long long *__restrict__ prop, const double *__restrict__ logq_prop,
                         unsigned long long *__restrict__ pat, double *__restrict__ logp, double *__restrict__ logq,
                         int *__restrict__ accepted, unsigned long long seed, unsigned long long step) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const tor_result r = tr[c];
  const double tor = r.hi + r.lo;
  const double lp_new = (r.status == TOR_OK && tor > 0.0) ? log(tor) - 0.5 * logdet_sigma : -INFINITY;
  const double lp_old = logp[c];
  int clicks = 0;
  for (int i = 0; i < words; ++i) clicks += __popcll(prop[(size_t)c * words + i]);
  const int failed = (k_cap > 0 && clicks > k_cap) ? -1 : (r.status == TOR_EPREC) ? -2 : -3;
  bool acc = false;
  if (lp_new > -INFINITY) {
    if (lp_old == -INFINITY) {
      acc = true;
    } else {
      const double log_alpha = (lp_new - lp_old) + (logq[c] - logq_prop[c]);
      const double u = philox_uniform(seed, step, (uint32_t)c, (uint32_t)M);
      acc = log(u) < log_alpha;
    }
  }
  if (acc) {
    for (int i = 0; i < words; ++i) pat[(size_t)c * words + i] = prop[(size_t)c * words + i];
    logp[c] = lp_new;
    logq[c] = logq_prop[c];
  }
  accepted[c] = acc ? 1 : (lp_new > -INFINITY ? 0 : failed);
}

// Delayed acceptance (Christen & Fox 2005) with a surrogate density s (the
// MADE network's log q): a plain proposal S' first passes a test on the
// surrogate, min(1, s(S') q(S) / (s(S) q(S'))) with draw j = M; only then is
// its exact p(S') computed, and the second test min(1, p(S') s(S) / (p(S) s(S')))
// with draw j = M + 1 corrects the surrogate's error exactly, so the chain
// still targets p.  Screened-out proposals (and those over the click cap) are
// replaced by the empty pattern in `eval`, whose Torontonian costs nothing.
__global__ void k_screen(int C, int M, int words, int k_cap, const unsigned long long *__restrict__ prop,
                         const double *__restrict__ logq_prop, const double *__restrict__ logs_prop,
                         const double *__restrict__ logp, const double *__restrict__ logq,
                         const double *__restrict__ logs, unsigned long long *__restrict__ eval,
                         int *__restrict__ accepted, unsigned long long seed, unsigned long long step) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int clicks = 0;
  for (int i = 0; i < words; ++i) clicks += __popcll(prop[(size_t)c * words + i]);
  int code = 1;                      // 1: evaluate exactly
  if (k_cap > 0 && clicks > k_cap) {
    code = -1;
  } else if (logp[c] > -INFINITY) {  // an initialised chain: the surrogate's test first
    const double log_alpha = (logs_prop[c] - logs[c]) + (logq[c] - logq_prop[c]);
    const double u = philox_uniform(seed, step, (uint32_t)c, (uint32_t)M);
    if (!(log(u) < log_alpha)) code = -4;
  }
  for (int i = 0; i < words; ++i) eval[(size_t)c * words + i] = (code == 1) ? prop[(size_t)c * words + i] : 0ull;
  accepted[c] = code;
}

__global__ void k_accept_da(int C, int M, int words, double logdet_sigma, const tor_result *__restrict__ tr,
                            const unsigned long long *__restrict__ prop, const double *__restrict__ logq_prop,
                            const double *__restrict__ logs_prop, unsigned long long *__restrict__ pat,
                            double *__restrict__ logp, double *__restrict__ logq, double *__restrict__ logs,
                            int *__restrict__ accepted, unsigned long long seed, unsigned long long step) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  if (accepted[c] != 1) return;  // over the cap (-1) or screened out by the surrogate (-4)
  const tor_result r = tr[c];
  const double tor = r.hi + r.lo;
  const double lp_new = (r.status == TOR_OK && tor > 0.0) ? log(tor) - 0.5 * logdet_sigma : -INFINITY;
  const double lp_old = logp[c];
  bool acc = false;
  if (lp_new > -INFINITY) {
    if (lp_old == -INFINITY) {
      acc = true;
    } else {
      const double log_alpha = (lp_new - lp_old) + (logs[c] - logs_prop[c]);
      const double u = philox_uniform(seed, step, (uint32_t)c, (uint32_t)(M + 1));
      acc = log(u) < log_alpha;
    }
  }
  if (acc) {
    for (int i = 0; i < words; ++i) pat[(size_t)c * words + i] = prop[(size_t)c * words + i];
    logp[c] = lp_new;
    logq[c] = logq_prop[c];
    logs[c] = logs_prop[c];
  }
  accepted[c] = acc ? 1 : (lp_new > -INFINITY ? 0 : (r.status == TOR_EPREC ? -2 : -3));
}

int launch_screen(int C, int M, int words, int k_cap, const unsigned long long *prop, const double *logq_prop,
                  const double *logs_prop, const double *logp, const double *logq, const double *logs,
                  unsigned long long *eval, int *accepted, unsigned long long seed, unsigned long long step,
                  cudaStream_t s) {
  k_screen<<<(C + 127) / 128, 128, 0, s>>>(C, M, words, k_cap, prop, logq_prop, logs_prop, logp, logq, logs, eval,
                                           accepted, seed, step);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_accept_da(int C, int M, int words, double logdet_sigma, const tor_result *tr,
                     const unsigned long long *prop, const double *logq_prop, const double *logs_prop,
                     unsigned long long *pat, double *logp, double *logq, double *logs, int *accepted,
                     unsigned long long seed, unsigned long long step, cudaStream_t s) {
  k_accept_da<<<(C + 127) / 128, 128, 0, s>>>(C, M, words, logdet_sigma, tr, prop, logq_prop, logs_prop, pat, logp,
                                              logq, logs, accepted, seed, step);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_propose_plain(const double *marg, int M, int C, int words, unsigned long long seed,
                         unsigned long long step, unsigned long long *prop, double *logq_prop, cudaStream_t s) {
  k_propose_plain<<<(C + 127) / 128, 128, 0, s>>>(marg, M, C, words, seed, step, prop, logq_prop);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_accept(int C, int M, int words, int k_cap, double logdet_sigma, const tor_result *tr,
                  const unsigned long long *prop, const double *logq_prop, unsigned long long *pat, double *logp,
                  double *logq, int *accepted, unsigned long long seed, unsigned long long step, cudaStream_t s) {
  k_accept<<<(C + 127) / 128, 128, 0, s>>>(C, M, words, k_cap, logdet_sigma, tr, prop, logq_prop, pat, logp, logq, accepted,
                                           seed, step);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tor
