// tor_partials.cu -- tor_sum_partials: the exact reduction of partial sums.
//
// Algorithm 1 splits the subset masks over ranks and closes with a sum of the
// ranks' partial results.  The partials here are fixed point with one scale
// (Sec. 5.1-5.2), so that sum is integer addition: exact, and the same in any
// order or grouping.  Each partial is a pair of L-limb little-endian two's
// complement integers (the signed sum of Eq. 2's terms, then the sum of their
// magnitudes), L = 8 for the 256-bit tier and 4 otherwise, as tor_chunks
// writes them.  Host code only.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>
#include "tor_internal.h"

int tor_sum_partials(const uint64_t *parts, int n, int tier, uint64_t *out) {
  char msg[96];
  if (!parts || !out) return tor::record_error(TOR_EINVAL, "null pointer");
  if (n < 0) {
    std::snprintf(msg, sizeof msg, "n = %d < 0", n);
    return tor::record_error(TOR_EINVAL, msg);
  }
  if (tier < TOR_PREC_FP64 || tier > TOR_PREC_FX256) return tor::record_error(TOR_EINVAL, "bad tier");
  const int L = (tier == TOR_PREC_FX256) ? 8 : 4;
  uint64_t acc[16] = {0};
  for (int i = 0; i < n; ++i) {
    const uint64_t *p = parts + (size_t)i * 2 * L;
    for (int h = 0; h < 2; ++h) {  // the signed sum, then the sum of magnitudes
      uint64_t carry = 0;
      for (int m = 0; m < L; ++m) {
        const uint64_t a = acc[h * L + m], b = p[h * L + m];
        const uint64_t s1 = a + b, c1 = s1 < a ? 1u : 0u;
        const uint64_t s2 = s1 + carry, c2 = s2 < s1 ? 1u : 0u;
        acc[h * L + m] = s2;
        carry = c1 + c2;
      }
    }
  }
  for (int m = 0; m < 2 * L; ++m) out[m] = acc[m];
  return TOR_OK;
}
