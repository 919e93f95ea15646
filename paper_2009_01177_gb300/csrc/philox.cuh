// philox.cuh -- Philox4x32-10 counter-based random numbers (Salmon, Moraes,
// Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011).
//
// Written from the published definition: 10 rounds of two 32x32->64-bit
// multiplications (multipliers 0xD2511F53 and 0xCD9E8D57) with the key
// bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.
// The MH sampler keys every draw by (seed; step, chain, index), so a draw is
// a pure function of its coordinates and any run can be replayed on the CPU.
#pragma once
#include <cstdint>

namespace tor {

struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void mulhilo32(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
  const uint64_t p = (uint64_t)a * (uint64_t)b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c.x, hi0, lo0);
    mulhilo32(0xCD9E8D57u, c.z, hi1, lo1);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// Uniform double in (0, 1) with 53 random bits, the j-th draw of
// (seed; step, chain): counter (step lo, step hi, chain, j/2), key (seed lo, seed hi);
// draw j uses words (x, y) for even j and (z, w) for odd j:
// u = ((a >> 6) * 2^27 + (b >> 5) + 1/2) * 2^-53.
__host__ __device__ inline double philox_uniform(uint64_t seed, uint64_t step, uint32_t chain, uint32_t j) {
  const U4 r = philox4x32_10(U4{(uint32_t)step, (uint32_t)(step >> 32), chain, j >> 1}, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
  const uint32_t a = (j & 1) ? r.z : r.x, b = (j & 1) ? r.w : r.y;
  const uint64_t m = ((uint64_t)(a >> 6) << 27) | (uint64_t)(b >> 5);
  return ((double)m + 0.5) * 0x1p-53;
}

}  // namespace tor
