// tor_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include "../../include/torontonian.h"

namespace tor {

// a-posteriori error model: |error| <= gamma(k) * u * sum_Z t_Z.  Each term
// carries the rounding of one 2x2 determinant, one reciprocal square root and
// one product per level of its subset (at most k levels), plus the backward
// error of the Schur updates; gamma = 4k covers those with margin.
__host__ __device__ inline double err_gamma(int k) { return 4.0 * (k > 1 ? k : 1); }
__host__ __device__ inline double unit_roundoff(int tier) {
  return tier == TOR_PREC_DD ? 0x1p-104 : 0x1p-53;
}

__host__ __device__ void fixed_to_result(const unsigned long long *w8, int k, int tier, int status,
                                         tor_result *out);

void launch_prep(const double *O, int k, int ld, int layout, double *B, double *Blo, cudaStream_t s);
void launch_dfs(int tier, int grid, int block, const double *B, const double *Blo, int k, int r1,
                unsigned long long c0, unsigned long long c1, double *scratch,
                unsigned long long *block_part, unsigned long long *chunk_part, int *status,
                cudaStream_t s);
void launch_finalize(const unsigned long long *block_part, int nblocks, int k, int tier,
                     const int *status, tor_result *out, unsigned long long *total8, cudaStream_t s);
void launch_dfma_peak(double *sink, int grid, int block, int iters, cudaStream_t s);
int scratch_entries(int tier, int k, int r1);
int dfs_max_blocks_per_sm(int tier, int block);
// store a message for tor_last_error() on the calling thread; returns code
int record_error(int code, const char *msg);

}  // namespace tor
