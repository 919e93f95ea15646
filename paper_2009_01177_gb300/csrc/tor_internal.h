// tor_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include "../../include/torontonian.h"
#include "fixacc.cuh"

namespace tor {

// a-posteriori error model: |error| <= gamma(k) * u * sum_Z t_Z.  Each term
// carries the rounding of one 2x2 determinant, one reciprocal square root and
// one product per level of its subset (at most k levels), plus the backward
// error of the Schur updates; gamma = 4k covers those with margin.
__host__ __device__ inline double err_gamma(int k) { return 4.0 * (k > 1 ? k : 1); }
// fixed point: absolute rounding 2^-104 per product, relative 2^-100 for the
// values >= 1/16 the walk carries (Schur entries, pivots, terms); 256-bit
// class (nine 29-bit limbs, 203 fraction bits): at most 3.5 units of 2^-203
// per product or fused two-product operation, under 2^-197 relative on values
// >= 1/16, 2^-196 with margin
__host__ __device__ inline double unit_roundoff(int tier) {
  return tier == TOR_PREC_DD      ? 0x1p-104
         : tier == TOR_PREC_FX128 ? 0x1p-100
         : tier == TOR_PREC_FX256 ? 0x1p-196
                                  : 0x1p-53;
}
constexpr int FX128_FRAC = 104;
// largest log2 t_max for which every intermediate fits: 2 log2 t_max < 127 - F - 1
constexpr float FX128_MAX_LOG2_TMAX = 11.0f;
// the 256-bit-class tier holds magnitudes below 2^57; the pivot inverses reach
// t_max^2 and the Schur coefficients D^-1 u a few times that, so t_max <= 2^26
constexpr float FX256_MAX_LOG2_TMAX = 26.0f;
// walked modes per fx9 chunk: its 64-bit column sums take at most 2^34 terms
constexpr int FX256_MAX_R1 = 34;

// device arrays of a batch plan (sized for n_max instances by tor_batch_reserve)
struct BatchPlan {
  unsigned char *tier;            // n: 0 = not scheduled (invalid), else TOR_PREC_FP64 | DD | FX128 | FX256
  unsigned char *r1;              // n: walked (low) modes per chunk
  unsigned char *escalated;       // n: re-run one tier up by the current AUTO round
  int *key;                       // n: sort key, -1 = not scheduled
  int *order;                     // n: instances sorted by (tier, r1 descending)
  int *flags;                     // n: ST_* status bits
  unsigned long long *item_off;   // n + 1: exclusive scan of chunk counts in sorted order
  unsigned long long *acc;        // n x 16: exact fixed-point sums (signed, abs; 4 or 8 limbs each)
  unsigned long long *range;      // 8: [begin, end) item range of each tier (FP64, DD, FX128, FX256)
  unsigned long long *counter;    // 4: work counter of each tier
  unsigned int *counts;           // 4: scheduled instances of tiers <= FP64, <= DD, <= FX128, <= FX256
  tor_result *result;             // n: last finalized results (input of the AUTO round)
};

// what a batch walks: per-instance matrices, or click patterns of one full matrix
struct BatchInput {
  const double *const *O;              // instance mode: n matrices (2k_i x 2k_i, `layout`)
  const int *k;                        // n click counts (pattern mode: popcounts, filled by the library)
  const int *ld;                       // instance mode: n leading dimensions
  int layout;
  const double *Ofull;                 // pattern mode: full 2M x 2M O, xxpp, leading dim ldfull
  const unsigned long long *patterns;  // pattern mode: n x words bitsets (bit j = mode j clicked)
  int M, ldfull, words;                // words == 0 selects instance mode
};

int launch_batch_plan(const int *k, const tor_bound *bounds, int n, int prec, int kmax,
                      const unsigned char *r1_table, int mode, double tol, const BatchPlan &p, cudaStream_t s);
int launch_batch_walk(int tier, int grid, int block, const BatchInput &in, const BatchPlan &p, double *scratch,
                      cudaStream_t s);
int launch_pattern_popcount(const unsigned long long *patterns, int n, int words, int *k, cudaStream_t s);
int launch_bounds_patterns(const double *Ofull, int M, int ld, const unsigned long long *patterns, int words,
                           int n, double tol, tor_bound *out, cudaStream_t s);
int launch_batch_finalize(const int *k, int n, int only_escalated, double tol, const BatchPlan &p,
                          tor_result *out, cudaStream_t s);
int batch_walk_max_blocks_per_sm(int tier, int block, bool patterns);

void launch_prep(const double *O, int k, int ld, int layout, double *B, double *Blo, cudaStream_t s);
// Up to two chunk segments per walk launch: segment 0 walks chunks [c0, c1)
// of r1 low modes each; segment 1 (empty when c0 == c1) walks finer chunks of
// a smaller r1.  Every thread takes its grid-stride share of segment 0 and
// then of segment 1, so a partial last wave of segment 0 can be cut into
// finer pieces that fill the machine.
struct WalkSegs {
  int r1[2];
  unsigned long long c0[2], c1[2];
};
inline WalkSegs one_segment(int r1, unsigned long long c0, unsigned long long c1) {
  return WalkSegs{{r1, r1}, {c0, 0ull}, {c1, 0ull}};
}
void launch_dfs(int tier, int grid, int block, const double *B, const double *Blo, int k, const WalkSegs &seg,
                double *scratch, unsigned long long *block_part, unsigned long long *chunk_part, int *status,
                cudaStream_t s);
void launch_finalize(const unsigned long long *block_part, int nblocks, int k, int tier,
                     const int *status, tor_result *out, cudaStream_t s);
void launch_dfma_peak(double *sink, int grid, int block, int iters, cudaStream_t s);
void launch_imad_peak(long long *sink, int grid, int block, int iters, cudaStream_t s);
// writes Tor = 1 (the k = 0 result) of tier `tier` to out, on the stream
int launch_result_one(tor_result *out, int tier, cudaStream_t s);
// all-pattern tables (tor_table.cu)
int table_walk_max_blocks_per_sm(int tier, int block);
int launch_table_walk(int tier, int grid, int block, const double *B, const double *Blo, int k, int r1,
                      double *scratch, const unsigned int *order, Fx256 *table, int *status, cudaStream_t s);
int launch_table_transform(Fx256 *t, double *s, int M, cudaStream_t st);
int launch_table_finalize(const Fx256 *t, const double *s, int M, int tier, const int *status, tor_result *out,
                          cudaStream_t st);
int launch_fx256_fma2(const int *s, const int *a1, const int *b1, const int *a2, const int *b2, int n, int *out,
                      int *ovf, cudaStream_t st);
int scratch_entries(int tier, int k, int r1);
int dfs_max_blocks_per_sm(int tier, int block);
int launch_bounds_batch(const double *const *O, const int *k, const int *ld, int n, int layout, double tol,
                        tor_bound *out, cudaStream_t s);
int launch_bounds_single(const double *O, int k, int ld, int layout, double tol, tor_bound *out,
                         cudaStream_t s);
int launch_propose_plain(const double *marg, int M, int C, int words, unsigned long long seed,
                         unsigned long long step, unsigned long long *prop, double *logq_prop, cudaStream_t s);
int launch_accept(int C, int M, int words, int k_cap, double logdet_sigma, const tor_result *tr,
                  const unsigned long long *prop, const double *logq_prop, unsigned long long *pat, double *logp,
                  double *logq, int *accepted, unsigned long long seed, unsigned long long step, cudaStream_t s);
int launch_screen(int C, int M, int words, int k_cap, const unsigned long long *prop, const double *logq_prop,
                  const double *logs_prop, const double *logp, const double *logq, const double *logs,
                  unsigned long long *eval, int *accepted, unsigned long long seed, unsigned long long step,
                  cudaStream_t s);
int launch_accept_da(int C, int M, int words, double logdet_sigma, const tor_result *tr,
                     const unsigned long long *prop, const double *logq_prop, const double *logs_prop,
                     unsigned long long *pat, double *logp, double *logq, double *logs, int *accepted,
                     unsigned long long seed, unsigned long long step, cudaStream_t s);
int mlp_modes(const tor_mlp *m);
// store a message for tor_last_error() on the calling thread; returns code
int record_error(int code, const char *msg);

}  // namespace tor
