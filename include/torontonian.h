/*
 * torontonian.h -- C ABI of the GB300 (sm_103a) Torontonian library.
 *
 * The library evaluates the Torontonian of a threshold-detection Gaussian
 * boson sampling click pattern (paper Sec. 3.1, Eq. 2):
 *
 *     Tor(O) = sum_{Z subset of [k]} (-1)^(k-|Z|) / sqrt(det(I - O_Z))
 *
 * where O is the 2k x 2k real-quadrature matrix O_S of the clicked modes,
 * O = I - Sigma^-1 (the paper's A), and O_Z keeps the x and p rows/columns
 * of the modes in Z (selection rule under Eq. 1).  The click probability of
 * Eq. 1 is p(S) = Tor(O_S) / sqrt(det Sigma).
 *
 * Conventions shared by every entry point
 *   - Matrices are FP64, row-major, with a leading dimension `ld` (in
 *     elements, ld >= 2k).  TOR_LAYOUT_XXPP is the paper's order (rows
 *     0..k-1 = x of the clicked modes, k..2k-1 = p); TOR_LAYOUT_XPXP is
 *     mode-interleaved (x_0, p_0, x_1, p_1, ...).
 *   - Pointers marked `dev` are device memory on the context's GPU, owned by
 *     the caller; pointers marked `host` are host memory owned by the caller.
 *     The library keeps no pointer after a call returns.
 *   - The library allocates device memory only inside a context (workspace
 *     that grows on demand and is released by tor_destroy).
 *   - Calls taking a stream enqueue work on it.  Entry points that write a
 *     `host` result synchronise that stream before returning; the others
 *     return after enqueueing and their `dev` results are valid once the
 *     stream has been synchronised.
 *   - Every entry point returns a TOR_* status; no C++ exception crosses the
 *     ABI.  tor_last_error() gives a message for the calling thread.
 *   - k = 0 gives Tor = 1 (only the empty set).  k > TOR_MAX_K is TOR_EINVAL.
 *   - A matrix for which some I - O_Z is not positive definite (a pivot
 *     <= 0, or not finite) gives TOR_ENOTPD and the result's status field is
 *     set; the numeric fields are then meaningless.
 *
 * Accuracy
 *   Subset terms t_Z = 1/sqrt(det(I - O_Z)) are computed in the tier's
 *   arithmetic (FP64, double-double, or 128- or 256-bit fixed point) and
 *   summed EXACTLY in fixed point (256-bit; 512-bit for the 256-bit tier), so
 *   the only error is the per-term rounding.  Each result
 *   carries sum_abs = sum_Z t_Z (condition number kappa = sum_abs/|Tor|) and
 *   err_est = gamma * u_tier * sum_abs, an a-posteriori bound on |error|.
 */
#ifndef TORONTONIAN_H
#define TORONTONIAN_H

#include <stdint.h>
#include <stddef.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TOR_MAX_K 64
#define TOR_LEVELS_MAX_K 48   /* largest k tor_levels takes */

enum {
    TOR_OK = 0,
    TOR_EINVAL = 1,     /* bad argument (size, pointer, enum) */
    TOR_ENOTPD = 2,     /* some I - O_Z not positive definite */
    TOR_ECUDA = 3,      /* a CUDA runtime call failed */
    TOR_ETIMEOUT = 4,   /* a device-side wait exceeded its spin limit */
    TOR_EPREC = 5,      /* the result's a-posteriori error exceeds the requested tolerance */
    TOR_ENOMEM = 6      /* workspace allocation failed */
};

enum { TOR_PREC_AUTO = 0, TOR_PREC_FP64 = 1, TOR_PREC_DD = 2, TOR_PREC_FX128 = 3, TOR_PREC_FX256 = 4 };
/* TOR_PREC_FX128: the paper's 128-bit fixed point with one scaling factor
 * (Sec. 5.1-5.2), 104 fraction bits, on the integer pipe.  Every intermediate
 * must stay below 2^23 in magnitude; the largest are the pivot inverses
 * 1/det2 <= t_max^2 with t_max = 1/sqrt(det(I - O)), so tor_single requires
 * t_max <= 2^11 (checked by the bound pass, TOR_EINVAL otherwise); a product
 * that still leaves the range sets the result's status to TOR_EINVAL.
 * Available in tor_single, tor_single_async, tor_chunks and tor_batch (the
 * asynchronous single and chunk calls do not run the range check).
 * TOR_PREC_FX256: the paper's 256-bit mode (Sec. 5.1-5.2) in nine 29-bit
 * signed limbs: 203 fraction bits, magnitudes below 2^57, so t_max <= 2^26 is
 * required (the pivot inverses reach t_max^2, the Schur coefficients a few
 * times that).  Its exact partial sums are 512-bit with 256 fraction bits:
 * tor_chunks writes 16 limbs per chunk for it (two 8-limb values) instead of
 * 8, and a chunk walks at most 2^34 subsets (k - chunk_bits <= 34).
 * Available in tor_single, tor_single_async, tor_chunks and tor_batch. */
enum { TOR_LAYOUT_XXPP = 0, TOR_LAYOUT_XPXP = 1 };

typedef struct tor_ctx tor_ctx;

/* Tor as a double-double hi + lo, with its error model. */
typedef struct {
    double hi, lo;      /* Tor = hi + lo */
    double sum_abs;     /* sum_Z t_Z (>= |Tor|) */
    double err_est;     /* a-posteriori bound on |computed - exact| */
    int tier;           /* TOR_PREC_FP64, _DD, _FX128 or _FX256: arithmetic used */
    int status;         /* TOR_OK or TOR_ENOTPD for this instance */
} tor_result;

/* FP32 bound pass output (paper Sec. 5.1 bounds, Eq. bitlen of Sec. 5.4). */
typedef struct {
    float log_tmax;       /* ln t_max = -1/2 ln det(I - O): the largest term (Sec. 5.1 upper bound) */
    float log_tor_est;    /* ln of the product estimate prod_j (tau_j - 1) of Tor */
    float log_kappa_est;  /* ln of the estimated condition number sum t / |Tor| */
    float bits_needed;    /* log2 kappa_est + log2(gamma) + log2(1/tol) */
    int tier;             /* routed tier: TOR_PREC_FP64, _FX128, _FX256 or _DD (see tor_bounds) */
} tor_bound;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  Returns TOR_OK or an error.
 * A context owns its workspaces and is used by one host thread at a time
 * (calls on it do not lock); separate contexts, on the same device or not,
 * may be used concurrently.  tor_single_noalloc and tor_levels take no
 * context: tor_levels uses only the caller's workspace; tor_single_noalloc
 * calls share one fixed array, so calls whose GPU work could overlap must be
 * serialised by the caller. */
int tor_create(tor_ctx **ctx, int device);

/* Release the context and its workspace (NULL is ignored). */
void tor_destroy(tor_ctx *ctx);

/* Message of the last error raised on the calling thread ("" if none). */
const char *tor_last_error(void);

/* Launch shape used by the DFS kernels: threads per block and blocks per SM
 * (0 = library default).  Takes effect on the next call. */
int tor_set_launch(tor_ctx *ctx, int threads_per_block, int blocks_per_sm);

/* Chunk depth d used by tor_single: chunks fix the top d modes of the subset
 * mask and each walks the 2^(k-d) subsets of the remaining modes.  -1 selects
 * the library's automatic choice (the default). */
int tor_set_chunk_bits(tor_ctx *ctx, int chunk_bits);

/* --------------------------------------------------------------- Tor calls */

/*
 * tor_single: Tor of one 2k x 2k matrix (Eq. 2).
 *   O     dev  2k x 2k FP64, leading dimension ld, in `layout` order.
 *   prec  TOR_PREC_FP64, TOR_PREC_DD, TOR_PREC_FX128, TOR_PREC_FX256, or
 *         TOR_PREC_AUTO: the FP32 bound pass of tor_bounds picks the starting
 *         tier for relative tolerance `tol`; while the result's a-posteriori
 *         bound err_est exceeds tol * |Tor| it is recomputed in the next tier
 *         with more precision that fits the instance's range (FP64 -> FX128
 *         when t_max <= 2^11, else FX256 when t_max <= 2^26, else
 *         double-double; FX128 -> FX256 or double-double; double-double ->
 *         FX256), and when none is left the call returns TOR_EPREC with the
 *         result filled in.  `tol` is ignored for the explicit tiers; the
 *         fixed-point tiers return TOR_EINVAL for instances outside their
 *         range.
 *   out   host result; the call synchronises `stream`.
 * The 2^k subsets are split into equal prefix chunks (the high modes of the
 * subset mask fixed per chunk, Algorithm 1's balanced partition) walked
 * depth-first so that each subset's factor extends its parent's.
 */
int tor_single(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec,
               double tol, cudaStream_t stream, tor_result *out);

/*
 * tor_single_async: as tor_single, but the result goes to device memory
 * `out_dev` and the call returns after enqueueing (capturable in a CUDA
 * graph once the workspace has been sized by an earlier call with the same
 * k and precision).  prec: an explicit tier (TOR_PREC_FP64, _DD, _FX128 or
 * _FX256); the fixed-point range is not checked here (tor_single checks it),
 * a product that leaves the range sets the result's status to TOR_EINVAL.
 */
int tor_single_async(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec,
                     cudaStream_t stream, tor_result *out_dev);

/*
 * tor_chunks: partial sums over a range of prefix chunks, for sharding the
 * 2^k subsets across processes or calls, resuming long runs, and checking
 * sampled chunks against an independent evaluation.
 *   prec        an explicit tier (TOR_PREC_FP64, _DD, _FX128 or _FX256).
 *   chunk_bits  d in [0, min(k, 63)]: chunk c covers the subset masks
 *               [c 2^(k-d), (c+1) 2^(k-d)), i.e. modes k-d..k-1 are fixed by
 *               the bits of c.  k >= 1.
 *   c_begin, c_end  the chunk range [c_begin, c_end) to evaluate (TOR_EINVAL
 *               beyond 2^d).  Asynchronous on `stream`.
 *   part_dev    dev, (c_end - c_begin) x 8 uint64: per chunk the exact sum of
 *               (-1)^(k-|Z|) t_Z and of t_Z, each a 256-bit two's-complement
 *               fixed-point number with 128 fractional bits, little-endian
 *               64-bit limbs (limbs 0..3 = signed sum, 4..7 = sum_abs).  For
 *               TOR_PREC_FX256: x 16 uint64, two 512-bit values with 256
 *               fractional bits (limbs 0..7 and 8..15); its chunks walk at
 *               most 2^34 subsets (k - chunk_bits <= 34, else TOR_EINVAL).
 *   Partials of disjoint ranges add exactly (integer addition), so any split
 *   gives the same total bit for bit.
 */
int tor_chunks(tor_ctx *ctx, const double *O, int k, int ld, int layout, int prec,
               int chunk_bits, uint64_t c_begin, uint64_t c_end, cudaStream_t stream,
               uint64_t *part_dev);

/*
 * tor_single_noalloc: tor_single_async for callers that cannot allocate
 * device memory (no context; the paper has no counterpart -- this is a
 * library-integration entry point).  It performs no cudaMalloc or cudaFree:
 * all scratch lives in one fixed 48 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   O        dev  2k x 2k FP64, leading dimension ld, in `layout` order.
 *   prec     TOR_PREC_FP64 or TOR_PREC_DD.
 *   out_dev  dev  one tor_result, valid after `stream` is synchronised.
 * Runs on the current device.  Instances whose scratch exceeds the array are
 * rejected with TOR_EINVAL (on a 152-SM GB300: FP64 up to k = 25,
 * double-double up to k = 17).  All calls share the array: calls that
 * overlap on the GPU race and must be serialised by the caller.  The first
 * call on a device looks up the array's address; make it before any stream
 * capture.  Every call only enqueues work on `stream` (k = 0 included: its
 * constant result is written by a kernel).  Results equal tor_single's for
 * the same tier.
 */
int tor_single_noalloc(const double *O, int k, int ld, int layout, int prec,
                       cudaStream_t stream, tor_result *out_dev);

/*
 * tor_all_patterns: Tor(O_S) for EVERY click pattern S of one M-mode state.
 * For the full matrix, (O_S)_Z = O_Z (the selection rule of Eq. 1 applied
 * twice), so the terms t_Z = 1/sqrt(det(I - O_Z)) of Eq. 2 are shared by all
 * patterns and Tor(O_S) = sum over Z inside S of (-1)^(|S|-|Z|) t_Z is the
 * Moebius transform of the t table: one walk over the 2^M subsets stores
 * every t_Z exactly (256-bit fixed point, 128 fraction bits), and an integer
 * transform turns the table into all 2^M Torontonians.  2^M determinants
 * instead of 3^M; each result has the same error model as tor_single.
 *   O       dev  2M x 2M FP64 O = I - Sigma^-1, xxpp order, leading dim ld.
 *   prec    TOR_PREC_FP64, TOR_PREC_DD or TOR_PREC_FX128 (the state's
 *           t_max <= 2^11 is checked for the latter).
 *   out_dev dev  2^M results; entry S (bit j = mode j clicked) holds
 *           Tor(O_S), so p(S) = Tor(O_S) / sqrt(det Sigma).  A status bit
 *           raised by any subset (not positive definite) marks every entry.
 * Workspace: 40 bytes per pattern (M = 30: 43 GB) plus the walk's stacks.
 * Asynchronous on `stream` (it synchronises once when the walk-order table
 * is first made).  M in [1, TOR_TABLE_MAX_M].
 */
#define TOR_TABLE_MAX_M 30
int tor_all_patterns(tor_ctx *ctx, const double *O, int M, int ld, int prec, cudaStream_t stream,
                     tor_result *out_dev);

/*
 * tor_levels: Tor by the paper's own schedule, Algorithm 1 level by level
 * (all Z with |Z| = m together, m = 0..k) with each level's C(k, m) masks
 * shared out by Algorithm 2 (unranking, then the next mask of the same
 * popcount), and a fresh elimination of B_Z = I - O_Z for every subset, summed
 * exactly.  A second, independent GPU evaluation of Eq. 2 (another subset
 * order, another factorization of every term) for cross-checks beyond the CPU
 * oracle's reach; about k/3 times the work of tor_single's walk per subset.
 *   O, k, ld, layout   as for tor_single; k in [0, TOR_LEVELS_MAX_K].
 *   prec        TOR_PREC_FP64, TOR_PREC_DD or TOR_PREC_FX128 for every level,
 *   level_prec  host, k + 1 tiers for the levels m = 0..k (the paper's per-|Z|
 *               precision choice), or NULL to use prec throughout.
 *   workspace   dev, caller-owned, at least tor_levels_workspace() bytes.
 *   out_dev     dev, one result; err_est adds 4k u(tier) sum t over the levels
 *               and tier is the least precise tier used.
 * Asynchronous on `stream` (no allocation); failures are described by
 * tor_levels_last_error().
 */
int tor_levels_workspace(int k, int device, size_t *bytes);
int tor_levels(const double *O, int k, int ld, int layout, int prec, const int *level_prec, void *workspace,
               size_t workspace_bytes, cudaStream_t stream, tor_result *out_dev);
const char *tor_levels_last_error(void);

/* Algorithm 2's mask functions (host, no GPU).  tor_level_next_mask: the next
 * smaller mask with the same popcount (the paper's example: 010011 -> 001110),
 * 0 when none is left.  tor_level_kth_mask: the r-th (0-based) mask of
 * popcount m over k bits in decreasing order; TOR_EINVAL for r >= C(k, m). */
uint64_t tor_level_next_mask(uint64_t mask);
int tor_level_kth_mask(int k, int m, uint64_t r, uint64_t *mask);

/* tor_fx256_fma2: n elementwise s + a1 b1 + a2 b2 exactly as the
 * TOR_PREC_FX256 walk forms its Schur updates (Sec. 4.2 elimination in the
 * fixed point of Sec. 5.1-5.2), exposed so tests can check the arithmetic bit
 * for bit.  Each operand is n x 9 int32 limbs on the device, value
 * sum_i l_i 2^(29 i - 203) (any limbs below 2^29 in magnitude); the result
 * is n x 9 limbs in [-2^28, 2^28) whose value is the exact sum of the
 * product columns c >= 6 (limb pairs i + j >= 6) and of s, rounded to nearest
 * at 2^-203 (ties up); ovf_dev[i] = 1 when its magnitude reaches 2^57.  Asynchronous on
 * `stream`; TOR_EINVAL for n < 0 or null pointers. */
int tor_fx256_fma2(const int32_t *s_dev, const int32_t *a1_dev, const int32_t *b1_dev, const int32_t *a2_dev,
                   const int32_t *b2_dev, int n, int32_t *out_dev, int *ovf_dev, cudaStream_t stream);

/* Convert one fixed-point pair as written by tor_chunks (8 limbs, or 16 for
 * TOR_PREC_FX256), possibly summed over shards, to a tor_result (host, no
 * GPU needed). */
int tor_fixed_to_result(const uint64_t *limbs, int k, int tier, tor_result *out);

/* tor_sum_partials: the exact sum of n fixed-point pairs as written by
 * tor_chunks, the reduction over ranks that closes Algorithm 1 (each rank's
 * partial sum of Eq. 2's terms; Sec. 5.1-5.2 fixed point, so the sum is exact
 * and independent of the order).  Host code, no GPU needed.
 *   parts  host  n x 2L little-endian uint64 limbs per pair: the signed sum
 *                (L limbs, two's complement), then the sum of terms (L limbs);
 *                L = 8 for TOR_PREC_FX256, else 4.
 *   n           number of pairs, >= 0 (n = 0 writes zeros).
 *   tier        the tier that wrote them (TOR_PREC_FP64 .. TOR_PREC_FX256).
 *   out    host  2L limbs: both sums modulo 2^(64 L), caller-owned; it may
 *                alias parts' first pair.
 * TOR_EINVAL for null pointers, n < 0 or a bad tier. */
int tor_sum_partials(const uint64_t *parts, int n, int tier, uint64_t *out);

/*
 * tor_batch: Tor of n matrices of different k (e.g. the patterns a sampler
 * proposes), each by Eq. 2 (Sec. 3.1): the alternating sum over all 2^k_i
 * subsets Z of 1/sqrt(det(I - O_Z)), with Algorithm 1's balanced partition of
 * each instance's subsets into equal prefix chunks.  Scheduled on the
 * device: a plan kernel lays all (instance, chunk) pairs on one item axis per
 * tier, sorted by chunk size, and one persistent walk kernel per tier drains
 * it; partial sums are added exactly per instance.  Asynchronous; no host
 * round trip once the workspace is reserved, so the whole call can be
 * captured in a CUDA graph.
 *   O     dev  array of n device pointers (each 2k_i x 2k_i FP64, `layout`).
 *   k,ld  dev  arrays of n ints.
 *   prec  TOR_PREC_FP64, TOR_PREC_DD, TOR_PREC_FX128 or TOR_PREC_FX256
 *         (instances outside a fixed-point tier's range get TOR_EINVAL), or
 *         TOR_PREC_AUTO (per-instance tier from the bound pass, the
 *         precision choice of Sec. 5.4; results whose err_est exceeds
 *         tol * |Tor| are recomputed in the next tier with more precision that
 *         holds them, FP64 -> FX128 -> FX256, double-double outside the
 *         fixed-point ranges, in up to two more rounds; results still above
 *         get status TOR_EPREC).
 *   out   dev  n results; per-instance status TOR_OK, TOR_ENOTPD, TOR_EPREC,
 *         or TOR_EINVAL (k outside [0, TOR_MAX_K], or above the k_max of an
 *         explicit tor_batch_reserve).
 * Without an explicit tor_batch_reserve, every call reads k to the host to
 * size (and grow) the workspace, which synchronises `stream`.  After one, a
 * call allocates nothing unless n exceeds its n_max.
 */
int tor_batch(tor_ctx *ctx, const double *const *O, const int *k, const int *ld, int n,
              int layout, int prec, double tol, cudaStream_t stream, tor_result *out);

/*
 * tor_batch_patterns: tor_batch for n click patterns of one state, without
 * forming the submatrices: O_S is gathered on the fly from the full matrix by
 * the selection rule of Eq. 1 (rows/cols j and M + j of each clicked mode j).
 *   O         dev  2M x 2M FP64 O = I - Sigma^-1 in xxpp order, leading dim ld.
 *   patterns  dev  n x ceil(M/64) uint64 bitsets, bit j of word j/64 = mode j
 *             clicked (M <= 128; at most TOR_MAX_K clicks per pattern).
 *   out       dev  n results, Tor(O_S) of each pattern.  p(S) = Tor / sqrt(det Sigma).
 * Same scheduling and precision rules as tor_batch; the workspace is sized
 * for k_max = min(M, TOR_MAX_K) (allocating only when n or that k_max grows),
 * so every pattern of the state fits.
 */
int tor_batch_patterns(tor_ctx *ctx, const double *O, int M, int ld, const uint64_t *patterns, int n,
                       int prec, double tol, cudaStream_t stream, tor_result *out);

/* Size the batch workspace for up to n_max instances of at most k_max clicks
 * (allocates; call before capturing tor_batch in a CUDA graph).  From then on
 * tor_batch trusts the reservation: no host reads, instances with k > k_max
 * get status TOR_EINVAL. */
int tor_batch_reserve(tor_ctx *ctx, int n_max, int k_max);

/*
 * tor_bounds: FP32 bound pass (paper Sec. 5.1, Eq. upbound/lowbound; Sec. 5.4
 * Eq. bitlen) for n matrices; picks the tier needed for tolerance `tol`.
 *   O, k, ld  dev arrays as for tor_batch.   out  dev, n bounds.
 * Per instance: tau_j = 1/sqrt(det B_jj) of each mode's 2x2 block of
 * B = I - O; log_tor_est = sum ln(tau_j - 1); log_kappa_est =
 * sum ln(tau_j + 1) - log_tor_est; log_tmax = -1/2 ln det B from an FP32
 * Cholesky; bits_needed = log2 kappa_est + log2(4k) + log2(1/tol); tier =
 * TOR_PREC_FP64 if bits_needed <= 72 (FP64's 52 bits plus 20 bits of slack
 * for the estimate's pessimism; AUTO callers verify the result's
 * a-posteriori bound and escalate), else TOR_PREC_FX128 if t_max <= 2^11 and
 * bits_needed <= 120 (the fixed-point unit's 100 bits plus the same slack),
 * else TOR_PREC_DD if bits_needed <= 124, else TOR_PREC_FX256 if
 * t_max <= 2^26, else TOR_PREC_DD.  B not positive definite in FP32
 * gives bits_needed = +inf and tier TOR_PREC_DD.  An instance with k
 * outside [0, TOR_MAX_K] or a null matrix gets tier 0 and NaN fields.
 * The estimates are heuristic: on Haar-mixed lossy GBS states kappa_est
 * over-estimates the true condition number by 10^2 to 10^13.
 */
int tor_bounds(tor_ctx *ctx, const double *const *O, const int *k, const int *ld, int n,
               int layout, double tol, cudaStream_t stream, tor_bound *out);

/* ----------------------------------------------- learned proposal (MADE) */

/*
 * A masked autoregressive network over click patterns, the proposal of an
 * independence Metropolis-Hastings sampler (the paper samples by MCMC,
 * Sec. 7.1.1, without fixing the proposal; this network is the project's
 * addition).  q(x) = prod_j Bernoulli(x_j; sigmoid(l_j(x_<j))), l from an MLP
 * M -> hidden -> hidden -> hidden -> M with ReLU and MADE masks (input j has
 * degree j+1, hidden unit h degree 1 + (h mod (M-1)), output j sees hidden
 * units of degree <= j).  BF16 weights on tensor cores, FP32 accumulation,
 * FP32 master weights with masked Adam (beta 0.9 / 0.999, eps 1e-8).
 * Parameter order for get/set: W1[hidden x M], b1, W2, b2, W3, b3,
 * W4[M x hidden], b4[M], row-major.  Calls run on the current device;
 * functions with host pointers synchronise.
 */
typedef struct tor_mlp tor_mlp;
int tor_mlp_create(tor_ctx *ctx, int M, int hidden, uint64_t seed, tor_mlp **out);
void tor_mlp_destroy(tor_mlp *m);
int tor_mlp_num_params(const tor_mlp *m);
/* which: 0 weights, 1 gradients of the last grad/train call, 2 the 0/1 masks */
int tor_mlp_get_params(const tor_mlp *m, float *host, int which);
int tor_mlp_set_params(tor_mlp *m, const float *host);   /* masked entries forced to 0 */
/* start at the plain proposal: last layer 0, output biases logit(marg_host[j]) */
int tor_mlp_set_marginals(tor_mlp *m, const double *marg_host);
/* log q(x) for B patterns (dev bitsets, ceil(M/64) words each) -> dev doubles */
int tor_mlp_logq(tor_mlp *m, const uint64_t *patterns, int B, double *logq, cudaStream_t stream);
/* the M logits of each pattern, to host (B x M floats) */
int tor_mlp_logits(tor_mlp *m, const uint64_t *patterns, int B, float *logits_host);
/* gradients of L = -(sum_b w_b log q(x_b)) / sum_b w_b (w: dev, B floats); loss to host if non-null */
int tor_mlp_grad(tor_mlp *m, const uint64_t *patterns, const float *w, int B, float *loss_host,
                 cudaStream_t stream);
/* one Adam step on L with learning rate lr */
int tor_mlp_train_step(tor_mlp *m, const uint64_t *patterns, const float *w, int B, float lr,
                       float *loss_host, cudaStream_t stream);
/* B ancestral samples (dev bitsets out) and their log q (dev); draw j of sample b
 * is Philox4x32-10 at (seed; step, b, j) */
int tor_mlp_sample(tor_mlp *m, int B, uint64_t seed, uint64_t step, uint64_t *patterns, double *logq,
                   cudaStream_t stream);

/* ------------------------------------------------------------ MH sampling */

/*
 * gbs_sample_step: one independence Metropolis-Hastings step of C chains
 * targeting p(S) = Tor(O_S) / sqrt(det Sigma) (Eq. 1).
 *   O             dev  full 2M x 2M O = I - Sigma^-1, xxpp, leading dim ld (M <= 128).
 *   logdet_sigma  ln det Sigma.
 *   marg_p        dev  M single-mode click probabilities (plain proposal:
 *                 independent Bernoulli per mode); ignored when proposal != NULL.
 *   proposal      NULL for the plain proposal, or a tor_mlp over the same M.
 *   patterns      dev  C x ceil(M/64) uint64 chain states (in/out).
 *   logp, logq    dev  C doubles: ln p and ln q of the current states (in/out);
 *                 logp = -inf marks an uninitialised chain (accepts any
 *                 proposal with p > 0).  After retraining the network, refresh
 *                 logq of the current states with tor_mlp_logq.
 *   accepted      dev  C ints: 1 the proposal was accepted; 0 it was rejected
 *                 by the Metropolis-Hastings test; negative, it was rejected
 *                 because p(S') is not known to the tolerance, so that callers
 *                 can count those rejections: -1 more clicks than k_cap (not
 *                 evaluated), -2 its Torontonian missed tol in the most precise
 *                 tier whose range holds it (TOR_EPREC), -3 any other failed
 *                 evaluation (not positive definite, out of range) or Tor <= 0.
 *   seed, step    Philox4x32-10 key and counter: draw j of chain c is at
 *                 (seed; step, c, j), j < M for the proposal, j = M to accept.
 *   prec, tol     tier for the exact Torontonians, as for tor_batch.
 *   k_cap         > 0: proposals with more than k_cap clicks are rejected without
 *                 evaluating them (an exact Torontonian costs 2^k), so the chains
 *                 target p(S | |S| <= k_cap); <= 0: no cap beyond TOR_MAX_K.
 * Asynchronous; the Torontonians use tor_batch_patterns' workspace rules.
 */
int gbs_sample_step(tor_ctx *ctx, const double *O, int M, int ld, double logdet_sigma,
                    const double *marg_p, tor_mlp *proposal, int C, uint64_t *patterns,
                    double *logp, double *logq, int *accepted, uint64_t seed, uint64_t step,
                    int prec, double tol, int k_cap, cudaStream_t stream);

/*
 * gbs_sample_step_da: one Metropolis-Hastings step of C chains targeting
 * p(S) = Tor(O_S) / sqrt(det Sigma) (Eq. 1, the paper's MCMC use, Sec. 7.1.1)
 * by delayed acceptance (Christen & Fox 2005) with the network as a cheap
 * surrogate of p: the plain proposal S' (as in gbs_sample_step) first passes
 * a test on the surrogate, min(1, s(S') q(S) / (s(S) q(S'))), Philox draw
 * j = M; only the proposals that pass have their exact Torontonian computed,
 * and a second test, min(1, p(S') s(S) / (p(S) s(S'))), draw j = M + 1,
 * corrects the surrogate's error exactly, so the chain targets p whatever the
 * surrogate.  Acceptance always rests on the exact Torontonian.
 *   surrogate  a tor_mlp over the same M (s = its normalised density q_net).
 *   logs       dev  C doubles: ln s of the current states (in/out; refresh
 *              with tor_mlp_logq after retraining the network).
 *   accepted   as gbs_sample_step, plus -4: rejected by the surrogate's test
 *              (no Torontonian computed).  An uninitialised chain (logp = -inf)
 *              skips the surrogate's test.
 * The other arguments are those of gbs_sample_step (marg_p required).
 */
int gbs_sample_step_da(tor_ctx *ctx, const double *O, int M, int ld, double logdet_sigma, const double *marg_p,
                       tor_mlp *surrogate, int C, uint64_t *patterns, double *logp, double *logq, double *logs,
                       int *accepted, uint64_t seed, uint64_t step, int prec, double tol, int k_cap,
                       cudaStream_t stream);

/* -------------------------------------------------------------- utilities */

/* Kernel timing: when `on`, the walk kernel of every later call is bracketed
 * by CUDA events recorded on that call's stream. */
int tor_set_timing(tor_ctx *ctx, int on);

/* Duration in ms of the walk kernel of the most recent timed call (waits for
 * that kernel to finish).  TOR_EINVAL if no timed call was made. */
int tor_walk_time(tor_ctx *ctx, float *ms);

/* Duration in ms of the transform passes (sums of terms, then the Moebius
 * transform over all mask bits) of the most recent timed tor_all_patterns
 * call.  TOR_EINVAL if there was none. */
int tor_transform_time(tor_ctx *ctx, float *ms);

/*
 * tor_autotune: pick the chunk depth d (walked modes per chunk k - d) and
 * blocks per SM that run fastest for instances of k clicks in tier `prec`,
 * by timing candidates (k - d in {8, 10, 12, 13, 14, 15, 16}, 2-4 blocks per SM) on a
 * synthetic instance of that size (the walk's cost depends only on k); each
 * candidate walks two waves of chunks (or all of them, when fewer) whose
 * high chunk bits are half set, and its time is scaled to all 2^d.  The
 * choice is kept in the context (used by tor_single when chunk bits are
 * automatic, and by the batch planner for that k) and, if cache_path is not
 * NULL, appended to that file as one JSON object per line keyed by GPU name,
 * k and tier; a matching cached line is reused without timing.  Synchronous;
 * allocates a small instance.  k in [1, 40].
 */
int tor_autotune(tor_ctx *ctx, int k, int prec, const char *cache_path, int *chunk_bits_out,
                 int *blocks_per_sm_out);

/* Measured FP64 FMA throughput of this GPU (DFMA per second), from a
 * dependent-chain-free DFMA loop over all SMs; the roofline denominator. */
int tor_fp64_peak(tor_ctx *ctx, double *dfma_per_s, double *sm_clock_hz);

/* Measured throughput of the integer multiply-add that the fixed-point tiers
 * are built on: signed 32 x 32 -> 64-bit multiply-adds (mad.wide.s32) per
 * second, from independent chains over all SMs; the roofline denominator of
 * the 256-bit-class tier (whose limb products are exactly these operations). */
int tor_int_peak(tor_ctx *ctx, double *mad_per_s);

#ifdef __cplusplus
}
#endif
#endif /* TORONTONIAN_H */
