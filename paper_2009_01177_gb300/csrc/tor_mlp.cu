// tor_mlp.cu -- the learned independence proposal: a masked autoregressive MLP
// over click patterns, with hand-written BF16 tensor-core kernels.
//
// The paper samples click patterns by MCMC with about 100 probability
// evaluations per sample (Sec. 7.1.1) but does not say how proposals are
// made.  An independence Metropolis-Hastings proposal must be both easy to
// sample and exactly normalised, so this proposal is a MADE network
// (Germain et al., "MADE: Masked Autoencoder for Distribution Estimation",
// ICML 2015): q(x) = prod_j Bernoulli(x_j; sigmoid(l_j(x_<j))).
//
//   x in {0,1}^M -> 3 hidden layers of H (ReLU) -> M logits.
//   Degrees: input j has degree j+1; hidden unit h has degree
//   m(h) = 1 + (h mod (M-1)); a hidden unit sees units of degree <= m(h);
//   output j sees hidden units with m(h) <= j, so l_j depends on x_<j only.
//   log q(x) = sum_j [x_j log s(l_j) + (1 - x_j) log s(-l_j)],  s = sigmoid.
//
// Training minimises the weighted negative log-likelihood
//   L = -(sum_b w_b log q(x_b)) / sum_b w_b
// on patterns x_b with weights w_b (exact probabilities, importance weights,
// or 1 for samples of the exact chain): the forward KL to p up to a constant.
//
// Arithmetic: FP32 master weights and Adam state; BF16 copies of W and W^T
// feed mma.sync.m16n8k16 (BF16 in, FP32 accumulate).  The shapes (K = 16..256,
// batch up to a few thousand) are far too small for tcgen05's 128-row tiles
// to pay, so the legacy warp-level MMA is the right tool here; this network
// is not on the throughput-critical path (the Torontonians are).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <new>
#include <vector>
#include "tor_internal.h"
#include "philox.cuh"

namespace tor {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------- GEMM (NT)
// C[m, n] = sum_k A[m, k] B[n, k] (+ bias[n]) (relu) (* [aux[m,n] > 0]) with
// A: rows x K (lda), B: cols x K (ldb), both BF16, K and the leading
// dimensions multiples of 8 (16-byte rows of 8 BF16); the K tail past a
// multiple of 32 reads as zeros.
struct GemmArgs {
  const bf16 *A; int lda;
  const bf16 *B; int ldb;
  int m, n, K;
  const float *bias;     // optional, n
  int relu;
  const bf16 *aux; int ldaux;  // optional: multiply by (aux > 0), the ReLU derivative
  float *Cf; bf16 *Cb; int ldc;  // one of the two outputs
};

// Block tile 64 x 64 over K steps of 32, staged in shared memory with 16-byte
// loads; 4 warps each own a 32 x 32 tile = 2 x 4 mma.m16n8k16 accumulators.
// Shared rows are padded to 40 BF16 (80 bytes): the fragment reads of a warp
// (8 rows x 4 words) then fall in 32 distinct banks.
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ uint4 ld16(const bf16 *p, int row, int nrows, int ld, int k, int K) {
  if (row >= nrows || k >= K) return make_uint4(0u, 0u, 0u, 0u);
  return *reinterpret_cast<const uint4 *>(p + (size_t)row * ld + k);
}

__global__ void __launch_bounds__(128) k_gemm_nt(GemmArgs g) {
  __shared__ __align__(16) bf16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) bf16 Bs[GBN][GBK + GPAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3;
  const int bm = blockIdx.y * GBM, bn = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float c[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) c[i][j][e] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += GBK) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {  // 256 chunks of 8 BF16 per operand tile
      const int chunk = tid + t * 128, r = chunk >> 2, kc = (chunk & 3) * 8;
      *reinterpret_cast<uint4 *>(&As[r][kc]) = ld16(g.A, bm + r, g.m, g.lda, k0 + kc, g.K);
      *reinterpret_cast<uint4 *>(&Bs[r][kc]) = ld16(g.B, bn + r, g.n, g.ldb, k0 + kc, g.K);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gid;
        a[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + tig * 2]);
        a[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + tig * 2]);
        a[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + tig * 2 + 8]);
        a[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = wn + j * 8 + gid;
        b[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[r][kk + tig * 2]);
        b[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[r][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(c[i][j][0]), "+f"(c[i][j][1]), "+f"(c[i][j][2]), "+f"(c[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = bm + wm + i * 16 + gid + (e >= 2 ? 8 : 0);
        const int cc = bn + wn + j * 8 + tig * 2 + (e & 1);
        if (r >= g.m || cc >= g.n) continue;
        float v = c[i][j][e];
        if (g.bias) v += g.bias[cc];
        if (g.relu) v = fmaxf(v, 0.f);
        if (g.aux && !(__bfloat162float(g.aux[(size_t)r * g.ldaux + cc]) > 0.f)) v = 0.f;
        if (g.Cf) g.Cf[(size_t)r * g.ldc + cc] = v;
        else g.Cb[(size_t)r * g.ldc + cc] = __float2bfloat16(v);
      }
}

static void gemm(const GemmArgs &g, cudaStream_t s) {
  dim3 grid((g.n + GBN - 1) / GBN, (g.m + GBM - 1) / GBM);
  k_gemm_nt<<<grid, 128, 0, s>>>(g);
}

// ------------------------------------------------------ elementwise kernels
__device__ __forceinline__ float log_sigmoid(float z) {  // log(1 / (1 + e^-z)), stable
  return -(fmaxf(-z, 0.f) + log1pf(expf(-fabsf(z))));
}

__global__ void k_unpack(const unsigned long long *__restrict__ pat, int B, int Bp, int M, int Mp, int words,
                         bf16 *__restrict__ X) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Bp * Mp) return;
  const int b = idx / Mp, j = idx % Mp;
  float v = 0.f;
  if (b < B && j < M) v = (float)((pat[(size_t)b * words + (j >> 6)] >> (j & 63)) & 1ull);
  X[idx] = __float2bfloat16(v);
}

__global__ void k_logq(const float *__restrict__ logits, const bf16 *__restrict__ X, int B, int M, int Mp,
                       double *__restrict__ logq) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int j = 0; j < M; ++j) {
    const float l = logits[(size_t)b * Mp + j];
    const bool x = __bfloat162float(X[(size_t)b * Mp + j]) > 0.5f;
    s += (double)log_sigmoid(x ? l : -l);
  }
  logq[b] = s;
}

// dL/dl = w_b (s(l) - x) / sum w  (BF16 for the GEMMs, FP32 for the bias);
// loss = -(sum_b w_b log q_b) / sum w
__global__ void k_loss_grad(const float *__restrict__ logits, const bf16 *__restrict__ X,
                            const float *__restrict__ w, const float *__restrict__ wsum, int B, int Bp, int M, int Mp,
                            bf16 *__restrict__ dl, float *__restrict__ dl32, float *__restrict__ loss) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Bp * Mp) return;
  const int b = idx / Mp, j = idx % Mp;
  float g = 0.f;
  if (b < B && j < M) {
    const float l = logits[idx];
    const bool x = __bfloat162float(X[idx]) > 0.5f;
    const float sg = 1.f / (1.f + expf(-l));
    const float wb = w[b] / *wsum;
    g = wb * (sg - (x ? 1.f : 0.f));
    if (loss) atomicAdd(loss, -wb * log_sigmoid(x ? l : -l));
  }
  dl[idx] = __float2bfloat16(g);
  dl32[idx] = g;
}

__global__ void k_sum(const float *__restrict__ w, int n, float *__restrict__ out) {
  __shared__ float sh[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += w[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// out[c] = sum_r in[r, c] (FP32 or BF16 source), rows < R
template <class TIn>
__global__ void k_colsum(const TIn *__restrict__ in, int R, int Cn, int ld, float *__restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Cn) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += (float)in[(size_t)r * ld + c];
  out[c] = s;
}

__global__ void k_transpose(const bf16 *__restrict__ in, int R, int Cn, bf16 *__restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= R * Cn) return;
  const int r = idx / Cn, c = idx % Cn;
  out[(size_t)c * R + r] = in[idx];
}

__global__ void k_to_bf16(const float *__restrict__ W, int R, int Cn, bf16 *__restrict__ Wb,
                          bf16 *__restrict__ WbT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= R * Cn) return;
  const int r = idx / Cn, c = idx % Cn;
  const bf16 v = __float2bfloat16(W[idx]);
  Wb[idx] = v;
  WbT[(size_t)c * R + r] = v;
}

// masked Adam on FP32 master weights (Kingma & Ba 2015)
__global__ void k_adam(float *__restrict__ W, const float *__restrict__ G, const float *__restrict__ mask,
                       float *__restrict__ m, float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mk = mask ? mask[i] : 1.f;
  const float g = G[i] * mk;
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  W[i] = (W[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps)) * mk;
}

// ancestral sampling of column j: x_j ~ Bernoulli(s(l_j)), log q accumulated
// masked entries are not parameters: their gradient is zero
__global__ void k_mask_mul(float *__restrict__ G, const float *__restrict__ mask, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) G[i] *= mask[i];
}

__global__ void k_sample_col(const float *__restrict__ logits, int B, int Mp, int j, int words,
                             unsigned long long seed, unsigned long long step, bf16 *__restrict__ X,
                             unsigned long long *__restrict__ pat, double *__restrict__ logq) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float l = logits[(size_t)b * Mp + j];
  const double u = philox_uniform(seed, step, (uint32_t)b, (uint32_t)j);
  const double s = 1.0 / (1.0 + exp(-(double)l));
  const bool x = u < s;
  X[(size_t)b * Mp + j] = __float2bfloat16(x ? 1.f : 0.f);
  if (x) pat[(size_t)b * words + (j >> 6)] |= 1ull << (j & 63);
  logq[b] += (double)log_sigmoid(x ? l : -l);
}

__global__ void k_zero_patterns(unsigned long long *__restrict__ pat, bf16 *__restrict__ X, double *__restrict__ logq,
                                int B, int Bp, int Mp, int words) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < Bp * Mp) X[idx] = __float2bfloat16(0.f);
  if (idx < B * words) pat[idx] = 0ull;
  if (idx < B) logq[idx] = 0.0;
}

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace tor

using tor::bf16;

// ------------------------------------------------------------------ object
struct tor_mlp {
  int device = 0, M = 0, Mp = 0, H = 0, words = 0;
  long long t = 0;  // Adam step
  // FP32 master parameters, masks, Adam moments: one flat device block each
  // layer l: W_l [out_l x in_l] (padded), b_l [out_l]
  int out_[4], in_[4];
  size_t woff[4], boff[4], nparam = 0;
  float *P = nullptr, *Mk = nullptr, *Am = nullptr, *Av = nullptr, *G = nullptr;
  bf16 *Wb[4] = {}, *WbT[4] = {};
  // activations (capacity Bcap rows, padded to 16)
  int Bcap = 0;
  bf16 *X = nullptr, *Hh[3] = {}, *dH[3] = {}, *dl = nullptr, *T1 = nullptr, *T2 = nullptr;
  float *logits = nullptr, *dl32 = nullptr, *dh32 = nullptr, *wsum = nullptr, *loss = nullptr, *ones = nullptr;
};

namespace {

thread_local char g_mlp_err[256];
int mfail(int code, const char *msg) {
  return tor::record_error(code, msg);
}
#define MCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      snprintf(g_mlp_err, sizeof(g_mlp_err), "%s: %s", #call, cudaGetErrorString(e_));   \
      return mfail(TOR_ECUDA, g_mlp_err);                                                \
    }                                                                                    \
  } while (0)

int mlp_reserve(tor_mlp *m, int B) {
  if (B <= m->Bcap) return TOR_OK;
  const int Bp = ((B + 15) / 16) * 16;
  void *old[] = {m->X, m->Hh[0], m->Hh[1], m->Hh[2], m->dH[0], m->dH[1], m->dH[2], m->dl, m->T1, m->T2,
                 m->logits, m->dl32, m->dh32, m->ones};
  cudaDeviceSynchronize();
  for (void *p : old)
    if (p) cudaFree(p);
  const size_t H = m->H, Mp = m->Mp, Bq = Bp;
  MCK(cudaMalloc(&m->X, sizeof(bf16) * Bq * Mp));
  for (int l = 0; l < 3; ++l) {
    MCK(cudaMalloc(&m->Hh[l], sizeof(bf16) * Bq * H));
    MCK(cudaMalloc(&m->dH[l], sizeof(bf16) * Bq * H));
  }
  MCK(cudaMalloc(&m->dl, sizeof(bf16) * Bq * Mp));
  const size_t tmax = Bq * (H > Mp ? H : Mp);
  MCK(cudaMalloc(&m->T1, sizeof(bf16) * tmax));
  MCK(cudaMalloc(&m->T2, sizeof(bf16) * tmax));
  MCK(cudaMalloc(&m->logits, sizeof(float) * Bq * Mp));
  MCK(cudaMalloc(&m->dl32, sizeof(float) * Bq * Mp));
  MCK(cudaMalloc(&m->dh32, sizeof(float) * Bq * H));
  MCK(cudaMalloc(&m->ones, sizeof(float) * Bq));
  std::vector<float> ones(Bq, 1.f);
  MCK(cudaMemcpy(m->ones, ones.data(), sizeof(float) * Bq, cudaMemcpyHostToDevice));
  m->Bcap = Bp;
  return TOR_OK;
}

void refresh_bf16(tor_mlp *m, cudaStream_t s) {
  for (int l = 0; l < 4; ++l) {
    const int n = m->out_[l] * m->in_[l];
    tor::k_to_bf16<<<tor::cdiv(n, 256), 256, 0, s>>>(m->P + m->woff[l], m->out_[l], m->in_[l], m->Wb[l], m->WbT[l]);
  }
}

// forward from m->X (Bp rows) to m->logits
void forward(tor_mlp *m, int B, cudaStream_t s) {
  const int Bp = ((B + 15) / 16) * 16;
  const bf16 *in = m->X;
  int ldin = m->Mp;
  for (int l = 0; l < 3; ++l) {
    tor::GemmArgs g{in, ldin, m->Wb[l], m->in_[l], Bp, m->H, m->in_[l], m->P + m->boff[l], 1, nullptr, 0,
                    nullptr, m->Hh[l], m->H};
    tor::gemm(g, s);
    in = m->Hh[l];
    ldin = m->H;
  }
  tor::GemmArgs g{in, ldin, m->Wb[3], m->H, Bp, m->Mp, m->H, m->P + m->boff[3], 0, nullptr, 0, m->logits, nullptr,
                  m->Mp};
  tor::gemm(g, s);
}

// gradients of the weighted NLL into m->G (forward must have run on m->X)
void backward(tor_mlp *m, int B, const float *w, cudaStream_t s) {
  const int Bp = ((B + 15) / 16) * 16;
  const int H = m->H, Mp = m->Mp;
  tor::k_sum<<<1, 256, 0, s>>>(w, B, m->wsum);
  cudaMemsetAsync(m->loss, 0, sizeof(float), s);
  tor::k_loss_grad<<<tor::cdiv(Bp * Mp, 256), 256, 0, s>>>(m->logits, m->X, w, m->wsum, B, Bp, m->M, Mp, m->dl,
                                                           m->dl32, m->loss);
  // layer 4: dW4 = dl^T H3, db4 = colsum(dl), dH3 = (dl W4) * [H3 > 0]
  const bf16 *acts[4] = {m->X, m->Hh[0], m->Hh[1], m->Hh[2]};
  const int widths[4] = {Mp, H, H, H};
  const bf16 *dy = m->dl;
  int wy = Mp;
  for (int l = 3; l >= 0; --l) {
    // dW_l [out x in] = dy^T [out x Bp] . act^T [in x Bp]^T
    tor::k_transpose<<<tor::cdiv(Bp * wy, 256), 256, 0, s>>>(dy, Bp, wy, m->T1);
    tor::k_transpose<<<tor::cdiv(Bp * widths[l], 256), 256, 0, s>>>(acts[l], Bp, widths[l], m->T2);
    tor::GemmArgs gw{m->T1, Bp, m->T2, Bp, m->out_[l], m->in_[l], Bp, nullptr, 0, nullptr, 0,
                     m->G + m->woff[l], nullptr, m->in_[l]};
    tor::gemm(gw, s);
    if (l == 3)
      tor::k_colsum<float><<<tor::cdiv(Mp, 128), 128, 0, s>>>(m->dl32, B, Mp, Mp, m->G + m->boff[3]);
    else
      tor::k_colsum<bf16><<<tor::cdiv(H, 128), 128, 0, s>>>(dy, B, H, H, m->G + m->boff[l]);
    if (l == 0) break;
    // d act_l = dy . W_l  ([Bp x out] . [out x in]) as NT with W_l^T [in x out]
    tor::GemmArgs gx{dy, wy, m->WbT[l], m->out_[l], Bp, m->in_[l], m->out_[l], nullptr, 0, acts[l], widths[l],
                     nullptr, m->dH[l - 1], H};
    tor::gemm(gx, s);
    dy = m->dH[l - 1];
    wy = H;
  }
  tor::k_mask_mul<<<tor::cdiv((int)m->nparam, 256), 256, 0, s>>>(m->G, m->Mk, (int)m->nparam);
}

}  // namespace

int tor::mlp_modes(const tor_mlp *m) { return m ? m->M : -1; }

extern "C" {

int tor_mlp_create(tor_ctx *ctx, int M, int hidden, uint64_t seed, tor_mlp **out) {
  (void)ctx;
  if (!out) return mfail(TOR_EINVAL, "null output pointer");
  *out = nullptr;
  if (M < 2 || M > 128) return mfail(TOR_EINVAL, "M outside [2, 128]");
  if (hidden < 16 || hidden > 1024 || hidden % 16) return mfail(TOR_EINVAL, "hidden must be a multiple of 16 in [16, 1024]");
  tor_mlp *m = new (std::nothrow) tor_mlp();
  if (!m) return mfail(TOR_ENOMEM, "host allocation failed");
  cudaGetDevice(&m->device);
  m->M = M;
  m->Mp = ((M + 15) / 16) * 16;
  m->H = hidden;
  m->words = (M + 63) / 64;
  const int outs[4] = {hidden, hidden, hidden, m->Mp}, ins[4] = {m->Mp, hidden, hidden, hidden};
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    m->out_[l] = outs[l];
    m->in_[l] = ins[l];
    m->woff[l] = off;
    off += (size_t)outs[l] * ins[l];
    m->boff[l] = off;
    off += outs[l];
  }
  m->nparam = off;
  // masks and initial weights on the host (MADE degrees, see the file header)
  std::vector<float> P(off, 0.f), Mk(off, 0.f);
  auto deg_hidden = [&](int h) { return 1 + (h % (M - 1)); };
  uint64_t ctr = 0;
  auto normal = [&]() {  // Box-Muller on Philox draws (step = 2^40 + counter, chain 0)
    const double u1 = tor::philox_uniform(seed, (1ull << 40) + ctr, 0u, 0u);
    const double u2 = tor::philox_uniform(seed, (1ull << 40) + ctr, 0u, 1u);
    ++ctr;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  };
  for (int l = 0; l < 4; ++l) {
    for (int o = 0; o < outs[l]; ++o)
      for (int i = 0; i < ins[l]; ++i) {
        bool allow;
        if (l == 0) allow = (i < M) && deg_hidden(o) >= i + 1;
        else if (l < 3) allow = deg_hidden(o) >= deg_hidden(i);
        else allow = (o < M) && (o + 1) > deg_hidden(i);
        const size_t e = m->woff[l] + (size_t)o * ins[l] + i;
        Mk[e] = allow ? 1.f : 0.f;
        P[e] = allow ? (float)(normal() * sqrt(2.0 / ins[l])) : 0.f;
      }
    for (int o = 0; o < outs[l]; ++o) Mk[m->boff[l] + o] = (l < 3 || o < M) ? 1.f : 0.f;
  }
  int rc = TOR_OK;
  auto alloc = [&](float **p) {
    if (cudaMalloc(p, sizeof(float) * off) != cudaSuccess) rc = TOR_ENOMEM;
  };
  alloc(&m->P); alloc(&m->Mk); alloc(&m->Am); alloc(&m->Av); alloc(&m->G);
  for (int l = 0; l < 4 && rc == TOR_OK; ++l) {
    const size_t n = (size_t)outs[l] * ins[l];
    if (cudaMalloc(&m->Wb[l], sizeof(bf16) * n) != cudaSuccess) rc = TOR_ENOMEM;
    if (cudaMalloc(&m->WbT[l], sizeof(bf16) * n) != cudaSuccess) rc = TOR_ENOMEM;
  }
  if (rc == TOR_OK && (cudaMalloc(&m->wsum, sizeof(float)) != cudaSuccess ||
                       cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess))
    rc = TOR_ENOMEM;
  if (rc != TOR_OK) {
    tor_mlp_destroy(m);
    return mfail(rc, "MLP device allocation failed");
  }
  cudaMemcpy(m->P, P.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
  cudaMemcpy(m->Mk, Mk.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
  cudaMemset(m->Am, 0, sizeof(float) * off);
  cudaMemset(m->Av, 0, sizeof(float) * off);
  refresh_bf16(m, 0);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    tor_mlp_destroy(m);
    return mfail(TOR_ECUDA, "MLP initialisation failed");
  }
  *out = m;
  return TOR_OK;
}

void tor_mlp_destroy(tor_mlp *m) {
  if (!m) return;
  cudaDeviceSynchronize();
  void *ps[] = {m->P, m->Mk, m->Am, m->Av, m->G, m->X, m->Hh[0], m->Hh[1], m->Hh[2], m->dH[0], m->dH[1], m->dH[2],
                m->dl, m->T1, m->T2, m->logits, m->dl32, m->dh32, m->wsum, m->loss, m->ones,
                m->Wb[0], m->Wb[1], m->Wb[2], m->Wb[3], m->WbT[0], m->WbT[1], m->WbT[2], m->WbT[3]};
  for (void *p : ps)
    if (p) cudaFree(p);
  delete m;
}

int tor_mlp_num_params(const tor_mlp *m) {
  if (!m) return -1;
  return 3 * m->H + 2 * m->H * m->H + 2 * m->H * m->M + m->M;
}

// parameters in natural (unpadded) order W1[H x M], b1, W2[H x H], b2, W3, b3, W4[M x H], b4[M];
// which = 0: weights, 1: gradients of the last tor_mlp_grad / train step, 2: the 0/1 masks
int tor_mlp_get_params(const tor_mlp *m, float *host, int which) {
  if (!m || !host) return mfail(TOR_EINVAL, "null pointer");
  const float *src = which == 1 ? m->G : (which == 2 ? m->Mk : m->P);
  std::vector<float> P(m->nparam);
  MCK(cudaMemcpy(P.data(), src, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost));
  size_t o = 0;
  const int realo[4] = {m->H, m->H, m->H, m->M}, reali[4] = {m->M, m->H, m->H, m->H};
  for (int l = 0; l < 4; ++l) {
    for (int r = 0; r < realo[l]; ++r)
      for (int c = 0; c < reali[l]; ++c) host[o++] = P[m->woff[l] + (size_t)r * m->in_[l] + c];
    for (int r = 0; r < realo[l]; ++r) host[o++] = P[m->boff[l] + r];
  }
  return TOR_OK;
}

int tor_mlp_set_params(tor_mlp *m, const float *host) {
  if (!m || !host) return mfail(TOR_EINVAL, "null pointer");
  std::vector<float> P(m->nparam, 0.f), Mk(m->nparam);
  MCK(cudaMemcpy(Mk.data(), m->Mk, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost));
  size_t o = 0;
  const int realo[4] = {m->H, m->H, m->H, m->M}, reali[4] = {m->M, m->H, m->H, m->H};
  for (int l = 0; l < 4; ++l) {
    for (int r = 0; r < realo[l]; ++r)
      for (int c = 0; c < reali[l]; ++c) {
        const size_t e = m->woff[l] + (size_t)r * m->in_[l] + c;
        P[e] = host[o++] * Mk[e];  // masked entries stay zero
      }
    for (int r = 0; r < realo[l]; ++r) P[m->boff[l] + r] = host[o++];
  }
  MCK(cudaMemcpy(m->P, P.data(), sizeof(float) * m->nparam, cudaMemcpyHostToDevice));
  refresh_bf16(m, 0);
  MCK(cudaDeviceSynchronize());
  return TOR_OK;
}

// Start the network at the product of independent marginals: W4 = 0 and
// b4_j = logit(marg_j), so q(x) = prod_j marg_j^x_j (1 - marg_j)^(1 - x_j) (the
// plain proposal) until training adds the correlations the hidden layers see.
int tor_mlp_set_marginals(tor_mlp *m, const double *marg_host) {
  if (!m || !marg_host) return mfail(TOR_EINVAL, "null pointer");
  for (int j = 0; j < m->M; ++j)
    if (!(marg_host[j] > 0.0 && marg_host[j] < 1.0)) return mfail(TOR_EINVAL, "marginals must lie in (0, 1)");
  std::vector<float> P(m->nparam);
  MCK(cudaMemcpy(P.data(), m->P, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost));
  for (size_t e = 0; e < (size_t)m->out_[3] * m->in_[3]; ++e) P[m->woff[3] + e] = 0.f;
  for (int j = 0; j < m->M; ++j) P[m->boff[3] + j] = (float)log(marg_host[j] / (1.0 - marg_host[j]));
  MCK(cudaMemcpy(m->P, P.data(), sizeof(float) * m->nparam, cudaMemcpyHostToDevice));
  refresh_bf16(m, 0);
  MCK(cudaDeviceSynchronize());
  return TOR_OK;
}

int tor_mlp_logq(tor_mlp *m, const uint64_t *patterns, int B, double *logq, cudaStream_t s) {
  if (!m || !patterns || !logq || B < 0) return mfail(TOR_EINVAL, "bad argument");
  if (B == 0) return TOR_OK;
  int rc = mlp_reserve(m, B);
  if (rc) return rc;
  const int Bp = ((B + 15) / 16) * 16;
  tor::k_unpack<<<tor::cdiv(Bp * m->Mp, 256), 256, 0, s>>>((const unsigned long long *)patterns, B, Bp, m->M, m->Mp,
                                                          m->words, m->X);
  forward(m, B, s);
  tor::k_logq<<<tor::cdiv(B, 128), 128, 0, s>>>(m->logits, m->X, B, m->M, m->Mp, logq);
  MCK(cudaGetLastError());
  return TOR_OK;
}

int tor_mlp_logits(tor_mlp *m, const uint64_t *patterns, int B, float *logits_host) {
  if (!m || !patterns || !logits_host || B < 1) return mfail(TOR_EINVAL, "bad argument");
  int rc = mlp_reserve(m, B);
  if (rc) return rc;
  const int Bp = ((B + 15) / 16) * 16;
  tor::k_unpack<<<tor::cdiv(Bp * m->Mp, 256), 256>>>((const unsigned long long *)patterns, B, Bp, m->M, m->Mp,
                                                     m->words, m->X);
  forward(m, B, 0);
  std::vector<float> L((size_t)B * m->Mp);
  MCK(cudaMemcpy(L.data(), m->logits, sizeof(float) * L.size(), cudaMemcpyDeviceToHost));
  for (int b = 0; b < B; ++b)
    for (int j = 0; j < m->M; ++j) logits_host[(size_t)b * m->M + j] = L[(size_t)b * m->Mp + j];
  return TOR_OK;
}

int tor_mlp_grad(tor_mlp *m, const uint64_t *patterns, const float *w, int B, float *loss_host, cudaStream_t s) {
  if (!m || !patterns || !w || B < 1) return mfail(TOR_EINVAL, "bad argument");
  int rc = mlp_reserve(m, B);
  if (rc) return rc;
  const int Bp = ((B + 15) / 16) * 16;
  tor::k_unpack<<<tor::cdiv(Bp * m->Mp, 256), 256, 0, s>>>((const unsigned long long *)patterns, B, Bp, m->M, m->Mp,
                                                          m->words, m->X);
  forward(m, B, s);
  backward(m, B, w, s);
  if (loss_host) {
    MCK(cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
  }
  MCK(cudaGetLastError());
  return TOR_OK;
}

int tor_mlp_train_step(tor_mlp *m, const uint64_t *patterns, const float *w, int B, float lr, float *loss_host,
                       cudaStream_t s) {
  int rc = tor_mlp_grad(m, patterns, w, B, nullptr, s);
  if (rc) return rc;
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
  const int n = (int)m->nparam;
  tor::k_adam<<<tor::cdiv(n, 256), 256, 0, s>>>(m->P, m->G, m->Mk, m->Am, m->Av, n, lr, b1, b2, 1e-8f, c1, c2);
  refresh_bf16(m, s);
  if (loss_host) {
    MCK(cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
  }
  MCK(cudaGetLastError());
  return TOR_OK;
}

int tor_mlp_sample(tor_mlp *m, int B, uint64_t seed, uint64_t step, uint64_t *patterns, double *logq,
                   cudaStream_t s) {
  if (!m || !patterns || !logq || B < 0) return mfail(TOR_EINVAL, "bad argument");
  if (B == 0) return TOR_OK;
  int rc = mlp_reserve(m, B);
  if (rc) return rc;
  const int Bp = ((B + 15) / 16) * 16;
  const int nz = Bp * m->Mp > B * m->words ? Bp * m->Mp : B * m->words;
  tor::k_zero_patterns<<<tor::cdiv(nz, 256), 256, 0, s>>>((unsigned long long *)patterns, m->X, logq, B, Bp, m->Mp,
                                                          m->words);
  for (int j = 0; j < m->M; ++j) {
    forward(m, B, s);  // l_j depends on x_<j only, which are already drawn
    tor::k_sample_col<<<tor::cdiv(B, 128), 128, 0, s>>>(m->logits, B, m->Mp, j, m->words, seed, step, m->X,
                                                        (unsigned long long *)patterns, logq);
  }
  MCK(cudaGetLastError());
  return TOR_OK;
}

}  // extern "C"
