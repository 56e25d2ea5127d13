// mlp.cu -- multilayer perceptron for the structural-step surrogate: BF16
// tensor-core GEMMs with FP32 accumulation (mma.sync m16n8k16), exact-erf
// GELU, mean-squared-error loss, backward pass and Adam, all on the GPU.
//
// Parameters live in FP32 (master copy) with BF16 copies of every weight
// matrix in both orientations (W[n_out][n_in] for the forward product and
// W^T for the input gradient).  Activations are kept in FP32 (pre-activation
// Z, for GELU') and BF16 (post-activation A, the next GEMM's operand).
//
// Not part of the paper: the surrogate pattern replaces the structural
// Newton solve of section "Structural modeling" with a learned initial guess
// that the FEM residual accepts or rejects.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "../../include/kbc_lbm.h"
#include "lbm_internal.h"

namespace kbc {

constexpr int kMlpMaxLayers = 8;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// D[16x8] += A[16x16] B[16x8], BF16 inputs, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

enum { EPI_NONE = 0, EPI_GELU = 1, EPI_GELU_GRAD = 2 };

// C[M x N] = sum_k A(m, k) B(k, n) with A(m,k) = A[m*sam + k*sak] and
// B(k,n) = B[k*sbk + n*sbn] (BF16), FP32 accumulation; one warp per 16x8
// output tile.  Epilogue: + bias[n]; EPI_GELU stores Z (pre) and GELU(Z);
// EPI_GELU_GRAD multiplies by GELU'(zpre[m*ldz+n]).  Outputs: FP32 c (ldc)
// and/or BF16 cb (ldcb) and its transpose cbt (ldcbt) when non-null.
template <int EPI>
__global__ void __launch_bounds__(128)
    k_gemm(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, long long sam, long long sak,
           const __nv_bfloat16 *__restrict__ B, long long sbk, long long sbn,
           const float *__restrict__ bias, const float *__restrict__ zpre, int ldz,
           float *__restrict__ c, int ldc, float *__restrict__ zout, int ldzo,
           __nv_bfloat16 *__restrict__ cb, int ldcb, __nv_bfloat16 *__restrict__ cbt, int ldcbt) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = (N + 7) / 8;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * 16 >= M) return;
  const int gid = lane >> 2, tig = lane & 3;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  auto ldA = [&](int m, int k) { return (m < M && k < K) ? A[m * sam + k * sak] : zero; };
  auto ldB = [&](int k, int n) { return (k < K && n < N) ? B[k * sbk + n * sbn] : zero; };
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const int m0 = tm * 16, n0 = tn * 8;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4], b[2];
    const int r0 = m0 + gid, r1 = m0 + gid + 8, kc = k0 + tig * 2;
    a[0] = pack2(ldA(r0, kc), ldA(r0, kc + 1));
    a[1] = pack2(ldA(r1, kc), ldA(r1, kc + 1));
    a[2] = pack2(ldA(r0, kc + 8), ldA(r0, kc + 9));
    a[3] = pack2(ldA(r1, kc + 8), ldA(r1, kc + 9));
    const int nc = n0 + gid;
    b[0] = pack2(ldB(kc, nc), ldB(kc + 1, nc));
    b[1] = pack2(ldB(kc + 8, nc), ldB(kc + 9, nc));
    mma_bf16(acc, a, b);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = m0 + gid + (q >= 2 ? 8 : 0);
    const int n = n0 + tig * 2 + (q & 1);
    if (m >= M || n >= N) continue;
    float v = acc[q] + (bias ? bias[n] : 0.f);
    if (EPI == EPI_GELU) {
      if (zout) zout[(long long)m * ldzo + n] = v;
      v = gelu(v);
    } else if (EPI == EPI_GELU_GRAD) {
      v *= gelu_grad(zpre[(long long)m * ldz + n]);
    }
    if (c) c[(long long)m * ldc + n] = v;
    if (cb) cb[(long long)m * ldcb + n] = __float2bfloat16(v);
    if (cbt) cbt[(long long)n * ldcbt + m] = __float2bfloat16(v);
  }
}

// Small-batch inference in one launch: all layers of the network for
// B <= 16 rows (one 16-row MMA tile) in one CTA; the BF16 activations stay in
// shared memory (two buffers of 16 x ld), the weights come from L2.  Every
// output element is computed as k_gemm computes it (same fragments, same
// k order, same epilogue), so results equal the layer-by-layer forward pass.
struct MlpInferDesc {
  int nl, B;
  int dims[kMlpMaxLayers + 1];
  const __nv_bfloat16 *w[kMlpMaxLayers];  // [dims[l+1]][dims[l]]
  const float *b[kMlpMaxLayers];
};
constexpr int kInferThreads = 512;

__global__ void __launch_bounds__(kInferThreads)
    k_mlp_infer(MlpInferDesc d, int ld, const float *__restrict__ xin, float *__restrict__ yhat) {
  extern __shared__ __align__(16) __nv_bfloat16 act[];
  __nv_bfloat16 *cur = act, *nxt = act + 16 * ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  const int n0 = d.dims[0];
  for (int t = tid; t < 16 * ld; t += blockDim.x) {
    const int m = t / ld, k = t % ld;
    cur[t] = (m < d.B && k < n0) ? __float2bfloat16(xin[m * n0 + k]) : zero;
  }
  __syncthreads();
  for (int l = 0; l < d.nl; ++l) {
    const int K = d.dims[l], N = d.dims[l + 1];
    const bool last = l == d.nl - 1;
    const __nv_bfloat16 *__restrict__ W = d.w[l];
    auto ldA = [&](int m, int k) { return (m < d.B && k < K) ? cur[m * ld + k] : zero; };
    auto ldB = [&](int k, int n) { return (k < K && n < N) ? W[(long long)n * K + k] : zero; };
    for (int tn = warp; tn < (N + 7) / 8; tn += nw) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int n0t = tn * 8, nc = n0t + gid;
#pragma unroll 4
      for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4], b[2];
        const int kc = k0 + tig * 2;
        a[0] = pack2(ldA(gid, kc), ldA(gid, kc + 1));
        a[1] = pack2(ldA(gid + 8, kc), ldA(gid + 8, kc + 1));
        a[2] = pack2(ldA(gid, kc + 8), ldA(gid, kc + 9));
        a[3] = pack2(ldA(gid + 8, kc + 8), ldA(gid + 8, kc + 9));
        b[0] = pack2(ldB(kc, nc), ldB(kc + 1, nc));
        b[1] = pack2(ldB(kc + 8, nc), ldB(kc + 9, nc));
        mma_bf16(acc, a, b);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = gid + (q >= 2 ? 8 : 0);
        const int n = n0t + tig * 2 + (q & 1);
        if (m >= d.B || n >= N) continue;
        const float v = acc[q] + d.b[l][n];
        if (last) yhat[(long long)m * N + n] = v;
        else nxt[m * ld + n] = __float2bfloat16(gelu(v));
      }
    }
    __syncthreads();
    __nv_bfloat16 *t = cur;
    cur = nxt;
    nxt = t;
  }
}

__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y,
                          __nv_bfloat16 *__restrict__ yt, int rows, int cols) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * cols) return;
  const int r = (int)(t / cols), c = (int)(t % cols);
  const __nv_bfloat16 v = __float2bfloat16(x[t]);
  if (y) y[t] = v;
  if (yt) yt[(long long)c * rows + r] = v;
}

// dY = 2 (Yhat - Y) / (B * n) and the loss sum((Yhat - Y)^2) / (B * n).
__global__ void k_mse(const float *__restrict__ yhat, const float *__restrict__ y, int B, int n,
                      __nv_bfloat16 *__restrict__ dy, __nv_bfloat16 *__restrict__ dyt,
                      float *__restrict__ loss) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (t < B * n) {
    const float d = yhat[t] - y[t];
    const float g = 2.f * d / (float)(B * n);
    dy[t] = __float2bfloat16(g);
    dyt[(long long)(t % n) * B + t / n] = __float2bfloat16(g);
    l = d * d / (float)(B * n);
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// db[n] = sum_m dZ[m][n] (FP32, from the BF16 copy of dZ).
__global__ void k_bias_grad(const __nv_bfloat16 *__restrict__ dz, int B, int n,
                            float *__restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f;
  for (int m = 0; m < B; ++m) s += __bfloat162float(dz[(long long)m * n + j]);
  db[j] = s;
}

// Adam on the FP32 master parameters; refreshes the BF16 copies (W, W^T).
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

}  // namespace kbc

using namespace kbc;

struct mlp_ctx {
  int nl = 0;                 // number of weight layers
  int dims[kMlpMaxLayers + 1];
  int max_batch = 0;
  double lr, b1, b2, eps;
  long long t = 0;            // Adam step count
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char *ws = nullptr;
  bool own_ws = false;
  long long nparam = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // flat: per layer W then b
  long long woff[kMlpMaxLayers], boff[kMlpMaxLayers];
  __nv_bfloat16 *wb[kMlpMaxLayers], *wbt[kMlpMaxLayers];
  float *z[kMlpMaxLayers];              // pre-activations [B][dims[l+1]]
  __nv_bfloat16 *a[kMlpMaxLayers + 1];  // activations (a[0] = input) [B][dims[l]]
  __nv_bfloat16 *at[kMlpMaxLayers + 1]; // transposed activations [dims[l]][B]
  float *yhat = nullptr, *ytarget = nullptr, *xin = nullptr, *loss = nullptr;
  __nv_bfloat16 *dz = nullptr, *dzt = nullptr, *da = nullptr;
  char msg[256] = {0};
};

namespace {

size_t al(size_t b) { return (b + 255) / 256 * 256; }

size_t mlp_layout(const mlp_config *c, mlp_ctx *x) {
  size_t off = 0;
  long long np = 0;
  int maxd = 0;
  for (int l = 0; l <= c->n_layers; ++l) maxd = c->dims[l] > maxd ? c->dims[l] : maxd;
  for (int l = 0; l < c->n_layers; ++l) {
    if (x) x->woff[l] = np;
    np += (long long)c->dims[l] * c->dims[l + 1];
    if (x) x->boff[l] = np;
    np += c->dims[l + 1];
  }
  const size_t B = (size_t)c->max_batch;
  size_t o_p = off; off += al(sizeof(float) * np);
  size_t o_g = off; off += al(sizeof(float) * np);
  size_t o_m = off; off += al(sizeof(float) * np);
  size_t o_v = off; off += al(sizeof(float) * np);
  size_t o_wb[kMlpMaxLayers], o_wbt[kMlpMaxLayers], o_z[kMlpMaxLayers];
  size_t o_a[kMlpMaxLayers + 1], o_at[kMlpMaxLayers + 1];
  for (int l = 0; l < c->n_layers; ++l) {
    const size_t w = (size_t)c->dims[l] * c->dims[l + 1];
    o_wb[l] = off; off += al(2 * w);
    o_wbt[l] = off; off += al(2 * w);
    o_z[l] = off; off += al(sizeof(float) * B * c->dims[l + 1]);
  }
  for (int l = 0; l <= c->n_layers; ++l) {
    o_a[l] = off; off += al(2 * B * c->dims[l]);
    o_at[l] = off; off += al(2 * B * c->dims[l]);
  }
  const int nout = c->dims[c->n_layers];
  size_t o_yhat = off; off += al(sizeof(float) * B * nout);
  size_t o_y = off; off += al(sizeof(float) * B * nout);
  size_t o_x = off; off += al(sizeof(float) * B * c->dims[0]);
  size_t o_loss = off; off += 256;
  size_t o_dz = off; off += al(2 * B * maxd);
  size_t o_dzt = off; off += al(2 * B * maxd);
  size_t o_da = off; off += al(2 * B * maxd);
  if (x) {
    char *w = x->ws;
    x->nparam = np;
    x->p = (float *)(w + o_p); x->g = (float *)(w + o_g);
    x->m = (float *)(w + o_m); x->v = (float *)(w + o_v);
    for (int l = 0; l < c->n_layers; ++l) {
      x->wb[l] = (__nv_bfloat16 *)(w + o_wb[l]);
      x->wbt[l] = (__nv_bfloat16 *)(w + o_wbt[l]);
      x->z[l] = (float *)(w + o_z[l]);
    }
    for (int l = 0; l <= c->n_layers; ++l) {
      x->a[l] = (__nv_bfloat16 *)(w + o_a[l]);
      x->at[l] = (__nv_bfloat16 *)(w + o_at[l]);
    }
    x->yhat = (float *)(w + o_yhat); x->ytarget = (float *)(w + o_y);
    x->xin = (float *)(w + o_x); x->loss = (float *)(w + o_loss);
    x->dz = (__nv_bfloat16 *)(w + o_dz); x->dzt = (__nv_bfloat16 *)(w + o_dzt);
    x->da = (__nv_bfloat16 *)(w + o_da);
  }
  return off;
}

const char *mlp_validate(const mlp_config *c) {
  if (!c) return "config is NULL";
  if (c->n_layers < 1 || c->n_layers > kMlpMaxLayers) return "n_layers must be 1..8";
  for (int l = 0; l <= c->n_layers; ++l)
    if (c->dims[l] < 1 || c->dims[l] > 4096) return "layer widths must be 1..4096";
  if (c->max_batch < 1 || c->max_batch > 65536) return "max_batch must be 1..65536";
  if (!(c->lr > 0) || !(c->beta1 >= 0 && c->beta1 < 1) || !(c->beta2 >= 0 && c->beta2 < 1) ||
      !(c->eps > 0))
    return "bad Adam parameters";
  return nullptr;
}

thread_local char g_mlp_msg[256];

}  // namespace

#define MCK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      snprintf(x->msg, sizeof(x->msg), "%s: %s", #call, cudaGetErrorString(e_));    \
      return LBM_ECUDA;                                                             \
    }                                                                               \
  } while (0)

static unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

template <int EPI>
static cudaError_t gemm(cudaStream_t s, int M, int N, int K, const __nv_bfloat16 *A, long long sam,
                        long long sak, const __nv_bfloat16 *B, long long sbk, long long sbn,
                        const float *bias, const float *zpre, int ldz, float *c, int ldc,
                        float *zout, int ldzo, __nv_bfloat16 *cb, int ldcb, __nv_bfloat16 *cbt,
                        int ldcbt) {
  const long long warps = (long long)((M + 15) / 16) * ((N + 7) / 8);
  k_gemm<EPI><<<blocks_for(warps * 32, 128), 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias,
                                                         zpre, ldz, c, ldc, zout, ldzo, cb, ldcb,
                                                         cbt, ldcbt);
  return cudaGetLastError();
}

// BF16 copies of the weights from the FP32 master parameters.
static lbm_status refresh_bf16(mlp_ctx *x) {
  for (int l = 0; l < x->nl; ++l) {
    const int ni = x->dims[l], no = x->dims[l + 1];
    k_to_bf16<<<blocks_for((long long)ni * no, 256), 256, 0, x->stream>>>(x->p + x->woff[l], x->wb[l],
                                                                          x->wbt[l], no, ni);
    MCK(cudaGetLastError());
  }
  return LBM_OK;
}

// Forward pass for B rows already in x->xin (FP32, normalised inputs).
static lbm_status forward(mlp_ctx *x, int B) {
  const int n0 = x->dims[0];
  k_to_bf16<<<blocks_for((long long)B * n0, 256), 256, 0, x->stream>>>(x->xin, x->a[0], x->at[0], B,
                                                                       n0);
  MCK(cudaGetLastError());
  for (int l = 0; l < x->nl; ++l) {
    const int ni = x->dims[l], no = x->dims[l + 1];
    const bool last = l == x->nl - 1;
    // Z = A W^T + b: A(m,k) = a[m*ni + k], B(k,n) = W[n][k] = wb[n*ni + k]
    if (last)
      MCK(gemm<EPI_NONE>(x->stream, B, no, ni, x->a[l], ni, 1, x->wb[l], 1, ni, x->p + x->boff[l],
                         nullptr, 0, x->yhat, no, nullptr, 0, nullptr, 0, nullptr, 0));
    else
      MCK(gemm<EPI_GELU>(x->stream, B, no, ni, x->a[l], ni, 1, x->wb[l], 1, ni, x->p + x->boff[l],
                         nullptr, 0, nullptr, 0, x->z[l], no, x->a[l + 1], no, x->at[l + 1], B));
  }
  return LBM_OK;
}

// Single-launch inference (k_mlp_infer) for B <= 16 when two 16-row BF16
// activation buffers of the widest layer fit in shared memory; a context that
// needs more than the default 48 KB raises the kernel's limit to the 200 KB
// bound at creation.
static size_t infer_smem(const mlp_ctx *x, int *ld) {
  int maxw = 0;
  for (int l = 0; l <= x->nl; ++l) maxw = x->dims[l] > maxw ? x->dims[l] : maxw;
  *ld = (maxw + 15) / 16 * 16;
  return sizeof(__nv_bfloat16) * 2 * 16 * (size_t)*ld;
}
constexpr size_t kInferMaxSmem = 200u * 1024u;

static bool fused_ok(const mlp_ctx *x, int B) {
  int ld;
  return B >= 1 && B <= 16 && infer_smem(x, &ld) <= kInferMaxSmem;
}

static lbm_status forward_fused(mlp_ctx *x, int B, cudaStream_t s) {
  int ld;
  const size_t smem = infer_smem(x, &ld);
  MlpInferDesc d{};
  d.nl = x->nl;
  d.B = B;
  for (int l = 0; l <= x->nl; ++l) d.dims[l] = x->dims[l];
  for (int l = 0; l < x->nl; ++l) {
    d.w[l] = x->wb[l];
    d.b[l] = x->p + x->boff[l];
  }
  k_mlp_infer<<<1, kInferThreads, smem, s>>>(d, ld, x->xin, x->yhat);
  MCK(cudaGetLastError());
  return LBM_OK;
}

// Backward pass (after forward) from dY = dLoss/dYhat in dz / dzt; gradients
// into x->g.
static lbm_status backward(mlp_ctx *x, int B) {
  for (int l = x->nl - 1; l >= 0; --l) {
    const int ni = x->dims[l], no = x->dims[l + 1];
    // dW[no][ni] = dZ^T A: A(m=n_out row, k=batch) = dzt[o*B + b], B(k=b, n=i) = a[b*ni + i]
    MCK(gemm<EPI_NONE>(x->stream, no, ni, B, x->dzt, B, 1, x->a[l], ni, 1, nullptr, nullptr, 0,
                       x->g + x->woff[l], ni, nullptr, 0, nullptr, 0, nullptr, 0));
    k_bias_grad<<<blocks_for(no, 128), 128, 0, x->stream>>>(x->dz, B, no, x->g + x->boff[l]);
    MCK(cudaGetLastError());
    if (l == 0) break;
    // dA[B][ni] = dZ W, then dZ_prev = dA * GELU'(Z_prev): A(m=b,k=o) = dz[b*no + o],
    // B(k=o, n=i) = W[o][i] = wbt[i*no + o]
    MCK(gemm<EPI_GELU_GRAD>(x->stream, B, ni, no, x->dz, no, 1, x->wbt[l], 1, no, nullptr,
                            x->z[l - 1], ni, nullptr, 0, nullptr, 0, x->da, ni, x->dzt, B));
    MCK(cudaMemcpyAsync(x->dz, x->da, sizeof(__nv_bfloat16) * (size_t)B * ni,
                        cudaMemcpyDeviceToDevice, x->stream));
  }
  return LBM_OK;
}

extern "C" {

lbm_status mlp_workspace_size(const mlp_config *cfg, size_t *bytes) {
  if (!bytes || mlp_validate(cfg)) return LBM_EINVAL;
  *bytes = mlp_layout(cfg, nullptr);
  return LBM_OK;
}

lbm_status mlp_create(const mlp_config *cfg, void *workspace, size_t bytes, mlp_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (const char *why = mlp_validate(cfg)) {
    snprintf(g_mlp_msg, sizeof(g_mlp_msg), "mlp_create: %s", why);
    return LBM_EINVAL;
  }
  mlp_ctx *x = new (std::nothrow) mlp_ctx();
  if (!x) return LBM_ENOMEM;
  x->nl = cfg->n_layers;
  for (int l = 0; l <= x->nl; ++l) x->dims[l] = cfg->dims[l];
  x->max_batch = cfg->max_batch;
  x->lr = cfg->lr; x->b1 = cfg->beta1; x->b2 = cfg->beta2; x->eps = cfg->eps;
  const size_t need = mlp_layout(cfg, nullptr);
  if (workspace) {
    if (bytes < need || ((uintptr_t)workspace % 256)) {
      delete x;
      snprintf(g_mlp_msg, sizeof(g_mlp_msg), "mlp_create: workspace needs %zu bytes", need);
      return LBM_ENOMEM;
    }
    x->ws = (char *)workspace;
  } else {
    if (cudaMalloc((void **)&x->ws, need) != cudaSuccess) {
      delete x;
      return LBM_ENOMEM;
    }
    x->own_ws = true;
  }
  if (cfg->stream) {
    x->stream = (cudaStream_t)cfg->stream;
  } else {
    cudaStreamCreateWithFlags(&x->stream, cudaStreamNonBlocking);
    x->own_stream = true;
  }
  mlp_layout(cfg, x);
  cudaMemsetAsync(x->ws, 0, need, x->stream);
  int ld;
  const size_t smem = infer_smem(x, &ld);
  if (smem > 48u * 1024u && smem <= kInferMaxSmem &&
      cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kInferMaxSmem) !=
          cudaSuccess) {
    cudaGetLastError();
    mlp_destroy(x);
    return LBM_ECUDA;
  }
  *out = x;
  return LBM_OK;
}

lbm_status mlp_set_params(mlp_ctx *x, const float *params) {
  if (!x || !params) return LBM_EINVAL;
  MCK(cudaMemcpyAsync(x->p, params, sizeof(float) * x->nparam, cudaMemcpyDefault, x->stream));
  MCK(cudaMemsetAsync(x->m, 0, sizeof(float) * x->nparam, x->stream));
  MCK(cudaMemsetAsync(x->v, 0, sizeof(float) * x->nparam, x->stream));
  x->t = 0;
  lbm_status st = refresh_bf16(x);
  if (st != LBM_OK) return st;
  MCK(cudaStreamSynchronize(x->stream));
  return LBM_OK;
}

lbm_status mlp_get_params(mlp_ctx *x, float *params) {
  if (!x || !params) return LBM_EINVAL;
  MCK(cudaMemcpyAsync(params, x->p, sizeof(float) * x->nparam, cudaMemcpyDefault, x->stream));
  MCK(cudaStreamSynchronize(x->stream));
  return LBM_OK;
}

long long mlp_param_count(const mlp_ctx *x) { return x ? x->nparam : -1; }

lbm_status mlp_forward(mlp_ctx *x, const float *X, int B, float *Y) {
  if (!x || !X || !Y || B < 1 || B > x->max_batch) return LBM_EINVAL;
  MCK(cudaMemcpyAsync(x->xin, X, sizeof(float) * (size_t)B * x->dims[0], cudaMemcpyDefault,
                      x->stream));
  lbm_status st = fused_ok(x, B) ? forward_fused(x, B, x->stream) : forward(x, B);
  if (st != LBM_OK) return st;
  MCK(cudaMemcpyAsync(Y, x->yhat, sizeof(float) * (size_t)B * x->dims[x->nl], cudaMemcpyDefault,
                      x->stream));
  MCK(cudaStreamSynchronize(x->stream));
  return LBM_OK;
}

// Loss and gradients of mean((Yhat - Y)^2) for one batch, without updating.
lbm_status mlp_gradients(mlp_ctx *x, const float *X, const float *Y, int B, float *grads,
                         float *loss) {
  if (!x || !X || !Y || B < 1 || B > x->max_batch) return LBM_EINVAL;
  const int nout = x->dims[x->nl];
  MCK(cudaMemcpyAsync(x->xin, X, sizeof(float) * (size_t)B * x->dims[0], cudaMemcpyDefault,
                      x->stream));
  MCK(cudaMemcpyAsync(x->ytarget, Y, sizeof(float) * (size_t)B * nout, cudaMemcpyDefault,
                      x->stream));
  MCK(cudaMemsetAsync(x->loss, 0, sizeof(float), x->stream));
  lbm_status st = forward(x, B);
  if (st != LBM_OK) return st;
  k_mse<<<blocks_for((long long)B * nout, 256), 256, 0, x->stream>>>(x->yhat, x->ytarget, B, nout,
                                                                    x->dz, x->dzt, x->loss);
  MCK(cudaGetLastError());
  if ((st = backward(x, B)) != LBM_OK) return st;
  if (grads)
    MCK(cudaMemcpyAsync(grads, x->g, sizeof(float) * x->nparam, cudaMemcpyDefault, x->stream));
  if (loss) MCK(cudaMemcpyAsync(loss, x->loss, sizeof(float), cudaMemcpyDefault, x->stream));
  MCK(cudaStreamSynchronize(x->stream));
  return LBM_OK;
}

// One Adam step on a batch (X, Y already normalised).  Asynchronous unless
// loss is requested.
lbm_status mlp_train_step(mlp_ctx *x, const float *X, const float *Y, int B, float *loss) {
  if (!x || !X || !Y || B < 1 || B > x->max_batch) return LBM_EINVAL;
  const int nout = x->dims[x->nl];
  MCK(cudaMemcpyAsync(x->xin, X, sizeof(float) * (size_t)B * x->dims[0], cudaMemcpyDefault,
                      x->stream));
  MCK(cudaMemcpyAsync(x->ytarget, Y, sizeof(float) * (size_t)B * nout, cudaMemcpyDefault,
                      x->stream));
  MCK(cudaMemsetAsync(x->loss, 0, sizeof(float), x->stream));
  lbm_status st = forward(x, B);
  if (st != LBM_OK) return st;
  k_mse<<<blocks_for((long long)B * nout, 256), 256, 0, x->stream>>>(x->yhat, x->ytarget, B, nout,
                                                                    x->dz, x->dzt, x->loss);
  MCK(cudaGetLastError());
  if ((st = backward(x, B)) != LBM_OK) return st;
  x->t += 1;
  const float c1 = 1.f - (float)pow(x->b1, (double)x->t), c2 = 1.f - (float)pow(x->b2, (double)x->t);
  k_adam<<<blocks_for(x->nparam, 256), 256, 0, x->stream>>>(x->p, x->g, x->m, x->v, x->nparam,
                                                           (float)x->lr, (float)x->b1,
                                                           (float)x->b2, (float)x->eps, c1, c2);
  MCK(cudaGetLastError());
  if ((st = refresh_bf16(x)) != LBM_OK) return st;
  if (loss) {
    MCK(cudaMemcpyAsync(loss, x->loss, sizeof(float), cudaMemcpyDefault, x->stream));
    MCK(cudaStreamSynchronize(x->stream));
  }
  return LBM_OK;
}

lbm_status mlp_set_learning_rate(mlp_ctx *x, double lr) {
  if (!x || !(lr > 0.0)) return LBM_EINVAL;
  x->lr = lr;
  return LBM_OK;
}

const char *mlp_last_error(const mlp_ctx *x) { return x ? x->msg : g_mlp_msg; }

void mlp_destroy(mlp_ctx *x) {
  if (!x) return;
  if (x->stream) cudaStreamSynchronize(x->stream);
  if (x->own_stream) cudaStreamDestroy(x->stream);
  if (x->own_ws) cudaFree(x->ws);
  delete x;
}

}  // extern "C"

namespace kbc {

// Device-side forward for the coupled surrogate: input already in xin.
lbm_status mlp_forward_device(mlp_ctx *x, int B, cudaStream_t s, float **yhat, float **xin) {
  *yhat = x->yhat;
  *xin = x->xin;
  if (fused_ok(x, B)) return forward_fused(x, B, s);
  cudaStream_t old = x->stream;
  x->stream = s;
  lbm_status st = forward(x, B);
  x->stream = old;
  *yhat = x->yhat;
  *xin = x->xin;
  return st;
}

float *mlp_input_buffer(mlp_ctx *x) { return x->xin; }
int mlp_dim(const mlp_ctx *x, int l) { return x->dims[l]; }
int mlp_layers(const mlp_ctx *x) { return x->nl; }

}  // namespace kbc
