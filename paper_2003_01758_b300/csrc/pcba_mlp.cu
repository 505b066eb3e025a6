// Set-encoder network of the learned warm start (not part of the paper):
// training and inference kernels.  See include/pcba.h (pcba_mlp_*).
//
//   h1_p = relu(x_p W1 + b1), h2_p = relu(h1_p W2 + b2), h3_p = relu(h2_p W3 + b3)
//   z = max_p h3_p,  h4 = relu([z, u] W4 + b4),  h5 = relu(h4 W5 + b5),
//   y = tanh(h5 W6 + b6),  loss = (1/B) sum_b ||y_b - t_b||^2
//
// The dense layers run as GEMMs on the tensor cores (mma.sync m16n8k16, BF16
// operands rounded from the FP32 master copies, FP32 accumulation); a plain
// FP32 GEMM replaces them in the FP32 debug precision.  Weights are row-major
// [in][out]; the parameter vector is W1, b1, ..., W6, b6.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "pcba_warmstart.h"

int pcba_internal_fail(int code, const std::string& msg);

#define MLP_CK(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return pcba_internal_fail(PCBA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

// ---------------------------------------------------------------------------
// GEMM: C[M x N] (+)= A[M x K] B[K x N]; A(m,k) = A[m*lda+k] or, transposed,
// A[k*lda+m]; B(k,n) = B[k*ldb+n] or, transposed, B[n*ldb+k].
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 32, GLDS = GBK + 8;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Split-K: block z covers k in [z * kchunk, (z + 1) * kchunk) and, when the
// grid has more than one z, adds its partial sums into C atomically (C must
// then hold the accumulation target, beta = 1).
__global__ void __launch_bounds__(128) gemm_bf16(int M, int N, int K, const float* __restrict__ A,
                                                 int lda, int ta, const float* __restrict__ B,
                                                 int ldb, int tb, float* C, int ldc, int beta,
                                                 int kchunk) {
  __shared__ __align__(16) __nv_bfloat16 sA[GBM][GLDS];
  __shared__ __align__(16) __nv_bfloat16 sB[GBN][GLDS];
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
    for (int idx = tid; idx < GBM * GBK; idx += 128) {
      int m, k;
      if (ta) { k = idx / GBM; m = idx % GBM; } else { m = idx / GBK; k = idx % GBK; }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.0f;
      if (gm < M && gk < kend) v = ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      sA[m][k] = __float2bfloat16_rn(v);
    }
    for (int idx = tid; idx < GBN * GBK; idx += 128) {
      int n, k;
      if (tb) { n = idx / GBK; k = idx % GBK; } else { k = idx / GBN; n = idx % GBN; }
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.0f;
      if (gn < N && gk < kend) v = tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      sB[n][k] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int row = wm * 32 + mi * 16 + gid;
        af[mi][0] = *(const uint32_t*)&sA[row][kk + tig * 2];
        af[mi][1] = *(const uint32_t*)&sA[row + 8][kk + tig * 2];
        af[mi][2] = *(const uint32_t*)&sA[row][kk + 8 + tig * 2];
        af[mi][3] = *(const uint32_t*)&sA[row + 8][kk + 8 + tig * 2];
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int col = wn * 32 + ni * 8 + gid;
        bf[ni][0] = *(const uint32_t*)&sB[col][kk + tig * 2];
        bf[ni][1] = *(const uint32_t*)&sB[col][kk + 8 + tig * 2];
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bf[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = m0 + wm * 32 + mi * 16 + gid + (q >= 2 ? 8 : 0);
        const int c = n0 + wn * 32 + ni * 8 + tig * 2 + (q & 1);
        if (r < M && c < N) {
          float* dst = C + (size_t)r * ldc + c;
          if (gridDim.z > 1) atomicAdd(dst, acc[mi][ni][q]);
          else *dst = acc[mi][ni][q] + (beta ? *dst : 0.0f);
        }
      }
}

__global__ void gemm_f32(int M, int N, int K, const float* __restrict__ A, int lda, int ta,
                         const float* __restrict__ B, int ldb, int tb, float* C, int ldc,
                         int beta) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y * blockDim.y + threadIdx.y;
  if (m >= M || n >= N) return;
  float s = 0.0f;
  for (int k = 0; k < K; ++k) {
    const float a = ta ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
    const float b = tb ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
    s = fmaf(a, b, s);
  }
  float* dst = C + (size_t)m * ldc + n;
  *dst = s + (beta ? *dst : 0.0f);
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rb(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

// h1 = relu(x W1 + b1) for a small input dimension dp
__global__ void first_layer(const float* x, int P, int dp, const float* W1, const float* b1,
                            float* h1, int H, int bf16) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)P * H) return;
  const int p = (int)(t / H), j = (int)(t % H);
  float s = b1[j];
  for (int i = 0; i < dp; ++i) s = fmaf(rb(x[(size_t)p * dp + i], bf16), rb(W1[i * H + j], bf16), s);
  h1[t] = fmaxf(s, 0.0f);
}

__global__ void bias_relu(float* C, long long R, int N, const float* bias) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * N) return;
  C[t] = fmaxf(C[t] + bias[t % N], 0.0f);
}

// z[b][j] = max over the set of h3[p][j]; arg = the maximising point (the
// first one on ties).  Offsets are clamped to [0, P]; an empty set gives
// z = 0 and arg = -1 (no gradient).
__global__ void set_maxpool(const float* h3, const int* off, int B, int P, int H, float* z,
                            int* arg) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * H) return;
  const int b = t / H, j = t % H;
  const int p0 = max(off[b], 0), p1 = min(off[b + 1], P);
  float best = -INFINITY;
  int ib = -1;
  for (int p = p0; p < p1; ++p) {
    const float v = h3[(size_t)p * H + j];
    if (v > best) { best = v; ib = p; }
  }
  z[t] = ib < 0 ? 0.0f : best;
  arg[t] = ib;
}

__global__ void concat_rows(const float* z, int H, const float* g, int dg, float* u, int B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int W = H + dg;
  if (t >= B * W) return;
  const int b = t / W, j = t % W;
  u[t] = j < H ? z[b * H + j] : g[b * dg + (j - H)];
}

// y = tanh(s6), s6 = h5 W6 + b6 with 2 outputs (s6 kept for the backward pass)
__global__ void out_layer(const float* h5, int B, int H, const float* W6, const float* b6, float* y,
                          float* s6, int bf16) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * 2) return;
  const int b = t / 2, k = t % 2;
  float s = b6[k];
  for (int j = 0; j < H; ++j) s = fmaf(rb(h5[b * H + j], bf16), rb(W6[j * 2 + k], bf16), s);
  s6[t] = s;
  y[t] = tanhf(s);
}

// d6 = dL/ds6 for L = (1/B) sum ||y - t||^2; loss accumulated.  The tanh
// derivative is taken as 1 / cosh(s)^2, which keeps its relative accuracy
// where tanh saturates (1 - y^2 would cancel).
__global__ void loss_grad(const float* y, const float* s6, const float* tgt, int B, float* d6,
                          float* loss) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * 2) return;
  const float r = y[t] - tgt[t];
  const float sech = 1.0f / coshf(s6[t]);
  d6[t] = 2.0f * r / (float)B * (sech * sech);
  atomicAdd(loss, r * r / (float)B);
}

// gW6 = h5^T d6, gb6 = sum d6, dh5 = (d6 W6^T) * (h5 > 0)
__global__ void out_back(const float* h5, const float* d6, const float* W6, int B, int H,
                         float* gW6, float* gb6, float* dh5) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < H * 2) {
    const int j = t / 2, k = t % 2;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s = fmaf(h5[b * H + j], d6[b * 2 + k], s);
    gW6[t] = s;
  }
  if (t < 2) {
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += d6[b * 2 + t];
    gb6[t] = s;
  }
  if (t < B * H) {
    const int b = t / H, j = t % H;
    const float s = d6[b * 2] * W6[j * 2] + d6[b * 2 + 1] * W6[j * 2 + 1];
    dh5[t] = h5[t] > 0.0f ? s : 0.0f;
  }
}

__global__ void relu_mask(float* d, const float* h, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && !(h[t] > 0.0f)) d[t] = 0.0f;
}

// gb[j] += sum over rows of d[r][j] (one block per 32 columns x 256 rows)
__global__ void col_sum(const float* d, long long R, int N, float* gb) {
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const long long r0 = (long long)blockIdx.y * 256 + (threadIdx.x >> 5) * 32;
  if (j >= N) return;
  float s = 0.0f;
  for (long long r = r0; r < r0 + 32 && r < R; ++r) s += d[r * N + j];
  atomicAdd(gb + j, s);
}

// dh3[arg[b][j]][j] = dz[b][j] (sets are disjoint, so every target is unique)
__global__ void pool_back(const float* du, int ldu, const int* arg, int B, int H, float* dh3) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * H) return;
  const int b = t / H, j = t % H;
  if (arg[t] >= 0) dh3[(size_t)arg[t] * H + j] = du[(size_t)b * ldu + j];
}

__global__ void adam(float* p, const float* g, float* m, float* v, long long n, float lr, float c1,
                     float c2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = 0.9f * m[t] + 0.1f * gt;
  const float vt = 0.999f * v[t] + 0.001f * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + 1e-8f);
}

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct pcba_mlp {
  int dp = 2, dg = 34, H = 128, prec = 16;
  int sms = 148;
  long long np = 0;
  long long off[12];  // offsets of W1, b1, ..., W6, b6 in the parameter vector
  float *d_par = nullptr, *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
  long long step = 0;
  long long launches = 0;  // kernels launched
  // workspace
  long long capP = 0, capB = 0;
  float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dA = nullptr, *dB = nullptr;
  float *z = nullptr, *u = nullptr, *h4 = nullptr, *h5 = nullptr, *y = nullptr, *du = nullptr;
  float *d4 = nullptr, *d5 = nullptr, *d6 = nullptr, *s6 = nullptr, *d_loss = nullptr;
  int* arg = nullptr;
  float* h_loss = nullptr;
};

namespace {

void free_ws(pcba_mlp* m) {
  float* f[] = {m->h1, m->h2, m->h3, m->dA, m->dB, m->z, m->u, m->h4, m->h5, m->y, m->du, m->d4,
                m->d5, m->d6, m->s6};
  for (float* p : f)
    if (p) cudaFree(p);
  if (m->arg) cudaFree(m->arg);
  m->h1 = m->h2 = m->h3 = m->dA = m->dB = m->z = m->u = m->h4 = m->h5 = m->y = m->du = m->d4 =
      m->d5 = m->d6 = m->s6 = nullptr;
  m->arg = nullptr;
  m->capP = m->capB = 0;
}

int ensure_ws(pcba_mlp* m, long long P, long long B) {
  if (P <= m->capP && B <= m->capB) return 0;
  cudaDeviceSynchronize();
  free_ws(m);
  const long long cP = std::max<long long>(P, 1024), cB = std::max<long long>(B, 64);
  const long long H = m->H, W = m->H + m->dg;
  float** pp[] = {&m->h1, &m->h2, &m->h3, &m->dA, &m->dB};
  for (float** q : pp)
    if (cudaMalloc((void**)q, sizeof(float) * cP * H) != cudaSuccess)
      return pcba_internal_fail(PCBA_ERR_OOM, "network workspace allocation failed");
  struct { float** p; long long n; } bb[] = {{&m->z, cB * H}, {&m->u, cB * W}, {&m->h4, cB * H},
                                             {&m->h5, cB * H}, {&m->y, cB * 2}, {&m->du, cB * W},
                                             {&m->d4, cB * H}, {&m->d5, cB * H}, {&m->d6, cB * 2},
                                             {&m->s6, cB * 2}};
  for (auto& q : bb)
    if (cudaMalloc((void**)q.p, sizeof(float) * q.n) != cudaSuccess)
      return pcba_internal_fail(PCBA_ERR_OOM, "network workspace allocation failed");
  if (cudaMalloc((void**)&m->arg, sizeof(int) * cB * H) != cudaSuccess)
    return pcba_internal_fail(PCBA_ERR_OOM, "network workspace allocation failed");
  m->capP = cP;
  m->capB = cB;
  return 0;
}

void gemm(const pcba_mlp* m, cudaStream_t s, int M, int N, int K, const float* A, int lda, int ta,
          const float* B, int ldb, int tb, float* C, int ldc, int beta) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  if (m->prec == 16) {
    const int tiles = ((N + GBN - 1) / GBN) * ((M + GBM - 1) / GBM);
    int splits = 1;
    if (beta && K > 4 * GBK * 8 && tiles < 2 * m->sms)
      splits = std::min((K + 8 * GBK - 1) / (8 * GBK), (2 * m->sms + tiles - 1) / tiles);
    const int kchunk = ((K + splits - 1) / splits + GBK - 1) / GBK * GBK;
    splits = (K + kchunk - 1) / kchunk;
    const dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, std::max(splits, 1));
    gemm_bf16<<<grid, 128, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, beta, kchunk);
  } else {
    const dim3 blk(16, 16), grid((N + 15) / 16, (M + 15) / 16);
    gemm_f32<<<grid, blk, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, beta);
  }
}

int check_batch(const pcba_mlp* m, int n_sets, int n_points) {
  if (!m) return pcba_internal_fail(PCBA_ERR_INVALID, "network is null");
  if (n_sets < 1 || n_points < n_sets)
    return pcba_internal_fail(PCBA_ERR_INVALID, "need n_sets >= 1 and a non-empty set each");
  return 0;
}

// forward pass; leaves activations in the workspace (12 kernels)
void forward(pcba_mlp* m, cudaStream_t s, const float* pts, const int* off, int B, int P,
             const float* glob) {
  m->launches += 12;
  const int H = m->H, W = m->H + m->dg;
  const float* par = m->d_par;
  const int bf16 = m->prec == 16;
  first_layer<<<blocks((long long)P * H), 256, 0, s>>>(pts, P, m->dp, par + m->off[0], par + m->off[1],
                                                       m->h1, H, bf16);
  gemm(m, s, P, H, H, m->h1, H, 0, par + m->off[2], H, 0, m->h2, H, 0);
  bias_relu<<<blocks((long long)P * H), 256, 0, s>>>(m->h2, P, H, par + m->off[3]);
  gemm(m, s, P, H, H, m->h2, H, 0, par + m->off[4], H, 0, m->h3, H, 0);
  bias_relu<<<blocks((long long)P * H), 256, 0, s>>>(m->h3, P, H, par + m->off[5]);
  set_maxpool<<<blocks((long long)B * H), 256, 0, s>>>(m->h3, off, B, P, H, m->z, m->arg);
  concat_rows<<<blocks((long long)B * W), 256, 0, s>>>(m->z, H, glob, m->dg, m->u, B);
  gemm(m, s, B, H, W, m->u, W, 0, par + m->off[6], H, 0, m->h4, H, 0);
  bias_relu<<<blocks((long long)B * H), 256, 0, s>>>(m->h4, B, H, par + m->off[7]);
  gemm(m, s, B, H, H, m->h4, H, 0, par + m->off[8], H, 0, m->h5, H, 0);
  bias_relu<<<blocks((long long)B * H), 256, 0, s>>>(m->h5, B, H, par + m->off[9]);
  out_layer<<<blocks((long long)B * 2), 256, 0, s>>>(m->h5, B, H, par + m->off[10], par + m->off[11],
                                                      m->y, m->s6, bf16);
}

// backward pass into d_grad (zeroed here) for targets tgt (21 kernels)
void backward(pcba_mlp* m, cudaStream_t s, const float* pts, const int* off, int B, int P,
              const float* tgt) {
  m->launches += 21;
  const int H = m->H, W = m->H + m->dg;
  const float* par = m->d_par;
  float* g = m->d_grad;
  cudaMemsetAsync(g, 0, sizeof(float) * m->np, s);
  cudaMemsetAsync(m->d_loss, 0, sizeof(float), s);
  loss_grad<<<blocks((long long)B * 2), 256, 0, s>>>(m->y, m->s6, tgt, B, m->d6, m->d_loss);
  out_back<<<blocks(std::max<long long>((long long)B * H, 2LL * H)), 256, 0, s>>>(
      m->h5, m->d6, par + m->off[10], B, H, g + m->off[10], g + m->off[11], m->d5);
  // layer 5: h5 = relu(h4 W5 + b5); m->d5 holds dL/dpre5
  gemm(m, s, H, H, B, m->h4, H, 1, m->d5, H, 0, g + m->off[8], H, 1);
  col_sum<<<dim3((H + 31) / 32, (unsigned)((B + 255) / 256)), 256, 0, s>>>(m->d5, B, H, g + m->off[9]);
  gemm(m, s, B, H, H, m->d5, H, 0, par + m->off[8], H, 1, m->d4, H, 0);
  relu_mask<<<blocks((long long)B * H), 256, 0, s>>>(m->d4, m->h4, (long long)B * H);
  // layer 4: h4 = relu(u W4 + b4)
  gemm(m, s, W, H, B, m->u, W, 1, m->d4, H, 0, g + m->off[6], H, 1);
  col_sum<<<dim3((H + 31) / 32, (unsigned)((B + 255) / 256)), 256, 0, s>>>(m->d4, B, H, g + m->off[7]);
  gemm(m, s, B, W, H, m->d4, H, 0, par + m->off[6], H, 1, m->du, W, 0);
  // max-pool: gradient to the maximising point of every column
  cudaMemsetAsync(m->dA, 0, sizeof(float) * (size_t)P * H, s);
  pool_back<<<blocks((long long)B * H), 256, 0, s>>>(m->du, W, m->arg, B, H, m->dA);
  // layer 3 (dA = dL/dh3)
  relu_mask<<<blocks((long long)P * H), 256, 0, s>>>(m->dA, m->h3, (long long)P * H);
  gemm(m, s, H, H, P, m->h2, H, 1, m->dA, H, 0, g + m->off[4], H, 1);
  col_sum<<<dim3((H + 31) / 32, (unsigned)((P + 255) / 256)), 256, 0, s>>>(m->dA, P, H, g + m->off[5]);
  gemm(m, s, P, H, H, m->dA, H, 0, par + m->off[4], H, 1, m->dB, H, 0);
  // layer 2 (dB = dL/dh2)
  relu_mask<<<blocks((long long)P * H), 256, 0, s>>>(m->dB, m->h2, (long long)P * H);
  gemm(m, s, H, H, P, m->h1, H, 1, m->dB, H, 0, g + m->off[2], H, 1);
  col_sum<<<dim3((H + 31) / 32, (unsigned)((P + 255) / 256)), 256, 0, s>>>(m->dB, P, H, g + m->off[3]);
  gemm(m, s, P, H, H, m->dB, H, 0, par + m->off[2], H, 1, m->dA, H, 0);
  // layer 1 (dA = dL/dh1)
  relu_mask<<<blocks((long long)P * H), 256, 0, s>>>(m->dA, m->h1, (long long)P * H);
  gemm(m, s, m->dp, H, P, pts, m->dp, 1, m->dA, H, 0, g + m->off[0], H, 1);
  col_sum<<<dim3((H + 31) / 32, (unsigned)((P + 255) / 256)), 256, 0, s>>>(m->dA, P, H, g + m->off[1]);
}

// splitmix64 + Box-Muller: the library's own seeded initialisation
double rand_normal(unsigned long long& st) {
  auto next = [&]() {
    unsigned long long z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const double u1 = ((next() >> 11) + 1.0) * 0x1p-53, u2 = (next() >> 11) * 0x1p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

extern "C" {

int pcba_mlp_create(pcba_mlp** out, int point_dim, int global_dim, int hidden, int precision,
                    unsigned long long seed) {
  if (!out) return pcba_internal_fail(PCBA_ERR_INVALID, "out is null");
  *out = nullptr;
  if (point_dim < 1 || global_dim < 0 || hidden < 1 || hidden > 4096 ||
      (precision != 16 && precision != 32))
    return pcba_internal_fail(PCBA_ERR_INVALID, "bad network shape or precision (16 or 32)");
  pcba_mlp* m = new pcba_mlp();
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, dev);
  m->dp = point_dim;
  m->dg = global_dim;
  m->H = hidden;
  m->prec = precision;
  const long long H = hidden;
  const long long sizes[12] = {point_dim * H, H, H * H, H, H * H, H, (H + global_dim) * H, H,
                               H * H, H, H * 2, 2};
  long long o = 0;
  for (int i = 0; i < 12; ++i) {
    m->off[i] = o;
    o += sizes[i];
  }
  m->np = o;
  std::vector<float> init((size_t)o, 0.0f);
  const long long fan_in[12] = {point_dim, 0, H, 0, H, 0, H + global_dim, 0, H, 0, H, 0};
  unsigned long long st = seed;
  for (int i = 0; i < 12; i += 2)
    for (long long q = 0; q < sizes[i]; ++q)
      init[(size_t)(m->off[i] + q)] = (float)(rand_normal(st) * std::sqrt(2.0 / (double)fan_in[i]));
  if (cudaMalloc((void**)&m->d_par, sizeof(float) * o) != cudaSuccess ||
      cudaMalloc((void**)&m->d_grad, sizeof(float) * o) != cudaSuccess ||
      cudaMalloc((void**)&m->d_m, sizeof(float) * o) != cudaSuccess ||
      cudaMalloc((void**)&m->d_v, sizeof(float) * o) != cudaSuccess ||
      cudaMalloc((void**)&m->d_loss, sizeof(float)) != cudaSuccess ||
      cudaMallocHost((void**)&m->h_loss, sizeof(float)) != cudaSuccess) {
    pcba_mlp_destroy(m);
    return pcba_internal_fail(PCBA_ERR_OOM, "network allocation failed");
  }
  cudaMemcpy(m->d_par, init.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
  cudaMemset(m->d_m, 0, sizeof(float) * o);
  cudaMemset(m->d_v, 0, sizeof(float) * o);
  *out = m;
  return 0;
}

void pcba_mlp_destroy(pcba_mlp* m) {
  if (!m) return;
  free_ws(m);
  float* f[] = {m->d_par, m->d_grad, m->d_m, m->d_v, m->d_loss};
  for (float* p : f)
    if (p) cudaFree(p);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  delete m;
}

long long pcba_mlp_num_params(const pcba_mlp* m) { return m ? m->np : 0; }

long long pcba_mlp_kernel_launches(const pcba_mlp* m) { return m ? m->launches : 0; }

int pcba_mlp_set_params(pcba_mlp* m, const float* host_params, long long n) {
  if (!m || !host_params || n != m->np) return pcba_internal_fail(PCBA_ERR_INVALID, "bad parameters");
  MLP_CK(cudaMemcpy(m->d_par, host_params, sizeof(float) * n, cudaMemcpyHostToDevice));
  MLP_CK(cudaMemset(m->d_m, 0, sizeof(float) * n));
  MLP_CK(cudaMemset(m->d_v, 0, sizeof(float) * n));
  m->step = 0;
  return 0;
}

int pcba_mlp_get_params(const pcba_mlp* m, float* host_params, long long n) {
  if (!m || !host_params || n != m->np) return pcba_internal_fail(PCBA_ERR_INVALID, "bad parameters");
  MLP_CK(cudaMemcpy(host_params, m->d_par, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return 0;
}

int pcba_mlp_forward(pcba_mlp* m, const float* d_points, const int* d_offsets, int n_sets,
                     int n_points, const float* d_global, float* d_out, void* stream) {
  int rc = check_batch(m, n_sets, n_points);
  if (rc) return rc;
  if ((rc = ensure_ws(m, n_points, n_sets))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  forward(m, s, d_points, d_offsets, n_sets, n_points, d_global);
  MLP_CK(cudaMemcpyAsync(d_out, m->y, sizeof(float) * 2 * n_sets, cudaMemcpyDeviceToDevice, s));
  MLP_CK(cudaGetLastError());
  return 0;
}

int pcba_mlp_gradient(pcba_mlp* m, const float* d_points, const int* d_offsets, int n_sets,
                      int n_points, const float* d_global, const float* d_target,
                      float* host_grad, float* loss, void* stream) {
  int rc = check_batch(m, n_sets, n_points);
  if (rc) return rc;
  if ((rc = ensure_ws(m, n_points, n_sets))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  forward(m, s, d_points, d_offsets, n_sets, n_points, d_global);
  backward(m, s, d_points, d_offsets, n_sets, n_points, d_target);
  MLP_CK(cudaGetLastError());
  if (host_grad)
    MLP_CK(cudaMemcpyAsync(host_grad, m->d_grad, sizeof(float) * m->np, cudaMemcpyDeviceToHost, s));
  MLP_CK(cudaMemcpyAsync(m->h_loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  MLP_CK(cudaStreamSynchronize(s));
  if (loss) *loss = *m->h_loss;
  return 0;
}

int pcba_mlp_train_step(pcba_mlp* m, const float* d_points, const int* d_offsets, int n_sets,
                        int n_points, const float* d_global, const float* d_target, float lr,
                        float* loss, void* stream) {
  int rc = check_batch(m, n_sets, n_points);
  if (rc) return rc;
  if ((rc = ensure_ws(m, n_points, n_sets))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  forward(m, s, d_points, d_offsets, n_sets, n_points, d_global);
  backward(m, s, d_points, d_offsets, n_sets, n_points, d_target);
  m->step += 1;
  const float c1 = 1.0f - (float)std::pow(0.9, (double)m->step);
  const float c2 = 1.0f - (float)std::pow(0.999, (double)m->step);
  adam<<<blocks(m->np), 256, 0, s>>>(m->d_par, m->d_grad, m->d_m, m->d_v, m->np, lr, c1, c2);
  m->launches += 1;
  MLP_CK(cudaGetLastError());
  if (loss) {
    MLP_CK(cudaMemcpyAsync(m->h_loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    MLP_CK(cudaStreamSynchronize(s));
    *loss = *m->h_loss;
  }
  return 0;
}

}  // extern "C"
