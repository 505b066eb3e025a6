// Set-encoder network of the learned warm start (not part of the paper):
// training and inference kernels.  See include/pcba.h (pcba_mlp_*).
//
//   h1_p = relu(x_p W1 + b1), h2_p = relu(h1_p W2 + b2), h3_p = relu(h2_p W3 + b3)
//   z = max_p h3_p,  h4 = relu([z, u] W4 + b4),  h5 = relu(h4 W5 + b5),
//   y = tanh(h5 W6 + b6),  loss = (1/B) sum_b ||y_b - t_b||^2
//
// The dense layers run as GEMMs on the 5th-generation tensor cores (tcgen05,
// BF16 operands rounded from the FP32 master copies, FP32 accumulation in
// tensor memory); a plain FP32 GEMM replaces them in the FP32 debug precision.  Weights are row-major
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
//
// BF16 precision runs on the 5th-generation tensor cores: one CTA computes a
// 128 x 128 tile of C with tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulation in tensor memory).  Operands are read as FP32, rounded to BF16
// and written to shared memory in the canonical K-major layout without
// swizzle: core matrices of 8 rows x 16 bytes, the 16 row groups of one 8-wide
// k slice contiguous (stride 128 B), k slices 2 KB apart.  K advances in
// chunks of 64 through two shared-memory stages; a single thread issues the
// MMAs (K = 16 each) and commits them to the stage's mbarrier, which the
// threads wait on (bounded) before refilling the stage.  The epilogue reads
// the accumulators with tcgen05.ld (warp w owns rows 32w .. 32w+31).
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_N = 128, TC_K = 64;
constexpr int TC_STAGE_BYTES = (TC_M + TC_N) * TC_K * 2;  // 32 KB: A then B
constexpr int TC_SMEM = 2 * TC_STAGE_BYTES + 1024;        // + alignment slack

__device__ __forceinline__ unsigned tc_smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle; LBO = 2048 B between
// k slices, SBO = 128 B between 8-row groups; descriptor version 1
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr) {
  return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)(2048 >> 4) << 16) |
         ((unsigned long long)(128 >> 4) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major
__device__ __forceinline__ unsigned tc_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(bar)) : "memory");
}

// bounded wait for the given phase parity; false after about one second
__device__ __forceinline__ bool tc_mbar_wait(unsigned long long* bar, unsigned parity) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc_smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

// stage one 128 x 64 operand block: row t of the tile (m for A, n for B) and
// eight k slices of 8 values each, written as 16-byte rows of core matrices
__device__ __forceinline__ void tc_stage(__nv_bfloat16* dst, const float* X, int ld, int trans,
                                         int r0, int rows, int k0, int kend, int t) {
  const int r = r0 + t;
  // rows of X contiguous in k, 16-byte aligned and fully inside: two float4 loads per slice
  const bool vec = !trans && r < rows && (ld & 3) == 0 && (k0 & 3) == 0 &&
                   (((size_t)X) & 15) == 0;
  // all eight slices unrolled: their loads are in flight together
#pragma unroll
  for (int c8 = 0; c8 < TC_K / 8; ++c8) {
    __align__(16) __nv_bfloat16 v[8];
    const int kb = k0 + c8 * 8;
    if (vec && kb + 8 <= kend) {
      const float4 a = *(const float4*)(X + (size_t)r * ld + kb);
      const float4 b = *(const float4*)(X + (size_t)r * ld + kb + 4);
      v[0] = __float2bfloat16_rn(a.x); v[1] = __float2bfloat16_rn(a.y);
      v[2] = __float2bfloat16_rn(a.z); v[3] = __float2bfloat16_rn(a.w);
      v[4] = __float2bfloat16_rn(b.x); v[5] = __float2bfloat16_rn(b.y);
      v[6] = __float2bfloat16_rn(b.z); v[7] = __float2bfloat16_rn(b.w);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = kb + e;
        float x = 0.0f;
        if (r < rows && k < kend) x = trans ? X[(size_t)k * ld + r] : X[(size_t)r * ld + k];
        v[e] = __float2bfloat16_rn(x);
      }
    }
    *(uint4*)(dst + ((c8 * 16 + (t >> 3)) * 64 + (t & 7) * 8)) = *(const uint4*)v;
  }
}

// A operand "row" = m, B operand "row" = n: A(m,k) and B(k,n) staged as [m][k], [n][k]
__global__ void __launch_bounds__(128) gemm_tc(int M, int N, int K, const float* __restrict__ A,
                                               int lda, int ta, const float* __restrict__ B,
                                               int ldb, int tb, float* C, int ldc, int beta,
                                               int kchunk, int* err) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) unsigned long long bars[3];
  __shared__ unsigned tmem_base;
  unsigned char* sm = (unsigned char*)(((size_t)tc_raw + 1023) & ~(size_t)1023);
  const int t = threadIdx.x, warp = t >> 5;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int nchunks = kend > kbeg ? (kend - kbeg + TC_K - 1) / TC_K : 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     tc_smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int q = 0; q < 3; ++q) tc_mbar_init(&bars[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  const unsigned idesc = tc_idesc(TC_M, TC_N);
  bool ok = true;
  for (int c = 0; c < nchunks && ok; ++c) {
    const int s = c & 1;
    unsigned char* stage = sm + s * TC_STAGE_BYTES;
    __nv_bfloat16* sA = (__nv_bfloat16*)stage;
    __nv_bfloat16* sB = (__nv_bfloat16*)(stage + TC_M * TC_K * 2);
    if (c >= 2) ok = tc_mbar_wait(&bars[s], (unsigned)((c - 2) >> 1) & 1u);
    if (!__syncthreads_and(ok ? 1 : 0)) {
      ok = false;
      break;
    }
    const int k0 = kbeg + c * TC_K;
    tc_stage(sA, A, lda, ta, m0, M, k0, kend, t);
    tc_stage(sB, B, ldb, !tb, n0, N, k0, kend, t);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < TC_K / 16; ++ks) {
        const unsigned long long ad = tc_desc(tc_smem_u32(sA) + ks * 2 * 2048);
        const unsigned long long bd = tc_desc(tc_smem_u32(sB) + ks * 2 * 2048);
        const unsigned acc = (c > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              tc_smem_u32(&bars[s]))
          : "memory");
    }
  }
  if (nchunks > 0) {
    if (t == 0)
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              tc_smem_u32(&bars[2]))
          : "memory");
    // all MMAs issued (also after a timeout) finish before tensor memory is read or freed
    const bool done = tc_mbar_wait(&bars[2], 0u);
    ok = __syncthreads_and((ok && done) ? 1 : 0) != 0;
    if (!done && t == 0) atomicExch(err, 1);
  }
  if (!ok && t == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && nchunks > 0) {
    const int row = m0 + warp * 32 + (t & 31);
    const bool split = gridDim.z > 1;
#pragma unroll 1
    for (int j = 0; j < TC_N / 32; ++j) {
      unsigned v[32];
      const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(j * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        const int cb = n0 + j * 32;
        float* drow = C + (size_t)row * ldc + cb;
        if (!split && cb + 32 <= N && (ldc & 3) == 0 && (((size_t)drow) & 15) == 0) {
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            float4 x = make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]),
                                   __uint_as_float(v[i + 2]), __uint_as_float(v[i + 3]));
            if (beta) {
              const float4 o = *(const float4*)(drow + i);
              x.x += o.x; x.y += o.y; x.z += o.z; x.w += o.w;
            }
            *(float4*)(drow + i) = x;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if (cb + i < N) {
              const float x = __uint_as_float(v[i]);
              if (split) atomicAdd(drow + i, x);
              else drow[i] = x + (beta ? drow[i] : 0.0f);
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
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
  int* d_err = nullptr;  // set by a tensor-core GEMM whose bounded wait ran out
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
    const int tiles = ((N + TC_N - 1) / TC_N) * ((M + TC_M - 1) / TC_M);
    int splits = 1;
    if (beta && K > 8 * TC_K && tiles < 2 * m->sms)
      splits = std::min((K + 4 * TC_K - 1) / (4 * TC_K), (2 * m->sms + tiles - 1) / tiles);
    const int kchunk = ((K + splits - 1) / splits + TC_K - 1) / TC_K * TC_K;
    splits = (K + kchunk - 1) / kchunk;
    const dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M, std::max(splits, 1));
    gemm_tc<<<grid, 128, TC_SMEM, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, beta, kchunk,
                                        m->d_err);
  } else {
    const dim3 blk(16, 16), grid((N + 15) / 16, (M + 15) / 16);
    gemm_f32<<<grid, blk, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, beta);
  }
}

// a tensor-core GEMM that timed out leaves a flag; reported (and cleared) at
// the next synchronising call
int check_err(pcba_mlp* m) {
  int e = 0;
  if (cudaMemcpy(&e, m->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return pcba_internal_fail(PCBA_ERR_CUDA, "network error flag unreadable");
  if (e) {
    cudaMemset(m->d_err, 0, sizeof(int));
    return pcba_internal_fail(PCBA_ERR_DEVICE_TIMEOUT, "a tensor-core GEMM wait timed out");
  }
  return 0;
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
      cudaMalloc((void**)&m->d_err, sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&m->h_loss, sizeof(float)) != cudaSuccess) {
    pcba_mlp_destroy(m);
    return pcba_internal_fail(PCBA_ERR_OOM, "network allocation failed");
  }
  cudaMemcpy(m->d_par, init.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
  cudaMemset(m->d_m, 0, sizeof(float) * o);
  cudaMemset(m->d_v, 0, sizeof(float) * o);
  cudaMemset(m->d_err, 0, sizeof(int));
  if (cudaFuncSetAttribute(gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) !=
      cudaSuccess) {
    pcba_mlp_destroy(m);
    return pcba_internal_fail(PCBA_ERR_CUDA, "cannot configure the tensor-core GEMM");
  }
  *out = m;
  return 0;
}

void pcba_mlp_destroy(pcba_mlp* m) {
  if (!m) return;
  free_ws(m);
  float* f[] = {m->d_par, m->d_grad, m->d_m, m->d_v, m->d_loss};
  for (float* p : f)
    if (p) cudaFree(p);
  if (m->d_err) cudaFree(m->d_err);
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
  return check_err(m);
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
    return check_err(m);
  }
  return 0;
}

}  // extern "C"
