// Kernels of one PCBA step (Algorithm 1) for many problems at once, plus the
// monomial-to-Bernstein conversion and the point checks.  The point
// evaluations (warm start, final check) live in pcba_eval.cuh, included
// below; the subdivision kernels (pcba_subdivide.cuh, pcba_linear.cuh) and
// the local polish of an incumbent (pcba_polish.cuh) are compiled in their
// own translation units (pcba_k2.cu, pcba_polish.cu).
//
//   k1_matrices / k1_convert  Alg. 1 line 1 (InitPatches, Sec. II-D): per axis
//                             the matrix T_r = (power -> Bernstein on [0,1]) x
//                             (affine map [lo,hi] -> [0,1]), applied as l mode
//                             products to every monomial tensor, in FP64.
//   k2_subdivide(_tma)        Alg. 2 + Alg. 3: bisect every item in direction r
//                             (de Casteljau at 1/2 on every fibre, Sec. II-E)
//                             and bound every child patch by the min and max of
//                             its coefficients (Thm. 1) into per-child records;
//                             the _tma variant stages parent tiles in shared
//                             memory with bulk tensor copies.
//   k_pup                     Def. 4: the solution estimate p_up (min over
//                             feasible children), and the returned box.
//   k_refresh                 FP32 mode: recomputes marked patches from the
//                             FP64 monomials over their box (tighter bounds).
//   k3_classify               Alg. 4 (readings R3-R5): keep = not infeasible
//                             (Def. 3) and not suboptimal (Def. 5); p_lo; scan of
//                             the keep flags; the last tile of each problem runs
//                             the stopping tests (Alg. 1 lines 4, 8, 9, 11) and
//                             the last tile overall plans the next step.
//   k4_index / k_move_control Alg. 5 (reading R11) on the slot map: the j-th
//                             hole below K_save receives the slot of the item at
//                             save position K_save-1-j; one block runs the
//                             device-side loop control (graph conditional)
//                             beside the moves.
//   k_eval                    warm start: certified candidate points seed p_up
//                             (FP32 with error bounds); final check of the
//                             returned point in FP64 with an error bound.
//   k_candidates, k_mono32,   warm-start helpers: candidate points around a
//   k_cost_grid               guess, FP32 copy of the monomials, and the cost
//                             on a grid (network features).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "pcba_device.cuh"

// ---------------------------------------------------------------------------
// small exact helpers
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// K1: monomial -> Bernstein
// ---------------------------------------------------------------------------
// mat layout: ((p * 3 + fam) * PCBA_MAXD + r) * 578 doubles: first T_r, then
// the entrywise bound |B||S| of the same size.
// T_r[i][j] = sum_{k <= min(i,j)} [C(i,k)/C(n,k)] * C(j,k) lo^(j-k) w^k maps
// the power coefficients of one fibre to its Bernstein coefficients over
// [lo, lo+w].  Since |T| <= |B||S| and the rounding of the computed T and of
// its products is bounded by gamma * |B||S| |a| entrywise, the conversion
// error of a patch is at most gamma * (|B_1||S_1| x ... x |B_l||S_l|) |a|.
__global__ void k1_matrices(Engine E, double* mat) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid == 0) E.plan->t0 = globaltimer();
  const int per = 3 * PCBA_MAXD * 17;
  if (gid >= E.np * per) return;
  const int p = gid / per;
  const int rem = gid - p * per;
  const int fam = rem / (PCBA_MAXD * 17);
  const int r = (rem / 17) % PCBA_MAXD;
  const int i = rem % 17;
  const ProbDesc& D = E.desc[p];
  if (r >= D.l) return;
  const int* deg = fam == 0 ? D.P : (fam == 1 ? D.G : D.H);
  const int n = deg[r];
  if (i > n) return;
  const double lo = D.lo[r], w = D.hi[r] - D.lo[r];
  double* T = mat + ((size_t)(p * 3 + fam) * PCBA_MAXD + r) * 578;
  double* A = T + 289;
  for (int j = 0; j <= n; ++j) {
    double t = 0.0, ta = 0.0;
    const int kmax = i < j ? i : j;
    for (int k = 0; k <= kmax; ++k) {
      const double term = dev_binom(i, k) / dev_binom(n, k) * dev_binom(j, k) *
                          dev_pow(lo, j - k) * dev_pow(w, k);
      t += term;
      ta += fabs(term);
    }
    T[i * (n + 1) + j] = t;
    A[i * (n + 1) + j] = ta * (1.0 + 0x1p-40);  // covers the rounding of the bound itself
  }
}

// One warp converts one patch: load the monomial tensor into shared memory,
// apply the l mode products, then store it into item 0 of the list.
template <typename T>
__global__ void __launch_bounds__(128) k1_convert(Engine E, const double* mat, int cmax, int wpb) {
  extern __shared__ double k1s[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* sA = k1s + (size_t)wid * (4 * cmax + 578);
  double* sB = sA + cmax;
  double* sX = sB + cmax;   // |a| carried through the |B||S| products
  double* sY = sX + cmax;
  double* sT = sY + cmax;
  const unsigned total = E.k1_pre[E.np];
  for (unsigned u = blockIdx.x * wpb + wid; u < total; u += gridDim.x * wpb) {
    const int p = find_problem(E.k1_pre, E.np, u);
    const ProbDesc& D = E.desc[p];
    const int q = (int)(u - E.k1_pre[p]);
    int fam, idx, C;
    const int* deg;
    long long aoff;
    if (q == 0) {
      fam = 0; idx = 0; deg = D.P; C = D.cp; aoff = 0;
    } else if (q <= D.alpha) {
      fam = 1; idx = q - 1; deg = D.G; C = D.cg; aoff = D.cp + (long long)idx * D.cg;
    } else {
      fam = 2; idx = q - 1 - D.alpha; deg = D.H; C = D.ch;
      aoff = D.cp + (long long)D.alpha * D.cg + (long long)idx * D.ch;
    }
    const double* a = E.mono + D.mono_off + aoff;
    for (int j = lane; j < C; j += 32) {
      const double v = a[j];
      sA[j] = v;
      sX[j] = fabs(v);
    }
    __syncwarp();
    double err64 = 0.0;
    if (!D.form_bernstein) {
      double gterms = 0.0;
      for (int r = 0; r < D.l; ++r) {
        const int n = deg[r];
        int stride = 1;
        for (int s = r + 1; s < D.l; ++s) stride *= deg[s] + 1;
        const double* Tg = mat + ((size_t)(p * 3 + fam) * PCBA_MAXD + r) * 578;
        for (int e = lane; e < (n + 1) * (n + 1); e += 32) {
          sT[e] = Tg[e];
          sT[289 + e] = Tg[289 + e];
        }
        gterms += 4.0 * n + 8.0;
        __syncwarp();
        const int blk = (n + 1) * stride;
        for (int o = lane; o < C; o += 32) {
          const int hp = o / blk;
          const int rem = o - hp * blk;
          const int i = rem / stride;
          const int in = rem - i * stride;
          const double* src = sA + hp * blk + in;
          const double* srcx = sX + hp * blk + in;
          double s = 0.0, sx = 0.0;
          for (int j = 0; j <= n; ++j) {
            s = fma(sT[i * (n + 1) + j], src[j * stride], s);
            sx = __dadd_ru(sx, __dmul_ru(sT[289 + i * (n + 1) + j], srcx[j * stride]));
          }
          sB[o] = s;
          sY[o] = sx;
        }
        __syncwarp();
        double* tmp = sA; sA = sB; sB = tmp;
        tmp = sX; sX = sY; sY = tmp;
      }
      // FP64 rounding of the conversion, per patch:
      //   |b - exact| <= gamma * max_J ((|B_1||S_1| x ... x |B_l||S_l|) |a|)_J
      double amax = 0.0;
      for (int j = lane; j < C; j += 32) amax = fmax(amax, sX[j]);
      for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      err64 = __dmul_ru(__dmul_ru(2.0 * gterms, 0x1p-53), amax);
    }
    if (E.root_raw) {
      double* raw = E.root_raw + D.mono_off + aoff;
      for (int j = lane; j < C; j += 32) raw[j] = sA[j];
    }
    char* item0 = E.arena + D.list_off;
    if constexpr (sizeof(T) == 8) {
      double* dst;
      size_t pad;
      if (fam == 0) { dst = (double*)(item0 + D.off_cost); pad = 1; }
      else if (fam == 1) { dst = (double*)(item0 + D.off_g) + idx; pad = D.apad; }
      else { dst = (double*)(item0 + D.off_h) + idx; pad = D.bpad; }
      for (int j = lane; j < C; j += 32) dst[(size_t)j * pad] = sA[j];
    } else if (fam != 0) {
      float* dst = (float*)(item0 + (fam == 1 ? D.off_g : D.off_h)) + idx;
      const size_t pad = fam == 1 ? D.apad : D.bpad;
      // dense families: stored relative to an FP32 offset o, the middle of
      // the coefficient range rounded to FP32, so that the rounding error
      // scales with the range; linear families' shared patches are stored
      // absolute here (k_init gives them their offsets)
      double o = 0.0;
      if (!D.lin) {
        double bmin = INFINITY, bmax = -INFINITY;
        for (int j = lane; j < C; j += 32) { bmin = fmin(bmin, sA[j]); bmax = fmax(bmax, sA[j]); }
        for (int w = 16; w > 0; w >>= 1) {
          bmin = fmin(bmin, __shfl_xor_sync(0xffffffffu, bmin, w));
          bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, w));
        }
        o = (double)__double2float_rn(0.5 * (bmin + bmax));
      }
      double emax = 0.0;
      for (int j = lane; j < C; j += 32) {
        if (D.lin) {
          const float s = __double2float_rn(sA[j]);
          dst[(size_t)j * pad] = s;
          emax = fmax(emax, fabs((double)s - sA[j]));  // exact in double
        } else {
          const double d = sA[j] - o;  // |d - (b - o)| <= |d| 2^-53
          const float s = __double2float_rn(d);
          dst[(size_t)j * pad] = s;
          emax = fmax(emax, __dadd_ru(fabs((double)s - d), __dmul_ru(fabs(d), 0x1p-52)));
        }
      }
      for (int w = 16; w > 0; w >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, w));
      if (lane == 0) {
        ((float*)(item0 + (fam == 1 ? D.off_eg : D.off_eh)))[idx] =
            __double2float_ru(__dadd_ru(emax, err64));
        if (!D.lin) ((float*)(item0 + (fam == 1 ? D.off_og : D.off_oh)))[idx] = (float)o;
      }
    } else {
      // cost: stored = value - O with O the centre of the coefficient range
      double bmin = INFINITY, bmax = -INFINITY;
      for (int j = lane; j < C; j += 32) { bmin = fmin(bmin, sA[j]); bmax = fmax(bmax, sA[j]); }
      for (int o = 16; o > 0; o >>= 1) {
        bmin = fmin(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
      }
      const double O = 0.5 * (bmin + bmax);
      float* dst = (float*)(item0 + D.off_cost);
      double emax = 0.0;
      for (int j = lane; j < C; j += 32) {
        const double d = sA[j] - O;               // |d - (b - O)| <= |d| 2^-53
        const float s = __double2float_rn(d);
        dst[j] = s;
        emax = fmax(emax, __dadd_ru(fabs((double)s - d), __dmul_ru(fabs(d), 0x1p-52)));
      }
      for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      if (lane == 0) {
        *(double*)(item0 + 32) = O;
        *(float*)(item0 + 40) = __double2float_ru(__dadd_ru(emax, err64));
      }
    }
    __syncwarp();
  }
}


// ---------------------------------------------------------------------------
// FP32 mode: refresh of marked patches from the FP64 monomials
// ---------------------------------------------------------------------------
// The error bound of an FP32 patch only grows from step to step, and most of
// it is collected in the first bisections, when Bernstein coefficients on the
// large boxes are far larger than the polynomial's values.  Right after the
// subdivision, this kernel takes the patches that step marked (their bound
// changed a decision, see mark_err) and recomputes each, in its child slot,
// directly from the FP64 monomial coefficients over the child's box (Sec.
// II-D, the conversion of k1_convert with the box of the item): the new bound
// is the FP64 conversion bound plus one rounding to FP32.  Unmarked patches
// keep their (larger, still valid) bound.  It runs beside k_pup, k3_classify
// and k4_index, which read only the child records, and must finish before
// k_move_control updates the slot map; the child boxes come from the state snapshot
// child_level, which those kernels do not change.
//
// One block of PCBA_KRB threads per marked item: the per-axis matrices of the
// item's box and the conversion are spread over the block's warps, which sit
// on different SM partitions, so that the FP64 work of one mark runs on
// several FP64 units at once (an FP64 instruction occupies its partition's
// unit for many cycles, whatever the other warps do).
#define PCBA_KRB 128

// Binomial coefficients C(n, k), n, k <= 16 (exact integers), and their
// rounded reciprocals, filled once by the library at start-up.
__constant__ double c_binom[17 * 17];
__constant__ double c_binom_inv[17 * 17];

// Doubles of per-axis scratch of refresh_matrices: the factors U and V
// ([17][17] each), the powers lo^e and w^e ([17] each), and U and V as
// FP32 absolute values rounded up ([17][17] each, one double of space per
// two floats).
#define PCBA_KR_SCRATCH (2 * 289 + 2 * 17 + 289)

// The mode products' axis r and in-axis index of flat item t over the axes'
// (n_r + 1)^2 grids (sq) or (n_r + 1) ranges.
__device__ __forceinline__ int refresh_axis(const int* deg, int l, bool sq, int& t) {
  int r = 0;
  for (; r < l - 1; ++r) {
    const int m = sq ? (deg[r] + 1) * (deg[r] + 1) : deg[r] + 1;
    if (t < m) break;
    t -= m;
  }
  return r;
}

// T_r[i][j] = sum_k C(i,k) C(j,k) / C(n,k) lo^(j-k) w^k (power basis on the
// box -> Bernstein basis), formed as sum_k U[i][k] V[j][k] with U[i][k] =
// C(i,k) / C(n,k) w^k and V[j][k] = C(j,k) lo^(j-k) (each factor computed
// once, a power with at most e - 1 products by repeated squaring), for every
// axis at once; A_r bounds the absolute-value sum sum_k |U[i][k]| |V[j][k]|
// from above in FP32 (factors and products rounded up, then widened by
// 2^-20, which covers the FP64 roundings of U and V), stored as the 289
// floats after T_r's 289 doubles.  scr: l x PCBA_KR_SCRATCH doubles; box:
// lo[0..l-1], then hi[0..l-1].  Whole block.
__device__ __forceinline__ void refresh_matrices(const double* binom, int l, const int* deg,
                                                 const double* box, double* sT, double* scr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int n1 = 0, n2 = 0;
  for (int r = 0; r < l; ++r) {
    n1 += deg[r] + 1;
    n2 += (deg[r] + 1) * (deg[r] + 1);
  }
  for (int t0 = tid; t0 < n1; t0 += nt) {
    int e = t0;
    const int r = refresh_axis(deg, l, false, e);
    double xa = box[r], xb = box[l + r] - box[r], a = 1.0, b = 1.0;
    for (int k = e; k > 0;) {
      if (k & 1) {
        a *= xa;
        b *= xb;
      }
      k >>= 1;
      if (k) {
        xa *= xa;
        xb *= xb;
      }
    }
    double* s = scr + r * PCBA_KR_SCRATCH;
    s[578 + e] = a;
    s[595 + e] = b;
  }
  __syncthreads();
  for (int t0 = tid; t0 < n2; t0 += nt) {
    int e = t0;
    const int r = refresh_axis(deg, l, true, e);
    const int n = deg[r], i = e / (n + 1), k = e - i * (n + 1);
    if (k > i) continue;
    double* s = scr + r * PCBA_KR_SCRATCH;
    float* f = (float*)(s + 612);
    const double u = binom[i * 17 + k] * c_binom_inv[n * 17 + k] * s[595 + k];
    const double v = binom[i * 17 + k] * s[578 + i - k];
    s[i * 17 + k] = u;
    s[289 + i * 17 + k] = v;
    f[i * 17 + k] = __double2float_ru(fabs(u));
    f[289 + i * 17 + k] = __double2float_ru(fabs(v));
  }
  __syncthreads();
  for (int t0 = tid; t0 < n2; t0 += nt) {
    int e = t0;
    const int r = refresh_axis(deg, l, true, e);
    const int n = deg[r], i = e / (n + 1), j = e - i * (n + 1);
    const double* s = scr + r * PCBA_KR_SCRATCH;
    const float* f = (const float*)(s + 612);
    double t = 0.0;
    float ta = 0.0f;
    const int kmax = i < j ? i : j;
    for (int k = 0; k <= kmax; ++k) {
      t = fma(s[i * 17 + k], s[289 + j * 17 + k], t);
      ta = __fmaf_ru(f[i * 17 + k], f[289 + j * 17 + k], ta);
    }
    double* T = sT + r * 578;
    T[e] = t;
    ((float*)(T + 289))[e] = __fmul_ru(ta, 1.0f + 0x1p-20f);
  }
  __syncthreads();
}

// Minimum or maximum of NV values over the block, in every thread; red holds
// NV x (warps per block) floats.
template <int NV, bool MAX>
__device__ __forceinline__ void refresh_block_reduce(float (&v)[NV], float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float y = __shfl_xor_sync(0xffffffffu, v[q], o);
      v[q] = MAX ? fmaxf(v[q], y) : fminf(v[q], y);
    }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[w * NV + q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    float x = red[q];
    for (int i = 1; i < nw; ++i) x = MAX ? fmaxf(x, red[i * NV + q]) : fminf(x, red[i * NV + q]);
    v[q] = x;
  }
  __syncthreads();
}

// Conversion of the nf (<= PCBA_MAX_SHARED) monomial tensors a[g C + j] of
// one multi-degree with the matrices in sT (l mode products, every pass over
// all nf C coefficients, each output summed in two partial sums: at most
// n + 1 roundings on any path, as a single chain); result in *sA.  The bound
// base (|A_1| x ... x |A_l|) |a| is carried in FP32 with every input and
// every fused multiply-add rounded up, so it stays an upper bound of the
// exact product and costs no FP64 operations (a value beyond the FP32 range
// gives an infinite bound: the patch is then never decided on).  err[g]
// receives patch g's conversion bound, rounded up (every thread).  Whole block; red:
// PCBA_MAX_SHARED x warps floats.
__device__ __forceinline__ void refresh_convert(const double* a, int nf, int C, int l,
                                                const int* deg, const double* sT, double*& sA,
                                                double*& sB, float*& sX, float*& sY, float* red,
                                                float* err) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int N = nf * C;
  for (int j = tid; j < N; j += nt) {
    const double v = a[j];
    sA[j] = v;
    sX[j] = __double2float_ru(fabs(v));
  }
  __syncthreads();
  int gterms = 0;
  for (int r = 0; r < l; ++r) {
    const int n = deg[r];
    int stride = 1;
    for (int q = r + 1; q < l; ++q) stride *= deg[q] + 1;
    const double* T = sT + r * 578;
    const float* A = (const float*)(T + 289);
    gterms += 4 * n + 8;
    const int blk = (n + 1) * stride;
    for (int o2 = tid; o2 < N; o2 += nt) {
      const int g = o2 / C;
      const int o = o2 - g * C;
      const int hp = o / blk;
      const int rem = o - hp * blk;
      const int i = rem / stride;
      const int in = rem - i * stride;
      const double* src = sA + g * C + hp * blk + in;
      const float* srcx = sX + g * C + hp * blk + in;
      const double* Ti = T + i * (n + 1);
      const float* Ai = A + i * (n + 1);
      double s0 = 0.0, s1 = 0.0;
      float x0 = 0.0f, x1 = 0.0f;
      int j = 0;
      for (; j < n; j += 2) {
        s0 = fma(Ti[j], src[j * stride], s0);
        s1 = fma(Ti[j + 1], src[(j + 1) * stride], s1);
        x0 = __fmaf_ru(Ai[j], srcx[j * stride], x0);
        x1 = __fmaf_ru(Ai[j + 1], srcx[(j + 1) * stride], x1);
      }
      if (j == n) {
        s0 = fma(Ti[j], src[j * stride], s0);
        x0 = __fmaf_ru(Ai[j], srcx[j * stride], x0);
      }
      sB[o2] = s0 + s1;
      sY[o2] = __fadd_ru(x0, x1);
    }
    __syncthreads();
    double* t = sA; sA = sB; sB = t;
    float* tf = sX; sX = sY; sY = tf;
  }
  float am[PCBA_MAX_SHARED] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int j = tid; j < N; j += nt) {
    const int g = j / C;
#pragma unroll
    for (int q = 0; q < PCBA_MAX_SHARED; ++q)
      if (q == g) am[q] = fmaxf(am[q], sX[j]);
  }
  refresh_block_reduce<PCBA_MAX_SHARED, true>(am, red);
  // 2 gterms 2^-53 am, rounded up in FP32 (2 gterms < 2^11: the scale is exact)
#pragma unroll
  for (int q = 0; q < PCBA_MAX_SHARED; ++q)
    err[q] = __fmul_ru((float)(2 * gterms) * 0x1p-53f, am[q]);
}

// An upper bound of |x| 2^-52 (at least the rounding error of an FP64 sum
// whose result is x) from x's exponent field alone, without an FP64
// instruction: |x| < 2^(E - 1022) for the biased exponent E.  At most twice
// |x| 2^-52 above 2^-126, +inf for a non-finite x.
__device__ __forceinline__ float refresh_ulp_bound(double x) {
  const int fe = max(((__double2hiint(x) >> 20) & 0x7ff) - 947, 1);
  return fe >= 255 ? INFINITY : __int_as_float(fe << 23);
}

// Stores the nf converted patches (sA, C each), each re-centred on an FP32
// offset O_g near the middle of its range, as FP32 values at
// dst[(j - g C) * pad + g]: stored = RN(b - O) with b - O formed in FP64 (error
// at most |b - O| 2^-53), so the bound is |stored - (b - O)| + |b - O| 2^-52
// (each rounded up), maximised over the patch, plus err[g].  Patch g's bound
// goes to eout[g], its offset to o64[g] (FP64) or, when o64 is null, o32[g].  The range
// is found in FP32 (any offset is valid; the middle only keeps the stored
// values small); a patch whose values leave the FP32 range takes its offset
// from an FP64 pass of one thread.  Whole block; red: 2 PCBA_MAX_SHARED x
// warps floats, sO: PCBA_MAX_SHARED doubles.
__device__ __forceinline__ void refresh_store(const double* sA, int nf, int C, const float* err,
                                              float* dst, size_t pad, float* eout, double* o64,
                                              float* o32, float* red, double* sO) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int N = nf * C;
  float mn[PCBA_MAX_SHARED], mx[PCBA_MAX_SHARED];
#pragma unroll
  for (int q = 0; q < PCBA_MAX_SHARED; ++q) {
    mn[q] = INFINITY;
    mx[q] = -INFINITY;
  }
  for (int j = tid; j < N; j += nt) {
    const int g = j / C;
    const float v = __double2float_rn(sA[j]);
#pragma unroll
    for (int q = 0; q < PCBA_MAX_SHARED; ++q)
      if (q == g) {
        mn[q] = fminf(mn[q], v);
        mx[q] = fmaxf(mx[q], v);
      }
  }
  refresh_block_reduce<PCBA_MAX_SHARED, false>(mn, red);
  refresh_block_reduce<PCBA_MAX_SHARED, true>(mx, red + PCBA_MAX_SHARED * (nt >> 5));
  if (tid < nf) {
    float o = 0.0f;
#pragma unroll
    for (int q = 0; q < PCBA_MAX_SHARED; ++q)
      if (q == tid) o = 0.5f * mn[q] + 0.5f * mx[q];
    if (!isfinite(o)) {
      double lo = INFINITY, hi = -INFINITY;
      for (int j = tid * C; j < (tid + 1) * C; ++j) {
        lo = fmin(lo, sA[j]);
        hi = fmax(hi, sA[j]);
      }
      o = __double2float_rn(0.5 * lo + 0.5 * hi);
      if (!isfinite(o)) o = 0.0f;
    }
    sO[tid] = (double)o;
  }
  __syncthreads();
  float em[PCBA_MAX_SHARED] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int j = tid; j < N; j += nt) {
    const int g = j / C;
    const double d = sA[j] - sO[g];  // |d - (b - O)| <= |d| 2^-53
    const float sv = __double2float_rn(d);
    dst[(size_t)(j - g * C) * pad + g] = sv;
    const float e = __fadd_ru(__double2float_ru(fabs((double)sv - d)), refresh_ulp_bound(d));
#pragma unroll
    for (int q = 0; q < PCBA_MAX_SHARED; ++q)
      if (q == g) em[q] = fmaxf(em[q], e);
  }
  refresh_block_reduce<PCBA_MAX_SHARED, true>(em, red);
  if (tid < nf) {
    float e = 0.0f;
#pragma unroll
    for (int q = 0; q < PCBA_MAX_SHARED; ++q)
      if (q == tid) e = em[q];
    eout[tid] = __fadd_ru(e, err[tid]);
    if (o64) o64[tid] = sO[tid];
    else o32[tid] = (float)sO[tid];
  }
}

// Shared memory of k_refresh (doubles): four patch buffers of cmax values,
// the matrices of lmax axes, their scratch, the box, offsets and reduction
// space.
__host__ __device__ constexpr size_t refresh_smem_doubles(int cmax, int lmax) {
  return 4 * (size_t)cmax + 2 * 289 * (size_t)lmax + (size_t)lmax * PCBA_KR_SCRATCH +
         2 * PCBA_MAXD + PCBA_MAX_SHARED + PCBA_MAX_SHARED * (PCBA_KRB / 32);
}

__global__ void __launch_bounds__(PCBA_KRB) k_refresh(Engine E, int cmax, int lmax) {
  extern __shared__ double krs[];
  // the list this step's subdivision filled (the loop control, which runs
  // beside this kernel, may already have counted the step)
  const int par = (int)E.plan->kr_par;
  const unsigned count = min(E.plan->mark_count[par], E.mark_cap);
  if (count == 0) return;
  const double* binom = c_binom;
  const int tid = threadIdx.x;
  double* sA = krs;
  double* sB = sA + cmax;
  float* sX = (float*)(sB + cmax);
  float* sY = (float*)(sB + 2 * cmax);
  double* sT = sB + 3 * cmax;
  double* scr = sT + 2 * 289 * lmax;
  double* box = scr + (size_t)lmax * PCBA_KR_SCRATCH;
  double* sO = box + 2 * PCBA_MAXD;
  float* red = (float*)(sO + PCBA_MAX_SHARED);  // 2 PCBA_MAX_SHARED x warps floats
  float err[PCBA_MAX_SHARED];
  const uint4* list = E.marks + (size_t)par * E.mark_cap;
  // marks are few (tens to thousands per step), each a chain of FP64 work:
  // one per block, consecutive marks on different SMs
  for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
    const uint4 m = list[q];  // (problem, child position, physical slot, family | patch << 2)
    const int p = (int)m.x, fam = (int)(m.w & 3u), ip = (int)(m.w >> 2);
    const ProbDesc* D = E.desc + p;
    const ProbState* S = E.state + p;
    const int slot = (int)m.y, l = D->l;
    if (slot >= S->child_twoK[par]) continue;
    const int nf = fam == PCBA_FAM_LIN ? D->alpha : 1;
    const int C = fam == 2 ? D->cp : (fam == 1 ? D->ch : D->cg);
    const int* deg = fam == 2 ? D->P : (fam == 1 ? D->H : D->G);
    if (nf * C > cmax) continue;
    char* item = E.arena + D->list_off + (size_t)m.z * D->item_bytes;
    if (tid < l) {
      const double w = ldexp(D->hi[tid] - D->lo[tid], -S->child_level[par][tid]);
      const unsigned idx = ((const unsigned*)item)[tid];
      box[tid] = D->lo[tid] + w * (double)idx;
      box[l + tid] = D->lo[tid] + w * (double)(idx + 1u);
    }
    __syncthreads();
    refresh_matrices(binom, l, deg, box, sT, scr);
    const double* mono = E.mono + D->mono_off;
    const double* a = fam == 2 ? mono
                               : mono + D->cp + (fam == 1 ? (long long)D->alpha * D->cg : 0) +
                                     (fam == PCBA_FAM_LIN ? 0 : (long long)ip * C);
    double *cA = sA, *cB = sB;
    float *cX = sX, *cY = sY;
    refresh_convert(a, nf, C, l, deg, sT, cA, cB, cX, cY, red, err);
    if (fam == 2) {
      // the cost patch, re-centred on its range
      refresh_store(cA, 1, C, err, (float*)(item + D->off_cost), 1, (float*)(item + 40),
                    (double*)(item + 32), nullptr, red, sO);
    } else if (fam == PCBA_FAM_LIN) {
      // every shared patch of a linear-family item, to the copy the next
      // step reads
      const int nxt = par ^ 1;
      float* earr = (float*)(item + D->off_eg + nxt * D->copy_e);
      refresh_store(cA, nf, C, err, (float*)(item + D->off_g + nxt * D->copy_g), D->apad, earr,
                    (double*)(earr + D->apad), nullptr, red, sO);
    } else {
      // one dense constraint patch, re-centred on an FP32 offset
      const size_t pad = fam ? D->bpad : D->apad;
      refresh_store(cA, 1, C, err, (float*)(item + (fam ? D->off_h : D->off_g)) + ip, pad,
                    (float*)(item + (fam ? D->off_eh : D->off_eg)) + ip, nullptr,
                    (float*)(item + (fam ? D->off_oh : D->off_og)) + ip, red, sO);
    }
    if (tid == 0) atomicAdd(&E.plan->refreshed_total, (unsigned long long)nf);
    __syncthreads();  // the buffers are reused by the next mark
  }
}

// rec_feasible on the keys (integer compares, no FP64): for a max-reduced
// field k (0 = nothing reduced, i.e. minus infinity), "value <= 0" holds
// exactly when k <= okey(+0.0) (both zeros included), and "value <= t" for
// t > 0 when k <= okey(t).  k_eq = okey(eq_tol).
__device__ __forceinline__ bool rec_feasible_key(const ChildRec& c, unsigned long long k_eq) {
  constexpr unsigned long long k0 = 0x8000000000000000ull;  // okey(+0.0)
  return c.gmaxmax <= k0 && c.hminmax <= k0 && c.hnegmaxmin <= k0 && c.habsmax <= k_eq;
}

// ---------------------------------------------------------------------------
// Def. 4: p_up over the feasible children, from the finished records
// ---------------------------------------------------------------------------
// Runs after the subdivision kernel, over the same child tiles as k3_classify:
// each warp reduces the pmax of its feasible children and one atomic min per
// warp lowers the problem's p_up key.
__device__ __forceinline__ void pup_phase(const Engine& E) {
  const unsigned tiles_total = E.plan->k3_tiles;
  const unsigned long long k_eq = okey(E.params->eq_tol);
  for (unsigned u = blockIdx.x; u < tiles_total; u += gridDim.x) {
    const int p = find_problem_warp(E.k3_pre, E.np, u, threadIdx.x & 31);
    const ProbDesc* D = E.desc + p;
    ProbState* S = E.state + p;
    const int twoK = 2 * S->K;
    const int c = (int)(u - E.k3_pre[p]) * PCBA_TPB + threadIdx.x;
    unsigned long long best = ~0ull, vbest = ~0ull;
    if (c < twoK) {
      const ChildRec* R = E.rec + D->slot_off + c;
      const ChildRec rc = load_rec_cg(R);
      if (rec_feasible_key(rc, k_eq)) best = rc.pmax;
      if (E.params->vertex) {
        // a corner at which every active constraint is certainly <= 0:
        // its cost bound, with the child and the corner
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (__ldcg(&R->vtxg[q]) > 0x80000000u) continue;  // okey32(+0.0)
          const unsigned long long key =
              ((unsigned long long)okey32(__ldcg(&R->vtxc[q])) << 32) | ((unsigned)c << 2) | q;
          vbest = key < vbest ? key : vbest;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
      best = other < best ? other : best;
      const unsigned long long vo = __shfl_xor_sync(0xffffffffu, vbest, o);
      vbest = vo < vbest ? vo : vbest;
    }
    if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&S->pup_key, best);
    if ((threadIdx.x & 31) == 0 && vbest != ~0ull) atomicMin(&S->vtx_key, vbest);
  }
}

__global__ void __launch_bounds__(PCBA_TPB) k_pup(Engine E) {
  pdl_begin();
  // the previous step's mark list: its refresh finished before this step's
  // subdivision began, and the next step's subdivision fills it again
  if (blockIdx.x == 0 && threadIdx.x == 0) E.plan->mark_count[(E.plan->steps_global & 1) ^ 1] = 0u;
  pup_phase(E);
}

// ---------------------------------------------------------------------------
// K3: classify, scan, finalize, plan
// ---------------------------------------------------------------------------
// The least certified corner cost of this step (vertex incumbents), +inf if none.
__device__ __forceinline__ double vertex_bound(unsigned long long vtx_key) {
  return vtx_key == ~0ull ? INFINITY : (double)okey32_dec((unsigned)(vtx_key >> 32));
}

__device__ void finalize_problem(const Engine& E, int p, unsigned* sscan) {
  const ProbDesc* D = E.desc + p;
  ProbState* S = E.state + p;
  const int twoK = 2 * S->K;
  const int ntiles = (twoK + PCBA_TPB - 1) / PCBA_TPB;
  unsigned* tc = E.tilecnt + D->tile_off;
  unsigned run = 0;
  for (int base = 0; base < ntiles; base += PCBA_TPB) {
    const int idx = base + threadIdx.x;
    const unsigned x = idx < ntiles ? __ldcg(tc + idx) : 0u;
    unsigned tot;
    const unsigned ex = block_exclusive_scan(x, sscan, &tot);
    if (idx < ntiles) tc[idx] = run + ex;
    run += tot;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  __threadfence();
  const SolveParams* P = E.params;
  const int K_save = (int)run;
  // every independent load first (the state, the returned box's slot, the
  // hole count's inputs), so that their latencies overlap; the stores follow
  const int l = D->l;
  const int r = S->r;
  const unsigned long long pup_key = S->pup_key, plo_key = S->plo_key, vkey = S->vtx_key;
  const double carry = S->p_up_carry;
  const unsigned long long bkey = S->best_key;
  const unsigned bs = bkey == ~0ull ? PCBA_NONE : (unsigned)(bkey >> 32);
  const int steps = S->steps, Kpar = S->K, ftop0 = S->ftop, hw0 = S->hw, nsweep = S->n;
  const long long peak = S->peak_items;
  const int trace_rows = D->trace_rows;
  const long long trace_off = D->trace_off, Mcap = D->M;
  const double opt_tol = P->opt_tol;
  const int max_iters = P->max_iters;
  const unsigned fr_ks = K_save < twoK ? __ldcg(E.flagrank + D->slot_off + K_save) : 0u;
  const unsigned tc_ks = K_save < twoK ? __ldcg(tc + K_save / PCBA_TPB) : 0u;
  const unsigned phys = bs != PCBA_NONE ? __ldcg(E.map + D->slot_off + bs) : 0u;
  // vertex incumbent: the child and corner of the least certified corner cost
  const double vtx = vertex_bound(vkey);
  const unsigned vslot = vkey == ~0ull ? PCBA_NONE : (unsigned)(vkey & 0xFFFFFFFFull) >> 2;
  const unsigned vphys = vslot != PCBA_NONE ? __ldcg(E.map + D->slot_off + vslot) : 0u;
  int level[PCBA_MAXD];
#pragma unroll
  for (int q = 0; q < PCBA_MAXD; ++q) level[q] = q < l ? S->level[q] : 0;
  unsigned bidx[PCBA_MAXD];
  if (bs != PCBA_NONE) {
    const unsigned* idx =
        (const unsigned*)(E.arena + D->list_off + (size_t)phys * D->item_bytes);
#pragma unroll
    for (int q = 0; q < PCBA_MAXD; ++q) bidx[q] = q < l ? __ldcg(idx + q) : 0u;
  }
  level[r] += 1;
  S->level[r] = level[r];
  const double p_up_step = okey_dec_min(pup_key);
  const double p_up = fmin(fmin(p_up_step, carry), vtx);
  if (bs == PCBA_NONE && vslot != PCBA_NONE && vtx < fmin(p_up_step, carry)) {
    // the corner is the incumbent: an exact point of the child's box
    const unsigned q = (unsigned)(vkey & 3ull);
    const unsigned* idx =
        (const unsigned*)(E.arena + D->list_off + (size_t)vphys * D->item_bytes);
    for (int a = 0; a < l; ++a) {
      const double w = ldexp(D->hi[a] - D->lo[a], -level[a]);
      const unsigned bit = (a < 2) ? ((q >> a) & 1u) : 0u;
      S->warm_x[a] = D->lo[a] + w * (double)(__ldcg(idx + a) + bit);
    }
    S->have_box = 0;
    S->from_warm = 1;
    S->p_up_carry = vtx;
    // the bound in the corner's cost: the child's cost-patch bound e_p (FP32)
    S->warm_err = E.precision == 32 ? (double)__ldcg((const float*)(idx) + 10) : 0.0;
  }
  if (bs != PCBA_NONE) {
    for (int q = 0; q < l; ++q) {
      S->best_index[q] = bidx[q];
      S->best_level[q] = level[q];
    }
    S->have_box = 1;
    S->from_warm = 0;
    S->p_up_carry = p_up_step;
    S->box_err = __uint_as_float((unsigned)(bkey & 0xFFFFFFFFull));
  }
  const double p_lo = okey_dec_min(plo_key);
  S->p_up = p_up;
  S->p_lo = p_lo;
  if (steps < trace_rows) {
    double* row = E.trace + (trace_off + steps) * 4;
    row[0] = (double)Kpar;
    row[1] = (double)K_save;
    row[2] = p_up;
    row[3] = p_lo;
  }
  S->steps = steps + 1;
  if ((long long)twoK > peak) S->peak_items = twoK;
  // free slots: this step popped K = twoK / 2 (stack first, then fresh slots);
  // k4_index pushes the slots of the twoK - K_save eliminated children
  {
    const int ftop1 = ftop0 > Kpar ? ftop0 - Kpar : 0;
    S->hw = hw0 + (Kpar > ftop0 ? Kpar - ftop0 : 0);
    S->ftop_push = ftop1;
    S->ftop = ftop1 + (twoK - K_save);
  }
  S->twoK = twoK;
  S->K_save = K_save;
  int status = PCBA_RUNNING;
  int F = 0;
  if (K_save == 0) {
    status = 1;  // INFEASIBLE (Alg. 1 line 8)
    S->K = twoK;
  } else if (p_up - p_lo <= opt_tol) {
    status = 0;  // OPTIMAL (Alg. 1 line 9)
    S->K = twoK;
  } else {
    // holes below K_save = K_save - (kept items below K_save)
    const unsigned grank = K_save < twoK ? tc_ks + (fr_ks & 0x7FFFFFFFu) : (unsigned)K_save;
    F = K_save - (int)grank;
    S->K = K_save;
    int rn = r + 1;
    int n_new = nsweep;
    if (rn == l) { rn = 0; n_new += 1; S->n = n_new; }
    S->r = rn;
    if (n_new >= max_iters) status = 3;                         // MAXITER (line 11)
    else if (level[rn] >= 31) status = 3;                       // 32-bit dyadic indices
    else if (2LL * K_save > Mcap) status = 2;                   // MEMCAP (line 4)
  }
  S->F = F;
  S->status = status;
  S->pup_key = ~0ull;
  S->plo_key = ~0ull;
  S->best_key = ~0ull;
  S->vtx_key = ~0ull;
  S->k3_arrive = 0u;
  if (status != PCBA_RUNNING) S->t_end = globaltimer();
}

__device__ void plan_next(const Engine& E, unsigned* sscan) {
  unsigned run2 = 0, run3 = 0, run4 = 0, runr = 0;
  for (int base = 0; base < E.np; base += PCBA_TPB) {
    const int p = base + threadIdx.x;
    unsigned a2 = 0, a3 = 0, a4 = 0, ar = 0;
    if (p < E.np) {
      ProbState* S = E.state + p;
      const ProbDesc* D = E.desc + p;
      const int st = *(volatile const int*)&S->status;
      const int K = *(volatile const int*)&S->K;
      const int F = *(volatile const int*)&S->F;
      const int steps = *(volatile const int*)&S->steps;
      if (st == PCBA_RUNNING) {
        a2 = (unsigned)K * (unsigned)D->tiles;
        ar = (unsigned)K;  // parent items (the linear split kernel's threads)
        a3 = (unsigned)((2 * K + PCBA_TPB - 1) / PCBA_TPB);
        (void)steps;
      }
      a4 = (unsigned)F * (unsigned)D->move_chunks;
    }
    unsigned t2, t3, t4, tr;
    const unsigned e2 = block_exclusive_scan(a2, sscan, &t2);
    const unsigned e3 = block_exclusive_scan(a3, sscan, &t3);
    const unsigned e4 = block_exclusive_scan(a4, sscan, &t4);
    const unsigned er = block_exclusive_scan(ar, sscan, &tr);
    if (p < E.np) {
      E.k2_pre[p] = run2 + e2;
      E.k3_pre_next[p] = run3 + e3;
      E.k4_pre[p] = run4 + e4;
      E.kr_pre[p] = runr + er;
    }
    run2 += t2;
    run3 += t3;
    run4 += t4;
    runr += tr;
  }
  if (threadIdx.x == 0) {
    E.k2_pre[E.np] = run2;
    E.k3_pre_next[E.np] = run3;
    E.k4_pre[E.np] = run4;
    E.kr_pre[E.np] = runr;
    E.plan->k2_units = run2;
    E.plan->k3_tiles_next = run3;
    E.plan->k4_units = run4;
    E.plan->kr_units = runr;
    E.plan->any_running = run2 > 0 ? 1 : 0;
    E.plan->k3_done = 0u;
    __threadfence();
  }
}

// block-wide minimum of two unsigned 64-bit values (sm: 16 entries); the
// result is valid in thread 0
__device__ __forceinline__ void block_min2_u64(unsigned long long& a, unsigned long long& b,
                                               unsigned long long* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long oa = __shfl_xor_sync(0xffffffffu, a, o);
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
    a = oa < a ? oa : a;
    b = ob < b ? ob : b;
  }
  if (lane == 0) {
    sm[2 * wid] = a;
    sm[2 * wid + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < PCBA_TPB / 32; ++w) {
      a = sm[2 * w] < a ? sm[2 * w] : a;
      b = sm[2 * w + 1] < b ? sm[2 * w + 1] : b;
    }
  __syncthreads();
}

__device__ __forceinline__ void classify_phase(const Engine& E, unsigned* sscan, double* sred,
                                               int& s_last, int& s_glast) {
  const unsigned tiles_total = E.plan->k3_tiles;
  const unsigned long long k_eq = okey(E.params->eq_tol);
  for (unsigned u = blockIdx.x; u < tiles_total; u += gridDim.x) {
    const int p = find_problem_warp(E.k3_pre, E.np, u, threadIdx.x & 31);
    const int tile = (int)(u - E.k3_pre[p]);
    const ProbDesc* D = E.desc + p;
    ProbState* S = E.state + p;
    const int twoK = 2 * S->K;
    const int ntiles = (twoK + PCBA_TPB - 1) / PCBA_TPB;
    const int c = tile * PCBA_TPB + threadIdx.x;
    const double p_up_step = okey_dec_min(S->pup_key);
    const double carry = S->p_up_carry;
    const double vtx = vertex_bound(S->vtx_key);
    const double p_up = fmin(fmin(p_up_step, carry), vtx);
    const unsigned long long k_pup = okey(p_up + 0.0);  // p_up = -0.0 becomes +0.0
    unsigned keep = 0;
    // least key of a kept child's pmin (the keys order like the values) and
    // least slot of a child that attains p_up: integer reductions, no FP64
    unsigned long long kmin = ~0ull;
    unsigned long long smin = ~0ull;
    ChildRec* R = E.rec + D->slot_off + c;
    if (c < twoK) {
      const ChildRec rc = load_rec_cg(R);
      // Def. 3 and the cut-off on the keys: "value > 0" for a max-reduced
      // field is key > okey(+0.0); pmin <= p_up is a key compare once a zero
      // p_up is taken as +0.0 (-0.0 <= +0.0 either way)
      constexpr unsigned long long k0 = 0x8000000000000000ull;  // okey(+0.0)
      const bool infeasible = rc.gminmax > k0 || rc.hminmax > k0 || rc.hnegmaxmin > k0;
      keep = (!infeasible && rc.pmin <= k_pup) ? 1u : 0u;
      if (keep) kmin = rc.pmin;
      if (p_up_step <= carry && p_up_step <= vtx && okey_dec(rc.pmax) == p_up_step &&
          rec_feasible_key(rc, k_eq))
        smin = ((unsigned long long)c << 32) | (rc.perr & 0xFFFFFFFFull);
    }
    unsigned cnt;
    const unsigned rank = block_exclusive_scan(keep, sscan, &cnt);
    if (c < twoK) E.flagrank[D->slot_off + c] = (keep << 31) | rank;
    block_min2_u64(kmin, smin, (unsigned long long*)sred);
    if (threadIdx.x == 0) {
      E.tilecnt[D->tile_off + tile] = cnt;
      if (kmin != ~0ull) atomicMin(&S->plo_key, kmin);
      if (smin != ~0ull) atomicMin(&S->best_key, smin);
      __threadfence();
      const unsigned old = atomicAdd(&S->k3_arrive, 1u);
      s_last = old == (unsigned)ntiles - 1;
    }
    __syncthreads();
    // the record back to the identity for the next step, after the fence
    // above (which need not wait for these stores: nothing in this kernel
    // reads the records again)
    if (c < twoK) {
      unsigned long long* w = (unsigned long long*)R;
#pragma unroll
      for (int q = 0; q < (int)(sizeof(ChildRec) / 8); ++q) w[q] = 0ull;
    }
    if (s_last) finalize_problem(E, p, sscan);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned g = atomicAdd(&E.plan->k3_done, 1u);
      s_glast = g == tiles_total - 1;
    }
    __syncthreads();
    if (s_glast) plan_next(E, sscan);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(PCBA_TPB) k3_classify(Engine E) {
  pdl_begin();
  __shared__ unsigned sscan[8];
  __shared__ double sred[8 * 2];
  __shared__ int s_last, s_glast;
  classify_phase(E, sscan, sred, s_last, s_glast);
}

// ---------------------------------------------------------------------------
// K4: Alg. 5 hole filling
// ---------------------------------------------------------------------------
__device__ __forceinline__ void index_phase(const Engine& E) {
  const unsigned tiles_total = E.plan->k3_tiles;
  for (unsigned u = blockIdx.x; u < tiles_total; u += gridDim.x) {
    const int p = find_problem_warp(E.k3_pre, E.np, u, threadIdx.x & 31);
    const ProbState* S = E.state + p;
    // a problem that stops at this step (MEMCAP, MAXITER) is still compacted
    // (its list is returned); only running problems recycle slots
    const bool running = S->status == PCBA_RUNNING;
    if (!running && S->F == 0) continue;
    const ProbDesc* D = E.desc + p;
    const int tile = (int)(u - E.k3_pre[p]);
    const int twoK = S->twoK, K_save = S->K_save;
    const int c = tile * PCBA_TPB + threadIdx.x;
    if (c >= twoK) continue;
    // (the child's slot is read with its flag, before it is known to be needed)
    const unsigned fr = E.flagrank[D->slot_off + c];
    const unsigned slot = E.map[D->slot_off + c];
    const int ftop_push = S->ftop_push;
    const unsigned keep = fr >> 31;
    const int grank = (int)(E.tilecnt[D->tile_off + tile] + (fr & 0x7FFFFFFFu));
    if (c < K_save && !keep) E.hole[D->slot_off + (c - grank)] = (unsigned)c;
    if (c >= K_save && keep) E.filler[D->slot_off + (K_save - 1 - grank)] = (unsigned)c;
    // the slot of an eliminated child goes back on the free stack (grank =
    // kept children before c, so c - grank eliminated ones precede it)
    if (running && !keep) E.fstack[D->slot_off + ftop_push + (c - grank)] = slot;
  }
}

__global__ void __launch_bounds__(PCBA_TPB) k4_index(Engine E) {
  pdl_begin();
  index_phase(E);
}

// Alg. 5 on the map: the j-th hole below K_save takes the slot of the item at
// save position K_save-1-j (reading R11); one thread per hole.
__device__ __forceinline__ void move_phase(const Engine& E, unsigned units) {
  const int lane = threadIdx.x & 31;
  // a warp's 32 consecutive units: its first unit's problem by a warp
  // search, and only when the units reach past that problem a second one
  // for the last unit and a per-lane search between the two
  for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x - lane); base < units;
       base += gridDim.x * blockDim.x) {
    const unsigned u = base + lane, ulast = min(units - 1u, base + 31u);
    const int p0 = find_problem_warp(E.k4_pre, E.np, base, lane);
    int p = p0;
    if (__ldg(E.k4_pre + p0 + 1) <= ulast) {
      const int p1 = find_problem_warp(E.k4_pre, E.np, ulast, lane);
      if (u < units) p = p0 + find_problem(E.k4_pre + p0, p1 - p0 + 1, u);
    }
    if (u >= units) continue;
    const ProbDesc* D = E.desc + p;
    const unsigned j = u - E.k4_pre[p];
    const unsigned h = E.hole[D->slot_off + j];
    const unsigned f = E.filler[D->slot_off + j];
    E.map[D->slot_off + h] = E.map[D->slot_off + f];
  }
}


// ---------------------------------------------------------------------------
// loop control, init, evaluation
// ---------------------------------------------------------------------------
// Runs once per loop iteration after the compaction: publishes the next
// step's K3 tile prefix, counts the step, applies the optional step limit and
// the hard guard, and sets the WHILE condition of the device loop.
__device__ __forceinline__ void control_phase(const Engine& E, cudaGraphConditionalHandle handle,
                                              int use_graph, int& s_code, int& s_run) {
  Plan* pl = E.plan;
  for (int q = threadIdx.x; q <= E.np; q += blockDim.x) E.k3_pre[q] = E.k3_pre_next[q];
  if (threadIdx.x == 0) {
    // the graph's loop body holds several iterations; those that run after
    // the loop's end have no classify tiles, do no work and are not steps
    const bool did = pl->k3_tiles > 0;
    pl->k3_tiles = pl->k3_tiles_next;
    // this step's marks (its refresh, which may still run, reads the same
    // count; k_pup of the next step clears the list once that is done)
    pl->marks_total += min(pl->mark_count[pl->steps_global & 1], E.mark_cap);
    pl->lin_next = 0u;
    pl->lin_next2 = 0u;
    pl->lin_qcount = 0u;
    if (did) pl->steps_global += 1;
    const int running = pl->any_running;
    const SolveParams* P = E.params;
    int code = 0;
    if (running && P->max_steps > 0 && pl->steps_global >= P->max_steps) code = 5;
    else if (running && P->time_limit_ns > 0ull && globaltimer() - pl->t0 >= P->time_limit_ns)
      code = 4;  // TIMEOUT: the time limit ran out between two steps
    else if (running && pl->steps_global >= P->step_guard) { code = PCBA_RUNNING + 1; pl->guard_hit = 1; }
    if (code) {
      // the plan was made for problems that are now stopped: leave the
      // iterations that may follow in the loop body nothing to do (each
      // copies the next step's tile count: it must stay zero too)
      pl->k2_units = 0u;
      pl->k3_tiles = 0u;
      pl->k3_tiles_next = 0u;
      pl->k4_units = 0u;
      pl->kr_units = 0u;
    }
    s_code = code;
    s_run = code ? 0 : running;
  }
  __syncthreads();
  if (s_code) {
    for (int q = threadIdx.x; q < E.np; q += blockDim.x) {
      ProbState* S = E.state + q;
      if (S->status == PCBA_RUNNING) {
        S->status = s_code;
        S->t_end = globaltimer();
      }
    }
  }
  // boxes of the children of the coming step, for k_refresh (by its
  // parity: the refresh of the step just done may still read its own)
  const int cpar = pl->steps_global & 1;
  for (int q = threadIdx.x; q < E.np; q += blockDim.x) {
    ProbState* S = E.state + q;
    for (int r = 0; r < PCBA_MAXD; ++r)
      S->child_level[cpar][r] = S->level[r] + (r == S->r ? 1 : 0);
    S->child_twoK[cpar] = 2 * S->K;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    pl->any_running = s_run;
    if (use_graph) cudaGraphSetConditional(handle, s_run ? 1u : 0u);
  }
}


// Alg. 5 on the slot map; the loop control runs beside it, in the block that
// takes the last ticket.
__global__ void __launch_bounds__(PCBA_TPB) k_move_control(Engine E,
                                                           cudaGraphConditionalHandle handle,
                                                           int use_graph) {
  pdl_begin();
  __shared__ int s_last, s_code, s_run;
  __shared__ unsigned s_units;
  // every block reads its part of the plan (this step's moves) before it
  // takes a ticket; the block with the last ticket runs the loop control,
  // which rewrites the plan but reads nothing the moves write, while the
  // other blocks move
  if (threadIdx.x == 0) {
    s_units = E.plan->k3_tiles > 0 ? E.plan->k4_units : 0u;  // no moves after the loop's end
    __threadfence();
    s_last = atomicAdd(&E.plan->k4_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  const unsigned units = s_units;
  if (s_last) {
    __threadfence();
    if (threadIdx.x == 0) E.plan->k4_done = 0u;
    control_phase(E, handle, use_graph, s_code, s_run);
  }
  move_phase(E, units);
}

__global__ void k_init(Engine E) {
  __shared__ unsigned sscan[8];
  unsigned run2 = 0, run3 = 0, runr = 0;
  for (int base = 0; base < E.np; base += PCBA_TPB) {
    const int p = base + threadIdx.x;
    unsigned a2 = 0, a3 = 0, ar = 0;
    if (p < E.np) {
      const ProbDesc* D = E.desc + p;
      ProbState* S = E.state + p;
      S->K = 1;
      S->twoK = 0;
      S->K_save = 0;
      S->F = 0;
      S->r = 0;
      S->n = 1;
      S->steps = 0;
      for (int q = 0; q < PCBA_MAXD; ++q) {
        S->level[q] = 0;
        S->best_index[q] = 0;
        S->best_level[q] = 0;
        S->child_level[0][q] = S->child_level[1][q] = q == 0 ? 1 : 0;
      }
      S->child_twoK[0] = S->child_twoK[1] = 2;
      S->ftop = 0;
      S->ftop_push = 0;
      S->hw = 1;
      E.map[D->slot_off] = 0u;
      S->best_key = ~0ull;
      S->vtx_key = ~0ull;
      S->box_err = 0.0f;
      S->k3_arrive = 0;
      S->have_box = 0;
      S->pup_key = ~0ull;
      S->plo_key = ~0ull;
      S->p_up = S->p_up_carry;
      S->p_lo = -INFINITY;
      S->peak_items = 1;
      S->t_end = 0;
      unsigned* idx = (unsigned*)(E.arena + D->list_off);
      for (int q = 0; q < D->l; ++q) idx[q] = 0u;
      // linear families: every constraint is active on the root box, whose
      // FP32 shared patches are stored relative to offsets 0
      if (D->lin && E.precision == 32)
        for (int q = 0; q < D->apad; ++q)
          ((double*)(E.arena + D->list_off + D->off_eg + 4LL * D->apad))[q] = 0.0;
      if (D->lin)
        *(unsigned long long*)(E.arena + D->list_off + D->off_sum) =
            D->lin_chunks >= 64 ? ~0ull : ((1ull << D->lin_chunks) - 1ull);
      unsigned* mw = (unsigned*)(E.arena + D->list_off + D->off_mask);
      for (int q = 0; q < D->mwords; ++q) {
        const int rem = D->nlin - 32 * q;
        mw[q] = rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
      }
      if (D->M < 2) {
        S->status = 2;  // MEMCAP before the first subdivision
        S->t_end = globaltimer();
      } else {
        S->status = PCBA_RUNNING;
        a2 = (unsigned)D->tiles;
        a3 = 1u;
        ar = 1u;
      }
    }
    unsigned t2, t3;
    const unsigned e2 = block_exclusive_scan(a2, sscan, &t2);
    const unsigned e3 = block_exclusive_scan(a3, sscan, &t3);
    unsigned tr;
    const unsigned er = block_exclusive_scan(ar, sscan, &tr);
    if (p < E.np) {
      E.k2_pre[p] = run2 + e2;
      E.k3_pre[p] = run3 + e3;
      E.k4_pre[p] = 0;
      E.kr_pre[p] = runr + er;
    }
    run2 += t2;
    run3 += t3;
    runr += tr;
  }
  if (threadIdx.x == 0) {
    E.k2_pre[E.np] = run2;
    E.k3_pre[E.np] = run3;
    E.k4_pre[E.np] = 0;
    Plan* pl = E.plan;
    pl->k2_units = run2;
    pl->k3_tiles = run3;
    pl->k3_tiles_next = 0;
    pl->k4_units = 0;
    pl->kr_units = runr;
    pl->mark_count[0] = 0u;
    pl->mark_count[1] = 0u;
    pl->kr_par = 0u;
    pl->marks_total = 0ull;
    pl->refreshed_total = 0ull;
    pl->lin_pairs = 0ull;
    pl->lin_full = 0ull;
    pl->lin_next = 0u;
    pl->lin_next2 = 0u;
    pl->lin_qcount = 0u;
    E.kr_pre[E.np] = runr;
    pl->k3_done = 0;
    pl->k4_done = 0u;
    pl->any_running = run2 > 0;
    pl->steps_global = 0;
    pl->guard_hit = 0;
  }
}

#include "pcba_eval.cuh"

