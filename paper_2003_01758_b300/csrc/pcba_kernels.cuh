// Kernels of one PCBA step (Algorithm 1) for many problems at once, plus the
// monomial-to-Bernstein conversion and the FP64 point check.
//
//   k1_matrices / k1_convert  Alg. 1 line 1 (InitPatches, Sec. II-D): per axis
//                             the matrix T_r = (power -> Bernstein on [0,1]) x
//                             (affine map [lo,hi] -> [0,1]), applied as l mode
//                             products to every monomial tensor, in FP64.
//   k2_subdivide              Alg. 2 + Alg. 3 + Def. 4: bisect every item in
//                             direction r (de Casteljau at 1/2 on every fibre,
//                             Sec. II-E), bound every child patch by the min and
//                             max of its coefficients (Thm. 1) and lower the
//                             solution estimate p_up with an atomic min.
//   k3_classify               Alg. 4 (readings R3-R5): keep = not infeasible
//                             (Def. 3) and not suboptimal (Def. 5); p_lo; scan of
//                             the keep flags; the last tile of each problem runs
//                             the stopping tests (Alg. 1 lines 4, 8, 9, 11) and
//                             the last tile overall plans the next step.
//   k4_index / k4_move        Alg. 5 (reading R11): the j-th hole below K_save
//                             receives the item at save position K_save-1-j.
//   k_control                 device-side loop control (graph conditional).
//   k_eval                    FP64 evaluation of p, g_i, h_j at a point with a
//                             rounding-error bound (warm start, final check).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "pcba_device.cuh"

// ---------------------------------------------------------------------------
// small exact helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dev_binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  if (k > n - k) k = n - k;
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
  return c;
}
__device__ __forceinline__ double dev_pow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

__device__ __forceinline__ float addrn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double addrn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mulrn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulrn(double a, double b) { return __dmul_rn(a, b); }

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
      double emax = 0.0;
      for (int j = lane; j < C; j += 32) {
        const float s = __double2float_rn(sA[j]);
        dst[(size_t)j * pad] = s;
        emax = fmax(emax, fabs((double)s - sA[j]));  // exact in double
      }
      for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      if (lane == 0)
        ((float*)(item0 + (fam == 1 ? D.off_eg : D.off_eh)))[idx] =
            __double2float_ru(__dadd_ru(emax, err64));
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
// K2: subdivide + bound + incumbent
// ---------------------------------------------------------------------------

// de Casteljau triangle at 1/2 on one fibre of N+1 coefficients (Sec. II-E):
// q^(0) = f, q_j^(k) = (q_j^(k-1) + q_{j+1}^(k-1)) / 2, left_i = q_0^(i),
// right_i = q_i^(N-i).  Round-to-nearest adds and exact halvings only.
template <typename T, int N>
__device__ __forceinline__ void split_fibre(T (&q)[N + 1], T (&L)[N + 1], T (&R)[N + 1]) {
  L[0] = q[0];
  R[N] = q[N];
#pragma unroll
  for (int k = 1; k <= N; ++k) {
#pragma unroll
    for (int j = 0; j <= N - k; ++j) q[j] = mulrn(addrn(q[j], q[j + 1]), T(0.5));
    L[k] = q[0];
    R[N - k] = q[N - k];
  }
}

template <typename T>
struct FibAcc {
  T minL, maxL, minR, maxR, m;
};

// Thread i walks every fibre of constraint patch i (column i of a
// coefficient-major [C][pad] block); the left child overwrites the parent.
// The de Casteljau triangle (see split_fibre) is evaluated in place: after
// level k, q[0] is left_k and q[N-k] is right_(N-k), and both are stored at
// once, so only the N+1 working values stay in registers.  Writing left_k over
// the parent's coefficient k is safe: it was loaded before the first level.
template <typename T, int N, bool RIG>
__device__ __forceinline__ void constraint_fibres(T* src, T* dR, size_t pad, int C, int stride,
                                                  int i, FibAcc<T>& a) {
  const int nf = C / (N + 1);
  const int blk = (N + 1) * stride;
  const size_t st = (size_t)stride * pad;
#pragma unroll 1
  for (int f = 0; f < nf; ++f) {
    const int o = f / stride;
    const int in = f - o * stride;
    T* colL = src + (size_t)(o * blk + in) * pad + i;
    T* colR = dR + (size_t)(o * blk + in) * pad + i;
    T q[N + 1];
#pragma unroll
    for (int j = 0; j <= N; ++j) q[j] = colL[j * st];
    if constexpr (RIG) {
#pragma unroll
      for (int j = 0; j <= N; ++j) a.m = fmax(a.m, fabs(q[j]));
    }
    colR[N * st] = q[N];
    a.minR = fmin(a.minR, q[N]);
    a.maxR = fmax(a.maxR, q[N]);
    a.minL = fmin(a.minL, q[0]);
    a.maxL = fmax(a.maxL, q[0]);
#pragma unroll
    for (int k = 1; k <= N; ++k) {
#pragma unroll
      for (int j = 0; j <= N - k; ++j) q[j] = mulrn(addrn(q[j], q[j + 1]), T(0.5));
      colL[k * st] = q[0];
      colR[(N - k) * st] = q[N - k];
      a.minL = fmin(a.minL, q[0]);
      a.maxL = fmax(a.maxL, q[0]);
      a.minR = fmin(a.minR, q[N - k]);
      a.maxR = fmax(a.maxR, q[N - k]);
    }
  }
}

// One cost fibre into shared staging buffers (same in-place triangle).
template <typename T, int N>
__device__ __forceinline__ void cost_fibre(const T* src, T* sL, T* sR, int base, int stride,
                                           double (&v)[5]) {
  T q[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    q[j] = src[base + j * stride];
    v[4] = fmax(v[4], (double)fabs(q[j]));
  }
  sL[base] = q[0];
  sR[base + N * stride] = q[N];
  v[0] = fmax(v[0], -(double)q[0]);
  v[1] = fmax(v[1], (double)q[0]);
  v[2] = fmax(v[2], -(double)q[N]);
  v[3] = fmax(v[3], (double)q[N]);
#pragma unroll
  for (int k = 1; k <= N; ++k) {
#pragma unroll
    for (int j = 0; j <= N - k; ++j) q[j] = mulrn(addrn(q[j], q[j + 1]), T(0.5));
    sL[base + k * stride] = q[0];
    sR[base + (N - k) * stride] = q[N - k];
    v[0] = fmax(v[0], -(double)q[0]);
    v[1] = fmax(v[1], (double)q[0]);
    v[2] = fmax(v[2], -(double)q[N - k]);
    v[3] = fmax(v[3], (double)q[N - k]);
  }
}

// Calls f(std::integral_constant<int, N>) for the runtime degree n, for
// N = 0..NMAX only: a kernel compiled for a smaller NMAX keeps fewer registers.
template <int NMAX, int N = 0, typename F>
__device__ __forceinline__ void dispatch_degree(int n, F&& f) {
  if constexpr (N <= NMAX) {
    if (n == N) {
      f(std::integral_constant<int, N>{});
      return;
    }
    dispatch_degree<NMAX, N + 1>(n, f);
  }
}

__device__ __forceinline__ int axis_stride(const int* deg, int l, int r) {
  int s = 1;
  for (int q = r + 1; q < l; ++q) s *= deg[q] + 1;
  return s;
}

// order-preserving 32-bit key of a float (0 = below everything)
__device__ __forceinline__ unsigned okey32(float x) {
  const unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float okey32_dec(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

template <int NV>
__device__ __forceinline__ void warp_max_d(double (&v)[NV]) {
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  }
}

// Cost patch of one parent, processed by one warp (tile 0, warp 0).
// FP64: children stored as computed.  FP32: each child is re-centred on the
// middle of its stored range, and its error bound grows by
//   n (m 2^-24 + 2^-149)          de Casteljau rounding, m = max |parent|,
//   half 2^-23 + 2^-149           re-centring, half = half the child's range,
//   |O'| 2^-52                    rounding of the new offset,
// all accumulated with upward rounding.
template <typename T, int NMAX>
__device__ void cost_part(const ProbDesc* D, char* parent, char* right, int r, ChildRec* recL,
                          ChildRec* recR, T* stage) {
  const int lane = threadIdx.x & 31;
  const int cp = D->cp;
  const int n = D->P[r];
  const int stride = axis_stride(D->P, D->l, r);
  const int nf = cp / (n + 1);
  const int blk = (n + 1) * stride;
  T* src = (T*)(parent + D->off_cost);
  T* dstR = (T*)(right + D->off_cost);
  T* sL = stage;
  T* sR = stage + cp;
  double O = 0.0, ep = 0.0;
  if constexpr (sizeof(T) == 4) {
    O = *(const double*)(parent + 32);
    ep = (double)*(const float*)(parent + 40);
  }
  double v[5] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
  for (int f = lane; f < nf; f += 32) {
    const int o = f / stride;
    const int base = o * blk + (f - o * stride);
    dispatch_degree<NMAX>(n, [&](auto nc) {
      cost_fibre<T, decltype(nc)::value>(src, sL, sR, base, stride, v);
    });
  }
  warp_max_d<5>(v);
  __syncwarp();
  const double minL = -v[0], maxL = v[1], minR = -v[2], maxR = v[3];
  if constexpr (sizeof(T) == 8) {
    for (int j = lane; j < cp; j += 32) {
      src[j] = sL[j];
      dstR[j] = sR[j];
    }
    if (lane == 0) {
      recL->pmin = okey(minL);
      recL->pmax = okey(maxL);
      recR->pmin = okey(minR);
      recR->pmax = okey(maxR);
    }
  } else {
    const float fn = (float)n;
    const float e1f = __fadd_ru(__fadd_ru((float)ep, __fmul_ru((float)v[4], fn * 0x1p-24f)),
                                fn * 0x1p-149f);
    const double e1 = (double)e1f;
    double mids[2], Os[2], efs[2], lows[2], highs[2];
    const double cmins[2] = {minL, minR}, cmaxs[2] = {maxL, maxR};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double mid = 0.5 * (cmins[c] + cmaxs[c]);  // exact
      const double half = __dsub_ru(cmaxs[c], mid);
      const double e2 = __dadd_ru(__dadd_ru(e1, __dmul_ru(half, 0x1p-23)), 0x1p-149);
      const double On = O + mid;
      const double e3 = __dadd_ru(e2, __dmul_ru(fabs(On), 0x1p-52));
      const float ef = __double2float_ru(e3);
      const double smin = (double)__double2float_rn(cmins[c] - mid);
      const double smax = (double)__double2float_rn(cmaxs[c] - mid);
      mids[c] = mid;
      Os[c] = On;
      efs[c] = (double)ef;
      lows[c] = __dsub_rd(__dadd_rd(On, smin), (double)ef);
      highs[c] = __dadd_ru(__dadd_ru(On, smax), (double)ef);
    }
    float* fsrc = (float*)src;
    float* fdst = (float*)dstR;
    const float* fL = (const float*)sL;
    const float* fR = (const float*)sR;
    for (int j = lane; j < cp; j += 32) {
      fsrc[j] = __double2float_rn((double)fL[j] - mids[0]);
      fdst[j] = __double2float_rn((double)fR[j] - mids[1]);
    }
    if (lane == 0) {
      *(double*)(parent + 32) = Os[0];
      *(float*)(parent + 40) = (float)efs[0];
      *(double*)(right + 32) = Os[1];
      *(float*)(right + 40) = (float)efs[1];
      recL->pmin = okey(lows[0]);
      recL->pmax = okey(highs[0]);
      recR->pmin = okey(lows[1]);
      recR->pmax = okey(highs[1]);
    }
  }
  __syncwarp();
}

// One warp's share (32 patches) of a tile of constraint patches of one family;
// the warp's maxima go to the child records with fire-and-forget atomics.
template <typename T, int NMAX>
__device__ void constraint_part(const ProbDesc* D, char* parent, char* right, int r, int fam,
                                int tt, ChildRec* recL, ChildRec* recR) {
  constexpr bool RIG = sizeof(T) == 4;
  const int lane = threadIdx.x & 31;
  const int i = tt * PCBA_TPB + threadIdx.x;
  const int cnt = fam ? D->beta : D->alpha;
  const size_t pad = fam ? D->bpad : D->apad;
  const int* deg = fam ? D->H : D->G;
  const int C = fam ? D->ch : D->cg;
  const long long off = fam ? D->off_h : D->off_g;
  T* src = (T*)(parent + off);
  T* dR = (T*)(right + off);
  const int n = deg[r];
  const int stride = axis_stride(deg, D->l, r);
  // reduced quantities of this thread (identity for masked lanes):
  //   fam 0: lo_L, hi_L, lo_R, hi_R;  fam 1: lo_L, -hi_L, |.|_L, lo_R, -hi_R, |.|_R
  T v[6] = {T(-INFINITY), T(-INFINITY), T(-INFINITY), T(-INFINITY), T(-INFINITY), T(-INFINITY)};
  if (i < cnt) {
    FibAcc<T> a;
    a.minL = a.minR = T(INFINITY);
    a.maxL = a.maxR = T(-INFINITY);
    a.m = T(0);
    dispatch_degree<NMAX>(n, [&](auto nc) {
      constraint_fibres<T, decltype(nc)::value, RIG>(src, dR, pad, C, stride, i, a);
    });
    T loL, hiL, loR, hiR;
    if constexpr (RIG) {
      float* ep = (float*)(parent + (fam ? D->off_eh : D->off_eg));
      float* er = (float*)(right + (fam ? D->off_eh : D->off_eg));
      const float fn = (float)n;
      const float ec = __fadd_ru(__fadd_ru(ep[i], __fmul_ru((float)a.m, fn * 0x1p-24f)),
                                 fn * 0x1p-149f);
      ep[i] = ec;
      er[i] = ec;
      loL = __fsub_rd((float)a.minL, ec);
      hiL = __fadd_ru((float)a.maxL, ec);
      loR = __fsub_rd((float)a.minR, ec);
      hiR = __fadd_ru((float)a.maxR, ec);
    } else {
      loL = a.minL;
      hiL = a.maxL;
      loR = a.minR;
      hiR = a.maxR;
    }
    if (fam == 0) {
      v[0] = loL; v[1] = hiL; v[2] = loR; v[3] = hiR;
    } else {
      v[0] = loL; v[1] = -hiL; v[2] = fmax(hiL, -loL);
      v[3] = loR; v[4] = -hiR; v[5] = fmax(hiR, -loR);
    }
  }
  const int nv = fam ? 6 : 4;
  double w[6];
  if constexpr (RIG) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const unsigned k = q < nv ? __reduce_max_sync(0xffffffffu, okey32(v[q])) : 0u;
      w[q] = (double)okey32_dec(k);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) w[q] = v[q];
    warp_max_d<6>(w);
  }
  const int base_lane_i = tt * PCBA_TPB + (threadIdx.x & ~31);
  if (lane == 0 && base_lane_i < cnt) {
    if (fam == 0) {
      atomicMax(&recL->gminmax, okey(w[0]));
      atomicMax(&recL->gmaxmax, okey(w[1]));
      atomicMax(&recR->gminmax, okey(w[2]));
      atomicMax(&recR->gmaxmax, okey(w[3]));
    } else {
      atomicMax(&recL->hminmax, okey(w[0]));
      atomicMax(&recL->hnegmaxmin, okey(w[1]));
      atomicMax(&recL->habsmax, okey(w[2]));
      atomicMax(&recR->hminmax, okey(w[3]));
      atomicMax(&recR->hnegmaxmin, okey(w[4]));
      atomicMax(&recR->habsmax, okey(w[5]));
    }
  }
}

// Def. 3 (a)-(b) on a finished record.
__device__ __forceinline__ bool rec_feasible(const ChildRec& c, double eq_tol) {
  const double gmaxmax = okey_dec_max(c.gmaxmax);
  const double hminmax = okey_dec_max(c.hminmax);
  const double hmaxmin = -okey_dec_max(c.hnegmaxmin);
  const double habsmax = okey_dec_max(c.habsmax);
  return gmaxmax <= 0.0 && hminmax <= 0.0 && hmaxmin >= 0.0 && habsmax <= eq_tol;
}

__device__ __forceinline__ ChildRec load_rec_cg(const ChildRec* p) {
  ChildRec c;
  const unsigned long long* s = (const unsigned long long*)p;
  c.pmin = __ldcg(s + 0);
  c.pmax = __ldcg(s + 1);
  c.gminmax = __ldcg(s + 2);
  c.gmaxmax = __ldcg(s + 3);
  c.hminmax = __ldcg(s + 4);
  c.hnegmaxmin = __ldcg(s + 5);
  c.habsmax = __ldcg(s + 6);
  c.pad = 0;
  return c;
}

// Work unit = (problem, parent item k, tile t).  Tile 0 also splits the cost
// patch (warp 0) and the box; every tile splits up to PCBA_TPB constraint
// patches, 32 per warp.  Warps never wait for each other inside a unit: each
// warp publishes its maxima with atomics and then counts itself in the item's
// arrival counter; the last of the tiles x 8 warps of an item to arrive reads
// the two complete child records and, for each feasible child, lowers p_up
// (Def. 4) with an atomic min.
//
// Each block takes one contiguous range of units, so consecutive units mostly
// belong to one problem; the problem's descriptor and step state are copied to
// shared memory once per problem.
template <typename T, int NMAX>
__global__ void __launch_bounds__(PCBA_TPB) k2_subdivide(Engine E) {
  extern __shared__ __align__(16) unsigned char k2stage[];
  __shared__ __align__(16) ProbDesc sD;
  __shared__ int sK, sR;
  const unsigned units = E.plan->k2_units;
  const double eq_tol = E.params->eq_tol;
  const unsigned per = (units + gridDim.x - 1) / gridDim.x;
  const unsigned u0 = blockIdx.x * per;
  const unsigned u1 = min(units, u0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr unsigned WARPS = PCBA_TPB / 32;
  int p = -1;
  unsigned pbeg = 0, pend = 0;
  for (unsigned u = u0; u < u1; ++u) {
    if (u >= pend) {
      p = find_problem(E.k2_pre, E.np, u);
      pbeg = E.k2_pre[p];
      pend = E.k2_pre[p + 1];
      __syncthreads();  // nobody still reads the previous descriptor
      const int* src = (const int*)(E.desc + p);
      int* dst = (int*)&sD;
      for (int q = threadIdx.x; q < (int)(sizeof(ProbDesc) / sizeof(int)); q += PCBA_TPB)
        dst[q] = src[q];
      if (threadIdx.x == 0) {
        sK = E.state[p].K;
        sR = E.state[p].r;
      }
      __syncthreads();
    }
    const ProbDesc* D = &sD;
    const int K = sK, r = sR, tiles = D->tiles;
    const unsigned local = u - pbeg;
    const int k = (int)(local / (unsigned)tiles);
    const int t = (int)(local - (unsigned)k * tiles);
    char* parent = E.arena + D->list_off + (size_t)k * D->item_bytes;
    char* right = E.arena + D->list_off + (size_t)(k + K) * D->item_bytes;
    ChildRec* recL = E.rec + D->slot_off + k;
    ChildRec* recR = E.rec + D->slot_off + k + K;
    if (t == 0 && warp == 0) {
      cost_part<T, NMAX>(D, parent, right, r, recL, recR, (T*)k2stage);
      if (lane == 0) {
        unsigned* iL = (unsigned*)parent;
        unsigned* iR = (unsigned*)right;
        for (int s = 0; s < D->l; ++s) iR[s] = iL[s];
        const unsigned v = iL[r];
        iL[r] = 2u * v;
        iR[r] = 2u * v + 1u;
      }
    }
    const int fam = t < D->tiles_g ? 0 : 1;
    const int tt = fam ? t - D->tiles_g : t;
    if (tt < (fam ? D->tiles_h : D->tiles_g))
      constraint_part<T, NMAX>(D, parent, right, r, fam, tt, recL, recR);
    if (lane == 0) {
      __threadfence();
      const unsigned old = atomicAdd(E.arrive + D->slot_off + k, 1u);
      if (old == (unsigned)tiles * WARPS - 1) {
        E.arrive[D->slot_off + k] = 0u;
        __threadfence();
        const ChildRec cl = load_rec_cg(recL);
        const ChildRec cr = load_rec_cg(recR);
        unsigned long long best = ~0ull;
        if (rec_feasible(cl, eq_tol)) best = cl.pmax;
        if (rec_feasible(cr, eq_tol) && cr.pmax < best) best = cr.pmax;
        if (best != ~0ull) atomicMin(&E.state[p].pup_key, best);
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// K3: classify, scan, finalize, plan
// ---------------------------------------------------------------------------
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
  const int l = D->l;
  const int r = S->r;
  S->level[r] += 1;
  const double p_up_step = okey_dec_min(S->pup_key);
  const double carry = S->p_up_carry;
  const double p_up = fmin(p_up_step, carry);
  const unsigned bs = S->best_slot;
  if (bs != PCBA_NONE) {
    const unsigned* idx = (const unsigned*)(E.arena + D->list_off + (size_t)bs * D->item_bytes);
    for (int q = 0; q < l; ++q) {
      S->best_index[q] = __ldcg(idx + q);
      S->best_level[q] = S->level[q];
    }
    S->have_box = 1;
    S->from_warm = 0;
    S->p_up_carry = p_up_step;
  }
  const double p_lo = okey_dec_min(S->plo_key);
  S->p_up = p_up;
  S->p_lo = p_lo;
  if (S->steps < D->trace_rows) {
    double* row = E.trace + (D->trace_off + S->steps) * 4;
    row[0] = (double)S->K;
    row[1] = (double)K_save;
    row[2] = p_up;
    row[3] = p_lo;
  }
  S->steps += 1;
  if ((long long)twoK > S->peak_items) S->peak_items = twoK;
  S->twoK = twoK;
  S->K_save = K_save;
  int status = PCBA_RUNNING;
  int F = 0;
  if (K_save == 0) {
    status = 1;  // INFEASIBLE (Alg. 1 line 8)
    S->K = twoK;
  } else if (p_up - p_lo <= P->opt_tol) {
    status = 0;  // OPTIMAL (Alg. 1 line 9)
    S->K = twoK;
  } else {
    // holes below K_save = K_save - (kept items below K_save)
    unsigned grank;
    if (K_save < twoK) {
      const unsigned fr = __ldcg(E.flagrank + D->slot_off + K_save);
      grank = __ldcg(tc + K_save / PCBA_TPB) + (fr & 0x7FFFFFFFu);
    } else {
      grank = (unsigned)K_save;
    }
    F = K_save - (int)grank;
    S->K = K_save;
    int rn = r + 1;
    if (rn == l) { rn = 0; S->n += 1; }
    S->r = rn;
    if (S->n >= P->max_iters) status = 3;                       // MAXITER (line 11)
    else if (S->level[rn] >= 31) status = 3;                    // 32-bit dyadic indices
    else if (2LL * K_save > D->M) status = 2;                   // MEMCAP (line 4)
  }
  S->F = F;
  S->status = status;
  S->pup_key = ~0ull;
  S->plo_key = ~0ull;
  S->best_slot = PCBA_NONE;
  S->k3_arrive = 0u;
  if (status != PCBA_RUNNING) S->t_end = globaltimer();
}

__device__ void plan_next(const Engine& E, unsigned* sscan) {
  unsigned run2 = 0, run3 = 0, run4 = 0;
  for (int base = 0; base < E.np; base += PCBA_TPB) {
    const int p = base + threadIdx.x;
    unsigned a2 = 0, a3 = 0, a4 = 0;
    if (p < E.np) {
      const ProbState* S = E.state + p;
      const ProbDesc* D = E.desc + p;
      const int st = *(volatile const int*)&S->status;
      const int K = *(volatile const int*)&S->K;
      const int F = *(volatile const int*)&S->F;
      if (st == PCBA_RUNNING) {
        a2 = (unsigned)K * (unsigned)D->tiles;
        a3 = (unsigned)((2 * K + PCBA_TPB - 1) / PCBA_TPB);
      }
      a4 = (unsigned)F * (unsigned)D->move_chunks;
    }
    unsigned t2, t3, t4;
    const unsigned e2 = block_exclusive_scan(a2, sscan, &t2);
    const unsigned e3 = block_exclusive_scan(a3, sscan, &t3);
    const unsigned e4 = block_exclusive_scan(a4, sscan, &t4);
    if (p < E.np) {
      E.k2_pre[p] = run2 + e2;
      E.k3_pre_next[p] = run3 + e3;
      E.k4_pre[p] = run4 + e4;
    }
    run2 += t2;
    run3 += t3;
    run4 += t4;
  }
  if (threadIdx.x == 0) {
    E.k2_pre[E.np] = run2;
    E.k3_pre_next[E.np] = run3;
    E.k4_pre[E.np] = run4;
    E.plan->k2_units = run2;
    E.plan->k3_tiles_next = run3;
    E.plan->k4_units = run4;
    E.plan->any_running = run2 > 0 ? 1 : 0;
    E.plan->k3_done = 0u;
    __threadfence();
  }
}

__global__ void __launch_bounds__(PCBA_TPB) k3_classify(Engine E) {
  __shared__ unsigned sscan[8];
  __shared__ double sred[8 * 2];
  __shared__ int s_last, s_glast;
  const unsigned tiles_total = E.plan->k3_tiles;
  const double eq_tol = E.params->eq_tol;
  for (unsigned u = blockIdx.x; u < tiles_total; u += gridDim.x) {
    const int p = find_problem(E.k3_pre, E.np, u);
    const int tile = (int)(u - E.k3_pre[p]);
    const ProbDesc* D = E.desc + p;
    ProbState* S = E.state + p;
    const int twoK = 2 * S->K;
    const int ntiles = (twoK + PCBA_TPB - 1) / PCBA_TPB;
    const int c = tile * PCBA_TPB + threadIdx.x;
    const double p_up_step = okey_dec_min(S->pup_key);
    const double carry = S->p_up_carry;
    const double p_up = fmin(p_up_step, carry);
    unsigned keep = 0;
    double v[2] = {-INFINITY, -INFINITY};  // -min kept pmin, -best slot
    if (c < twoK) {
      ChildRec* R = E.rec + D->slot_off + c;
      const ChildRec rc = load_rec_cg(R);
      unsigned long long* w = (unsigned long long*)R;
#pragma unroll
      for (int q = 0; q < 8; ++q) w[q] = 0ull;  // identity for the next step
      const double pmin = okey_dec(rc.pmin);
      const double pmax = okey_dec(rc.pmax);
      const double gminmax = okey_dec_max(rc.gminmax);
      const double hminmax = okey_dec_max(rc.hminmax);
      const double hmaxmin = -okey_dec_max(rc.hnegmaxmin);
      const bool infeasible = gminmax > 0.0 || hminmax > 0.0 || hmaxmin < 0.0;
      keep = (!infeasible && pmin <= p_up) ? 1u : 0u;
      if (keep) v[0] = -pmin;
      if (p_up_step <= carry && pmax == p_up_step && rec_feasible(rc, eq_tol)) v[1] = -(double)c;
    }
    unsigned cnt;
    const unsigned rank = block_exclusive_scan(keep, sscan, &cnt);
    if (c < twoK) E.flagrank[D->slot_off + c] = (keep << 31) | rank;
    block_max<2>(v, sred);
    if (threadIdx.x == 0) {
      E.tilecnt[D->tile_off + tile] = cnt;
      if (v[0] > -INFINITY) atomicMin(&S->plo_key, okey(-v[0]));
      if (v[1] > -INFINITY) atomicMin(&S->best_slot, (unsigned)(-v[1]));
      __threadfence();
      const unsigned old = atomicAdd(&S->k3_arrive, 1u);
      s_last = old == (unsigned)ntiles - 1;
    }
    __syncthreads();
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

// ---------------------------------------------------------------------------
// K4: Alg. 5 hole filling
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PCBA_TPB) k4_index(Engine E) {
  const unsigned tiles_total = E.plan->k3_tiles;
  for (unsigned u = blockIdx.x; u < tiles_total; u += gridDim.x) {
    const int p = find_problem(E.k3_pre, E.np, u);
    const ProbState* S = E.state + p;
    if (S->F == 0) continue;
    const ProbDesc* D = E.desc + p;
    const int tile = (int)(u - E.k3_pre[p]);
    const int twoK = S->twoK, K_save = S->K_save;
    const int c = tile * PCBA_TPB + threadIdx.x;
    if (c >= twoK) continue;
    const unsigned fr = E.flagrank[D->slot_off + c];
    const unsigned keep = fr >> 31;
    const int grank = (int)(E.tilecnt[D->tile_off + tile] + (fr & 0x7FFFFFFFu));
    if (c < K_save && !keep) E.hole[D->slot_off + (c - grank)] = (unsigned)c;
    if (c >= K_save && keep) E.filler[D->slot_off + (K_save - 1 - grank)] = (unsigned)c;
  }
}

__global__ void __launch_bounds__(PCBA_TPB) k4_move(Engine E) {
  const unsigned units = E.plan->k4_units;
  for (unsigned u = blockIdx.x; u < units; u += gridDim.x) {
    const int p = find_problem(E.k4_pre, E.np, u);
    const ProbDesc* D = E.desc + p;
    const unsigned local = u - E.k4_pre[p];
    const int chunks = D->move_chunks;
    const unsigned j = local / (unsigned)chunks;
    const int ch = (int)(local - j * (unsigned)chunks);
    const unsigned dst_slot = E.hole[D->slot_off + j];
    const unsigned src_slot = E.filler[D->slot_off + j];
    const long long n16 = D->item_bytes / 16;
    const long long per = (n16 + chunks - 1) / chunks;
    const long long b0 = (long long)ch * per;
    const long long b1 = b0 + per < n16 ? b0 + per : n16;
    const int4* s = (const int4*)(E.arena + D->list_off + (size_t)src_slot * D->item_bytes);
    int4* d = (int4*)(E.arena + D->list_off + (size_t)dst_slot * D->item_bytes);
    for (long long q = b0 + threadIdx.x; q < b1; q += PCBA_TPB) d[q] = __ldcs(s + q);
  }
}

// ---------------------------------------------------------------------------
// loop control, init, evaluation
// ---------------------------------------------------------------------------
// Runs once per loop iteration after the compaction: publishes the next
// step's K3 tile prefix, counts the step, applies the optional step limit and
// the hard guard, and sets the WHILE condition of the device loop.
__global__ void k_control(Engine E, cudaGraphConditionalHandle handle, int use_graph) {
  Plan* pl = E.plan;
  __shared__ int s_code, s_run;
  for (int q = threadIdx.x; q <= E.np; q += blockDim.x) E.k3_pre[q] = E.k3_pre_next[q];
  if (threadIdx.x == 0) {
    pl->k3_tiles = pl->k3_tiles_next;
    pl->steps_global += 1;
    const int running = pl->any_running;
    const SolveParams* P = E.params;
    int code = 0;
    if (running && P->max_steps > 0 && pl->steps_global >= P->max_steps) code = 5;
    else if (running && pl->steps_global >= P->step_guard) { code = PCBA_RUNNING + 1; pl->guard_hit = 1; }
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
  __syncthreads();
  if (threadIdx.x == 0) {
    pl->any_running = s_run;
    if (use_graph) cudaGraphSetConditional(handle, s_run ? 1u : 0u);
  }
}

__global__ void k_init(Engine E) {
  __shared__ unsigned sscan[8];
  unsigned run2 = 0, run3 = 0;
  for (int base = 0; base < E.np; base += PCBA_TPB) {
    const int p = base + threadIdx.x;
    unsigned a2 = 0, a3 = 0;
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
      for (int q = 0; q < PCBA_MAXD; ++q) { S->level[q] = 0; S->best_index[q] = 0; S->best_level[q] = 0; }
      S->best_slot = PCBA_NONE;
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
      if (D->M < 2) {
        S->status = 2;  // MEMCAP before the first subdivision
        S->t_end = globaltimer();
      } else {
        S->status = PCBA_RUNNING;
        a2 = (unsigned)D->tiles;
        a3 = 1u;
      }
    }
    unsigned t2, t3;
    const unsigned e2 = block_exclusive_scan(a2, sscan, &t2);
    const unsigned e3 = block_exclusive_scan(a3, sscan, &t3);
    if (p < E.np) {
      E.k2_pre[p] = run2 + e2;
      E.k3_pre[p] = run3 + e3;
      E.k4_pre[p] = 0;
    }
    run2 += t2;
    run3 += t3;
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
    pl->k3_done = 0;
    pl->any_running = run2 > 0;
    pl->steps_global = 0;
    pl->guard_hit = 0;
  }
}

// FP64 value of a dense monomial tensor at x (powers in spw[r * 17 + j]) and
// a bound on its rounding error: gamma_(C + d + l + 2) * sum |a_J x^J|.
__device__ __forceinline__ void eval_mono(const double* a, int l, const int* deg, int C,
                                          const double* spw, double* val, double* err) {
  double s = 0.0, sa = 0.0;
  int dsum = 0;
  for (int r = 0; r < l; ++r) dsum += deg[r];
  for (int idx = 0; idx < C; ++idx) {
    int rem = idx;
    double prod = a[idx];
    for (int r = l - 1; r >= 0; --r) {
      const int d1 = deg[r] + 1;
      const int j = rem % d1;
      rem /= d1;
      prod *= spw[r * 17 + j];
    }
    s += prod;
    sa += fabs(prod);
  }
  *val = s;
  *err = __dmul_ru(__dmul_ru(2.0 * (double)(C + dsum + l + 2), 0x1p-53), sa);
}

// mode 0: warm start.  If the point of problem p is certified feasible
// (g_i + err <= 0, |h_j| + err <= eq_tol) its cost + err becomes the carried
// incumbent.  mode 1: final check of the returned point, written to out.
struct EvalOut {
  double cost, cost_err, max_g, max_abs_h;
  int ok;
};

__global__ void __launch_bounds__(PCBA_TPB) k_eval(Engine E, int mode, void* results) {
  __shared__ double spw[PCBA_MAXD * 17];
  __shared__ double sx[PCBA_MAXD];
  __shared__ double red[8 * 2];
  __shared__ int s_has;
  const int p = blockIdx.x;
  const ProbDesc* D = E.desc + p;
  ProbState* S = E.state + p;
  const int l = D->l;
  if (threadIdx.x == 0) {
    s_has = 0;
    if (mode == 0) {
      if (E.warm && !isnan(E.warm[p * PCBA_MAXD])) {
        s_has = 1;
        for (int q = 0; q < l; ++q) sx[q] = E.warm[p * PCBA_MAXD + q];
      }
    } else {
      if (S->have_box) {
        s_has = 1;
        for (int q = 0; q < l; ++q) {
          const double w = ldexp(D->hi[q] - D->lo[q], -S->best_level[q]);
          const double blo = D->lo[q] + w * (double)S->best_index[q];
          const double bhi = D->lo[q] + w * (double)(S->best_index[q] + 1u);
          sx[q] = 0.5 * (blo + bhi);
        }
      } else if (S->from_warm) {
        s_has = 1;
        for (int q = 0; q < l; ++q) sx[q] = S->warm_x[q];
      }
    }
    if (s_has)
      for (int q = 0; q < l; ++q) {
        double pw = 1.0;
        for (int j = 0; j < 17; ++j) { spw[q * 17 + j] = pw; pw *= sx[q]; }
      }
  }
  __syncthreads();
  if (!s_has) {
    if (mode == 0 && threadIdx.x == 0) { S->p_up_carry = INFINITY; S->from_warm = 0; }
    if (mode == 1 && threadIdx.x == 0) {
      EvalOut* o = (EvalOut*)results + p;
      o->cost = NAN; o->cost_err = NAN; o->max_g = NAN; o->max_abs_h = NAN; o->ok = 0;
    }
    return;
  }
  const double* base = E.mono + D->mono_off;
  double v[2] = {-INFINITY, -INFINITY};
  const int total = D->alpha + D->beta;
  for (int q = threadIdx.x; q < total; q += PCBA_TPB) {
    double val, err;
    if (q < D->alpha) {
      eval_mono(base + D->cp + (long long)q * D->cg, l, D->G, D->cg, spw, &val, &err);
      v[0] = fmax(v[0], __dadd_ru(val, err));
    } else {
      const int j = q - D->alpha;
      eval_mono(base + D->cp + (long long)D->alpha * D->cg + (long long)j * D->ch, l, D->H, D->ch,
                spw, &val, &err);
      v[1] = fmax(v[1], __dadd_ru(fabs(val), err));
    }
  }
  block_max<2>(v, red);
  if (threadIdx.x == 0) {
    double pc, pe;
    eval_mono(base, l, D->P, D->cp, spw, &pc, &pe);
    if (mode == 0) {
      const bool ok = v[0] <= 0.0 && v[1] <= E.params->eq_tol;
      S->from_warm = ok ? 1 : 0;
      S->p_up_carry = ok ? __dadd_ru(pc, pe) : INFINITY;
      for (int q = 0; q < l; ++q) S->warm_x[q] = sx[q];
    } else {
      EvalOut* o = (EvalOut*)results + p;
      o->cost = pc;
      o->cost_err = pe;
      o->max_g = v[0];
      o->max_abs_h = v[1];
      o->ok = 1;
    }
  }
}
