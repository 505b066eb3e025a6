// Kernels of one PCBA step (Algorithm 1) for many problems at once, plus the
// monomial-to-Bernstein conversion and the FP64 point check.
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
//   k4_index / k4_move        Alg. 5 (reading R11): the j-th hole below K_save
//                             receives the item at save position K_save-1-j.
//   k_control                 device-side loop control (graph conditional).
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

// FP32 error bounds are stored with a mark in the sign bit, set when the bound
// itself changes a decision of Def. 3 for this patch: the stored coefficients
// (min s, max s) would decide it (infeasible, feasible, or inside the
// equality window) but the enclosure [s_min - e, s_max + e] does not.  The
// magnitude is the bound; k_refresh recomputes marked patches.
__device__ __forceinline__ float mark_err(float e, float smin, float smax, float lo, float hi,
                                          int fam, float eqt) {
  // a refresh cannot go below about one rounding of the coefficients: leave
  // patches whose bound is already close to that floor
  if (e <= 8.0f * fmaxf(fabsf(smin), fabsf(smax)) * 0x1p-24f) return e;
  bool flip;
  if (fam == 0) {
    flip = (lo <= 0.0f && hi >= 0.0f) && (smin > 0.0f || smax < 0.0f);
  } else {
    const bool inf_e = lo > 0.0f || hi < 0.0f, inf_s = smin > 0.0f || smax < 0.0f;
    const bool win_e = lo >= -eqt && lo <= 0.0f && hi >= 0.0f && hi <= eqt;
    const bool win_s = smin >= -eqt && smin <= 0.0f && smax >= 0.0f && smax <= eqt;
    flip = inf_e != inf_s || win_e != win_s;
  }
  return flip ? -e : e;
}

// Where a marked patch lives: problem, the two child slots, and the list of
// the current step (steps alternate between two lists).
struct MarkCtx {
  int p, kL, kR;
  uint4* list;
  unsigned* count;
  unsigned cap;
};

// Warp-aggregated append of the marked children of this warp's patches
// (fam 0/1: constraint family, fam 2: the cost patch, ip = patch index).
__device__ __forceinline__ void append_marks(const MarkCtx& m, bool mL, bool mR, int fam, int ip) {
  const unsigned bl = __ballot_sync(0xffffffffu, mL), br = __ballot_sync(0xffffffffu, mR);
  if (!(bl | br)) return;
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(m.count, (unsigned)(__popc(bl) + __popc(br)));
  base = __shfl_sync(0xffffffffu, base, 0);
  const unsigned below = (1u << lane) - 1u;
  if (mL) {
    const unsigned q = base + __popc(bl & below);
    if (q < m.cap) m.list[q] = make_uint4((unsigned)m.p, (unsigned)m.kL, (unsigned)fam, (unsigned)ip);
  }
  if (mR) {
    const unsigned q = base + __popc(bl) + __popc(br & below);
    if (q < m.cap) m.list[q] = make_uint4((unsigned)m.p, (unsigned)m.kR, (unsigned)fam, (unsigned)ip);
  }
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
// head: where the parent's head bytes (box, meta, cost) are read from: the
// parent item itself, or a shared-memory copy of them.
template <typename T, int NMAX>
__device__ void cost_part(const ProbDesc* D, const char* head, char* parent, char* right, int r,
                          ChildRec* recL, ChildRec* recR, T* stage, const MarkCtx& mk,
                          double cost_thr) {
  const int lane = threadIdx.x & 31;
  const int cp = D->cp;
  const int n = D->P[r];
  const int stride = axis_stride(D->P, D->l, r);
  const int nf = cp / (n + 1);
  const int blk = (n + 1) * stride;
  const T* src = (const T*)(head + D->off_cost);
  T* dstL = (T*)(parent + D->off_cost);
  T* dstR = (T*)(right + D->off_cost);
  T* sL = stage;
  T* sR = stage + cp;
  double O = 0.0, ep = 0.0;
  if constexpr (sizeof(T) == 4) {
    O = *(const double*)(head + 32);
    ep = (double)*(const float*)(head + 40);
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
      dstL[j] = sL[j];
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
    float* fsrc = (float*)dstL;
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
    // the cost bound is refreshed once it is a visible part of opt_tol
    append_marks(mk, lane == 0 && efs[0] > cost_thr, lane == 0 && efs[1] > cost_thr, 2, 0);
  }
  __syncwarp();
}

// One warp's share (32 patches) of a tile of constraint patches of one family;
// the warp's maxima go to the child records with fire-and-forget atomics.
template <typename T, int NMAX>
__device__ void constraint_part(const ProbDesc* D, char* parent, char* right, int r, int fam,
                                int tt, ChildRec* recL, ChildRec* recR, float eqt,
                                const MarkCtx& mk) {
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
  bool mL = false, mR = false;
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
      const float ec = __fadd_ru(__fadd_ru(fabsf(ep[i]), __fmul_ru((float)a.m, fn * 0x1p-24f)),
                                 fn * 0x1p-149f);
      loL = __fsub_rd((float)a.minL, ec);
      hiL = __fadd_ru((float)a.maxL, ec);
      loR = __fsub_rd((float)a.minR, ec);
      hiR = __fadd_ru((float)a.maxR, ec);
      const float eL = mark_err(ec, (float)a.minL, (float)a.maxL, loL, hiL, fam, eqt);
      const float eR = mark_err(ec, (float)a.minR, (float)a.maxR, loR, hiR, fam, eqt);
      ep[i] = eL;
      er[i] = eR;
      mL = __float_as_uint(eL) >> 31;
      mR = __float_as_uint(eR) >> 31;
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
  if constexpr (RIG) append_marks(mk, mL, mR, fam, i);
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
// warp publishes its bound maxima with fire-and-forget atomics into the two
// child records; p_up is computed from the finished records by k_pup.
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
  const float eqt = __double2float_ru(E.params->eq_tol);
  const double cost_thr = E.params->opt_tol * (1.0 / 64.0);
  const int mpar = E.plan->steps_global & 1;
  const unsigned per = (units + gridDim.x - 1) / gridDim.x;
  const unsigned u0 = blockIdx.x * per;
  const unsigned u1 = min(units, u0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    const MarkCtx mk{p, k, k + K, E.marks + (size_t)mpar * E.mark_cap, &E.plan->mark_count[mpar],
                     E.mark_cap};
    if (t == 0 && warp == 0) {
      cost_part<T, NMAX>(D, parent, parent, right, r, recL, recR, (T*)k2stage, mk, cost_thr);
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
      constraint_part<T, NMAX>(D, parent, right, r, fam, tt, recL, recR, eqt, mk);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// K2 with TMA staging (sm_90+ bulk tensor copies; used on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits for phase 'parity' of a stage barrier; gives up after ~1 s (a copy that
// never lands), records it in the plan and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  Plan* plan) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (unsigned it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && globaltimer() - t0 > 1000000000ull) {
      atomicExch(&plan->guard_hit, 2);
      return false;
    }
  }
}

// Resolves a warp work unit u = (problem p, parent item k, column group g).
struct WarpUnit {
  int p, k, g, fam, x;
};
__device__ __forceinline__ WarpUnit resolve_unit(const Engine& E, unsigned u, int& p,
                                                 unsigned& pbeg, unsigned& pend) {
  if (u >= pend || u < pbeg) {
    p = find_problem(E.k2_pre, E.np, u);
    pbeg = E.k2_pre[p];
    pend = E.k2_pre[p + 1];
  }
  const ProbDesc* D = E.desc + p;
  const int groups = D->tiles;
  const unsigned local = u - pbeg;
  WarpUnit w;
  w.p = p;
  w.k = (int)(local / (unsigned)groups);
  w.g = (int)(local - (unsigned)w.k * groups);
  if (w.g < D->groups_g) {
    w.fam = 0;
    w.x = w.g * 32;
  } else if (w.g < D->groups_g + D->groups_h) {
    w.fam = 1;
    w.x = (w.g - D->groups_g) * 32;
  } else {
    w.fam = -1;  // cost-only unit of a problem without constraints
    w.x = 0;
  }
  return w;
}

// Lane 0 starts the copies of one unit into a stage: the [C][32] column block
// of the parent (one 3-D tensor copy) and, in FP32 mode, its 32 error bounds.
// Bytes of the item head (box, cost meta, cost patch) copied for group 0.
__device__ __forceinline__ unsigned head_bytes(const ProbDesc* D, unsigned w) {
  return (unsigned)((D->off_cost + (long long)D->cp * w + 15) / 16 * 16);
}

template <typename T>
__device__ __forceinline__ void issue_unit(const Engine& E, const WarpUnit& w, T* stage,
                                           float* estage, unsigned char* head,
                                           unsigned long long* bar) {
  const ProbDesc* D = E.desc + w.p;
  const char* item = E.arena + D->list_off + (size_t)w.k * D->item_bytes;
  const unsigned hb = w.g == 0 ? head_bytes(D, (unsigned)sizeof(T)) : 0u;
  if (w.fam < 0) {
    mbar_arrive_expect_tx(bar, hb);
    bulk_load(head, item, hb, bar);
    return;
  }
  const int C = w.fam ? D->ch : D->cg;
  unsigned bytes = (unsigned)C * 32u * (unsigned)sizeof(T) + hb;
  if (sizeof(T) == 4) bytes += 128u;
  mbar_arrive_expect_tx(bar, bytes);
  if (hb) bulk_load(head, item, hb, bar);
  const char* tm = (const char*)E.tmaps + ((size_t)w.p * 2 + w.fam) * 128;
  tma_load_3d(stage, tm, w.x, 0, w.k, bar);
  if (sizeof(T) == 4)
    bulk_load(estage, item + (w.fam ? D->off_eh : D->off_eg) + (size_t)w.x * 4, 128u, bar);
}

// Fibres of one column (lane) of a staged [C][32] block: loads from shared
// memory, children stored straight to global memory (coalesced across lanes).
template <typename T, int N, bool RIG>
__device__ __forceinline__ void staged_fibres(const T* stage, T* gL, T* gR, size_t pad, int C,
                                              int stride, int lane, FibAcc<T>& a) {
  const int nf = C / (N + 1);
  const int blk = (N + 1) * stride;
  const size_t st = (size_t)stride * pad;
#pragma unroll 1
  for (int f = 0; f < nf; ++f) {
    const int o = f / stride;
    const int c0 = o * blk + (f - o * stride);
    const T* sc = stage + c0 * 32 + lane;
    T* colL = gL + (size_t)c0 * pad;
    T* colR = gR + (size_t)c0 * pad;
    T q[N + 1];
#pragma unroll
    for (int j = 0; j <= N; ++j) q[j] = sc[j * stride * 32];
    if constexpr (RIG) {
#pragma unroll
      for (int j = 0; j <= N; ++j) a.m = fmax(a.m, fabs(q[j]));
    }
    // left_0 = f_0 already sits in the parent slot the left child overwrites
    colR[N * st] = q[N];
    a.minL = fmin(a.minL, q[0]);
    a.maxL = fmax(a.maxL, q[0]);
    a.minR = fmin(a.minR, q[N]);
    a.maxR = fmax(a.maxR, q[N]);
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

// The bound reductions of one warp's 32 patches, published with atomics
// (same quantities as constraint_part).
template <typename T>
__device__ __forceinline__ void publish_bounds(int fam, bool any_valid, T (&v)[6],
                                               ChildRec* recL, ChildRec* recR) {
  constexpr bool RIG = sizeof(T) == 4;
  const int lane = threadIdx.x & 31;
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
  if (lane == 0 && any_valid) {
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

// Work unit = (problem, parent item k, group g of 32 constraint patches); one
// warp per unit.  Every warp runs its own pipeline of 'stages' shared-memory
// stages: while it computes unit j, the copies of units j+1 .. j+stages-1 are
// in flight (TMA, completion on an mbarrier).  Group 0 also splits the cost
// patch and the box, whose bytes (box, meta, cost) come with the same copy.
// The kernel only streams: no fence and no value-returning atomic on the way.
template <typename T, int NMAX>
__global__ void __launch_bounds__(256) k2_subdivide_tma(Engine E, int stages, int stage_elems,
                                                        int cpmax) {
  constexpr bool RIG = sizeof(T) == 4;
  extern __shared__ __align__(128) unsigned char k2t_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  // per warp: stages x (stage_elems T + 32 floats + head), then 2*cpmax T of cost
  // staging; head = box, cost meta and cost patch of the parent (group 0)
  const size_t head_cap = ((size_t)64 + (size_t)cpmax * sizeof(T) + 127) / 128 * 128;
  const size_t stage_bytes = (size_t)stage_elems * sizeof(T) + 128 + head_cap;
  const size_t warp_bytes = (size_t)stages * stage_bytes + (size_t)2 * cpmax * sizeof(T);
  const size_t warp_bytes_al = (warp_bytes + 127) / 128 * 128;
  unsigned char* wb = k2t_smem + (size_t)warp * warp_bytes_al;
  unsigned long long* bars =
      (unsigned long long*)(k2t_smem + (size_t)wpb * warp_bytes_al) + (size_t)warp * stages;
  T* cost_stage = (T*)(wb + (size_t)stages * stage_bytes);
  if (lane == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
  fence_proxy_async_smem();
  const unsigned units = E.plan->k2_units;
  const float eqt = __double2float_ru(E.params->eq_tol);
  const double cost_thr = E.params->opt_tol * (1.0 / 64.0);
  const int mpar = E.plan->steps_global & 1;
  const unsigned per = (units + gridDim.x - 1) / gridDim.x;
  const unsigned u0 = blockIdx.x * per;
  const unsigned u1 = min(units, u0 + per);
  const unsigned first = u0 + warp;
  const int J = first < u1 ? (int)((u1 - first + wpb - 1) / wpb) : 0;
  int ip = -1, cp_ = -1;
  unsigned ibeg = 0, iend = 0, cbeg = 0, cend = 0;
  // prologue
  for (int j = 0; j < J && j < stages; ++j) {
    if (lane == 0) {
      const WarpUnit w = resolve_unit(E, first + (unsigned)j * wpb, ip, ibeg, iend);
      unsigned char* st = wb + (size_t)j * stage_bytes;
      issue_unit<T>(E, w, (T*)st, (float*)(st + (size_t)stage_elems * sizeof(T)),
                    st + (size_t)stage_elems * sizeof(T) + 128, &bars[j]);
    }
  }
  for (int j = 0; j < J; ++j) {
    const int s = j % stages;
    const unsigned parity = (unsigned)(j / stages) & 1u;
    unsigned char* st = wb + (size_t)s * stage_bytes;
    const T* stage = (const T*)st;
    const float* estage = (const float*)(st + (size_t)stage_elems * sizeof(T));
    const WarpUnit w = resolve_unit(E, first + (unsigned)j * wpb, cp_, cbeg, cend);
    const ProbDesc* D = E.desc + w.p;
    ProbState* S = E.state + w.p;
    const int K = S->K, r = S->r;
    char* parent = E.arena + D->list_off + (size_t)w.k * D->item_bytes;
    char* right = E.arena + D->list_off + (size_t)(w.k + K) * D->item_bytes;
    ChildRec* recL = E.rec + D->slot_off + w.k;
    ChildRec* recR = E.rec + D->slot_off + w.k + K;
    const MarkCtx mk{w.p, w.k, w.k + K, E.marks + (size_t)mpar * E.mark_cap,
                     &E.plan->mark_count[mpar], E.mark_cap};
    bool ok = true;
    if (lane == 0) ok = mbar_wait_bounded(&bars[s], parity, E.plan);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (!ok) {
      // copies did not land (recorded in the plan): wait, bounded, for the
      // copies still in flight into this warp's other stages, then leave
      if (lane == 0)
        for (int jj = j + 1; jj < J && jj < j + stages; ++jj)
          mbar_wait_bounded(&bars[jj % stages], (unsigned)(jj / stages) & 1u, E.plan);
      __syncwarp();
      return;
    }
    if (w.g == 0) {
      const unsigned char* head = st + (size_t)stage_elems * sizeof(T) + 128;
      cost_part<T, NMAX>(D, (const char*)head, parent, right, r, recL, recR, cost_stage, mk,
                         cost_thr);
      if (lane == 0) {
        const unsigned* iP = (const unsigned*)head;
        unsigned* iL = (unsigned*)parent;
        unsigned* iR = (unsigned*)right;
        for (int q = 0; q < D->l; ++q) {
          iL[q] = iP[q];
          iR[q] = iP[q];
        }
        iL[r] = 2u * iP[r];
        iR[r] = 2u * iP[r] + 1u;
      }
    }
    if (w.fam >= 0) {
      const int fam = w.fam;
      const int cnt = fam ? D->beta : D->alpha;
      const size_t pad = fam ? D->bpad : D->apad;
      const int* deg = fam ? D->H : D->G;
      const int C = fam ? D->ch : D->cg;
      const long long off = fam ? D->off_h : D->off_g;
      const int n = deg[r];
      const int stride = axis_stride(deg, D->l, r);
      const int i = w.x + lane;
      T v[6] = {T(-INFINITY), T(-INFINITY), T(-INFINITY), T(-INFINITY), T(-INFINITY), T(-INFINITY)};
      bool mL = false, mR = false;
      if (i < cnt) {
        FibAcc<T> a;
        a.minL = a.minR = T(INFINITY);
        a.maxL = a.maxR = T(-INFINITY);
        a.m = T(0);
        T* gL = (T*)(parent + off) + i;
        T* gR = (T*)(right + off) + i;
        dispatch_degree<NMAX>(n, [&](auto nc) {
          staged_fibres<T, decltype(nc)::value, RIG>(stage, gL, gR, pad, C, stride, lane, a);
        });
        T loL, hiL, loR, hiR;
        if constexpr (RIG) {
          const float fnn = (float)n;
          const float ec = __fadd_ru(__fadd_ru(fabsf(estage[lane]),
                                               __fmul_ru((float)a.m, fnn * 0x1p-24f)),
                                     fnn * 0x1p-149f);
          loL = __fsub_rd((float)a.minL, ec);
          hiL = __fadd_ru((float)a.maxL, ec);
          loR = __fsub_rd((float)a.minR, ec);
          hiR = __fadd_ru((float)a.maxR, ec);
          const float eL = mark_err(ec, (float)a.minL, (float)a.maxL, loL, hiL, fam, eqt);
          const float eR = mark_err(ec, (float)a.minR, (float)a.maxR, loR, hiR, fam, eqt);
          ((float*)(parent + (fam ? D->off_eh : D->off_eg)))[i] = eL;
          ((float*)(right + (fam ? D->off_eh : D->off_eg)))[i] = eR;
          mL = __float_as_uint(eL) >> 31;
          mR = __float_as_uint(eR) >> 31;
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
      if constexpr (RIG) append_marks(mk, mL, mR, fam, i);
      publish_bounds<T>(fam, w.x < cnt, v, recL, recR);
    }
    // the stage is free again: reuse it for unit j + stages
    __syncwarp();
    fence_proxy_async_smem();
    if (lane == 0 && j + stages < J) {
      const WarpUnit wn = resolve_unit(E, first + (unsigned)(j + stages) * wpb, ip, ibeg, iend);
      issue_unit<T>(E, wn, (T*)st, (float*)(st + (size_t)stage_elems * sizeof(T)),
                    st + (size_t)stage_elems * sizeof(T) + 128, &bars[s]);
    }
    __syncwarp();
  }
  // every issued unit was consumed above: no copy is in flight at exit
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
// k4_move moves items; the child boxes come from the state snapshot
// child_level, which those kernels do not change.
//
// One warp per marked patch; the per-axis matrices of the item's box are
// built in the warp's shared memory.
// Binomial coefficients C(n, k), n, k <= 16 (exact integers), and their
// rounded reciprocals, filled once by the library at start-up.
__constant__ double c_binom[17 * 17];
__constant__ double c_binom_inv[17 * 17];

// T_r[i][j] = sum_k C(i,k) C(j,k) / C(n,k) lo^(j-k) w^k (power basis on the
// box -> Bernstein basis), and A_r its absolute-value sum widened by 2^-40,
// which covers the few roundings of every term (the reciprocal included).
__device__ __forceinline__ void refresh_matrices(const double* binom, int l, const int* deg,
                                                 const double* blo, const double* bhi,
                                                 double* sT, int lane) {
  for (int r = 0; r < l; ++r) {
    const int n = deg[r];
    const double lo = blo[r], w = bhi[r] - blo[r];
    // powers lo^e and w^e (same products as dev_pow, kept in registers)
    double lp[17], wp[17];
    lp[0] = 1.0;
    wp[0] = 1.0;
#pragma unroll
    for (int e = 1; e < 17; ++e) {
      lp[e] = lp[e - 1] * lo;
      wp[e] = wp[e - 1] * w;
    }
    double* T = sT + r * 578;
    double* A = T + 289;
    for (int e = lane; e < (n + 1) * (n + 1); e += 32) {
      const int i = e / (n + 1), j = e - (e / (n + 1)) * (n + 1);
      double t = 0.0, ta = 0.0;
      const int kmax = i < j ? i : j;
      for (int k = 0; k <= kmax; ++k) {
        const double term = binom[i * 17 + k] * c_binom_inv[n * 17 + k] * binom[j * 17 + k] *
                            lp[j - k] * wp[k];
        t += term;
        ta += fabs(term);
      }
      T[e] = t;
      A[e] = ta * (1.0 + 0x1p-40);
    }
  }
  __syncwarp();
}

// Warp-cooperative conversion of one monomial tensor a (C coefficients,
// multi-degree deg) with the matrices in sT; result in *sA, bound base in *sX.
__device__ __forceinline__ double refresh_convert(const double* a, int C, int l, const int* deg,
                                                  const double* sT, double*& sA, double*& sB,
                                                  double*& sX, double*& sY, int lane) {
  for (int j = lane; j < C; j += 32) {
    const double v = a[j];
    sA[j] = v;
    sX[j] = fabs(v);
  }
  __syncwarp();
  double gterms = 0.0;
  for (int r = 0; r < l; ++r) {
    const int n = deg[r];
    int stride = 1;
    for (int q = r + 1; q < l; ++q) stride *= deg[q] + 1;
    const double* T = sT + r * 578;
    const double* A = T + 289;
    gterms += 4.0 * n + 8.0;
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
        s = fma(T[i * (n + 1) + j], src[j * stride], s);
        sx = __dadd_ru(sx, __dmul_ru(A[i * (n + 1) + j], srcx[j * stride]));
      }
      sB[o] = s;
      sY[o] = sx;
    }
    __syncwarp();
    double* t = sA; sA = sB; sB = t;
    t = sX; sX = sY; sY = t;
  }
  double amax = 0.0;
  for (int j = lane; j < C; j += 32) amax = fmax(amax, sX[j]);
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  return __dmul_ru(__dmul_ru(2.0 * gterms, 0x1p-53), amax);
}

__global__ void __launch_bounds__(128) k_refresh(Engine E, int cmax, int lmax) {
  extern __shared__ double krs[];
  const int par = E.plan->steps_global & 1;  // the list this step's subdivision filled
  const unsigned count = min(E.plan->mark_count[par], E.mark_cap);
  if (count == 0) return;
  const double* binom = c_binom;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  double* wbase = krs + (size_t)warp * (4 * cmax + 2 * 289 * lmax);
  double* sA = wbase;
  double* sB = sA + cmax;
  double* sX = sB + cmax;
  double* sY = sX + cmax;
  double* sT = sY + cmax;
  const uint4* list = E.marks + (size_t)par * E.mark_cap;
  for (unsigned q = blockIdx.x * wpb + warp; q < count; q += gridDim.x * wpb) {
    const uint4 m = list[q];
    const int p = (int)m.x, fam = (int)m.z, ip = (int)m.w;
    const ProbDesc* D = E.desc + p;
    const ProbState* S = E.state + p;
    const int slot = (int)m.y;
    if (slot >= S->child_twoK) continue;
    char* item = E.arena + D->list_off + (size_t)slot * D->item_bytes;
    double blo[PCBA_MAXD], bhi[PCBA_MAXD];
    for (int r = 0; r < D->l; ++r) {
      const double w = ldexp(D->hi[r] - D->lo[r], -S->child_level[r]);
      const unsigned idx = ((const unsigned*)item)[r];
      blo[r] = D->lo[r] + w * (double)idx;
      bhi[r] = D->lo[r] + w * (double)(idx + 1u);
    }
    const double* mono = E.mono + D->mono_off;
    if (fam == 2) {
      if (D->cp > cmax) continue;
      // the cost patch: recomputed and re-centred on its range
      refresh_matrices(binom, D->l, D->P, blo, bhi, sT, lane);
      const double err64 = refresh_convert(mono, D->cp, D->l, D->P, sT, sA, sB, sX, sY, lane);
      double bmin = INFINITY, bmax = -INFINITY;
      for (int j = lane; j < D->cp; j += 32) { bmin = fmin(bmin, sA[j]); bmax = fmax(bmax, sA[j]); }
      for (int o = 16; o > 0; o >>= 1) {
        bmin = fmin(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
      }
      const double O = 0.5 * (bmin + bmax);
      float* dst = (float*)(item + D->off_cost);
      double emax = 0.0;
      for (int j = lane; j < D->cp; j += 32) {
        const double d = sA[j] - O;
        const float sv = __double2float_rn(d);
        dst[j] = sv;
        emax = fmax(emax, __dadd_ru(fabs((double)sv - d), __dmul_ru(fabs(d), 0x1p-52)));
      }
      for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      if (lane == 0) {
        *(double*)(item + 32) = O;
        *(float*)(item + 40) = __double2float_ru(__dadd_ru(emax, err64));
        atomicAdd(&E.plan->refreshed_total, 1ull);
      }
      __syncwarp();
      continue;
    }
    const int C = fam ? D->ch : D->cg;
    if (C > cmax) continue;
    const int* deg = fam ? D->H : D->G;
    refresh_matrices(binom, D->l, deg, blo, bhi, sT, lane);
    const size_t pad = fam ? D->bpad : D->apad;
    float* block = (float*)(item + (fam ? D->off_h : D->off_g));
    float* earr = (float*)(item + (fam ? D->off_eh : D->off_eg));
    const double* fam_mono = mono + D->cp + (fam ? (long long)D->alpha * D->cg : 0);
    const double err64 =
        refresh_convert(fam_mono + (long long)ip * C, C, D->l, deg, sT, sA, sB, sX, sY, lane);
    double emax = 0.0;
    for (int j = lane; j < C; j += 32) {
      const float sv = __double2float_rn(sA[j]);
      block[(size_t)j * pad + ip] = sv;
      emax = fmax(emax, fabs((double)sv - sA[j]));
    }
    for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if (lane == 0) {
      earr[ip] = __double2float_ru(__dadd_ru(emax, err64));
      atomicAdd(&E.plan->refreshed_total, 1ull);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Def. 4: p_up over the feasible children, from the finished records
// ---------------------------------------------------------------------------
// Runs after the subdivision kernel, over the same child tiles as k3_classify:
// each warp reduces the pmax of its feasible children and one atomic min per
// warp lowers the problem's p_up key.
__global__ void __launch_bounds__(PCBA_TPB) k_pup(Engine E) {
  const unsigned tiles_total = E.plan->k3_tiles;
  const double eq_tol = E.params->eq_tol;
  for (unsigned u = blockIdx.x; u < tiles_total; u += gridDim.x) {
    const int p = find_problem(E.k3_pre, E.np, u);
    const ProbDesc* D = E.desc + p;
    ProbState* S = E.state + p;
    const int twoK = 2 * S->K;
    const int c = (int)(u - E.k3_pre[p]) * PCBA_TPB + threadIdx.x;
    unsigned long long best = ~0ull;
    if (c < twoK) {
      const ChildRec rc = load_rec_cg(E.rec + D->slot_off + c);
      if (rec_feasible(rc, eq_tol)) best = rc.pmax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
      best = other < best ? other : best;
    }
    if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&S->pup_key, best);
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
  unsigned run2 = 0, run3 = 0, run4 = 0, runr = 0;
  for (int base = 0; base < E.np; base += PCBA_TPB) {
    const int p = base + threadIdx.x;
    unsigned a2 = 0, a3 = 0, a4 = 0, ar = 0;
    if (p < E.np) {
      const ProbState* S = E.state + p;
      const ProbDesc* D = E.desc + p;
      const int st = *(volatile const int*)&S->status;
      const int K = *(volatile const int*)&S->K;
      const int F = *(volatile const int*)&S->F;
      const int steps = *(volatile const int*)&S->steps;
      if (st == PCBA_RUNNING) {
        a2 = (unsigned)K * (unsigned)D->tiles;
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
    // the refresh of this iteration consumed this step's list
    pl->marks_total += min(pl->mark_count[pl->steps_global & 1], E.mark_cap);
    pl->mark_count[pl->steps_global & 1] = 0u;
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
  // boxes of the children of the coming step, for k_refresh
  for (int q = threadIdx.x; q < E.np; q += blockDim.x) {
    ProbState* S = E.state + q;
    for (int r = 0; r < PCBA_MAXD; ++r) S->child_level[r] = S->level[r] + (r == S->r ? 1 : 0);
    S->child_twoK = 2 * S->K;
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
      for (int q = 0; q < PCBA_MAXD; ++q) {
        S->level[q] = 0;
        S->best_index[q] = 0;
        S->best_level[q] = 0;
        S->child_level[q] = q == 0 ? 1 : 0;
      }
      S->child_twoK = 2;
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
      E.kr_pre[p] = 0;
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
    pl->kr_units = 0;
    pl->mark_count[0] = 0u;
    pl->mark_count[1] = 0u;
    pl->marks_total = 0ull;
    pl->refreshed_total = 0ull;
    E.kr_pre[E.np] = 0;
    pl->k3_done = 0;
    pl->any_running = run2 > 0;
    pl->steps_global = 0;
    pl->guard_hit = 0;
  }
}

// mode 0: warm start.  Candidate points of problem p (E.n_warm of them, at
// most PCBA_MAX_CAND; FP32 coordinates) are ranked by an FP32 upper bound on
// their cost, then checked in that order, PCBA_EVAL_CHUNK at a time: every
// constraint in FP32 with a rigorous error bound (g_i + err <= 0,
// |h_j| + err <= eq_tol).  The first certified-feasible candidate in rank
// order (ties: lower index) is chosen and its cost bound recomputed in FP64
// (cost + err) becomes the carried p_up.  A candidate is dropped at its first
// violated bound, and the constraints that dropped earlier candidates (a
// small ring of "killers") are tried first: neighbouring candidates tend to
// fail on the same constraint.
// mode 1: final check of the returned point in FP64, written to results.
struct EvalOut {
  double cost, cost_err, max_g, max_abs_h;
  int ok;
};

// FP32 copy (round to nearest) of every monomial coefficient
__global__ void k_mono32(const double* mono, float* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(mono[i]);
}

#define PCBA_EVAL_CHUNK 8
#define PCBA_MAX_CAND 1024

// Nested Horner evaluation in FP32 of a dense monomial tensor (coefficients
// a = the FP64 ones rounded to nearest FP32, row-major, last axis fastest) at
// an FP32 point x, together with S >= sum |a_J| |x^J| (the same recursion on
// absolute values, rounded up).  Horner with a fused multiply-add perturbs
// each term by at most gamma_(2 dsum) relative over the nested levels
// (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 5.1), and the
// coefficient rounding adds one more unit roundoff.
template <int L>
struct HornerF32 {
  __device__ __forceinline__ static void eval(const float* a, const int* deg, const int* stride,
                                              const float* x, const float* ax, float& v,
                                              float& s) {
    v = 0.0f;
    s = 0.0f;
    for (int i = deg[0]; i >= 0; --i) {
      float vi, si;
      HornerF32<L - 1>::eval(a + i * stride[0], deg + 1, stride + 1, x + 1, ax + 1, vi, si);
      v = fmaf(v, x[0], vi);
      s = __fmaf_ru(s, ax[0], si);
    }
  }
};
template <>
struct HornerF32<1> {
  __device__ __forceinline__ static void eval(const float* a, const int* deg, const int*,
                                              const float* x, const float* ax, float& v,
                                              float& s) {
    v = 0.0f;
    s = 0.0f;
    for (int i = deg[0]; i >= 0; --i) {
      const float af = __ldg(a + i);
      v = fmaf(v, x[0], af);
      s = __fmaf_ru(s, ax[0], fabsf(af));
    }
  }
};

// Value and rigorous error bound: |v - p(x)| <= err, where p has the FP64
// coefficients.  err = 2 (2 dsum + l + 4) 2^-24 S, which is at least twice the
// relative bound above, plus (C + dsum) 2^-149 M with M = prod max(1, |x_r|)^N_r
// for the absolute errors of subnormal intermediate results.
template <int L>
__device__ __forceinline__ void horner_f32_l(const float* a, const int* deg, const float* xin,
                                             float* val, float* err) {
  int d[L], st[L];
  float x[L], ax[L];
  int C = 1, dsum = 0;
  float M = 1.0f;
#pragma unroll
  for (int r = L - 1; r >= 0; --r) {
    d[r] = deg[r];
    st[r] = C;
    C *= d[r] + 1;
    dsum += d[r];
    x[r] = xin[r];
    ax[r] = fabsf(x[r]);
    const float m = fmaxf(1.0f, ax[r]);
    for (int k = 0; k < d[r]; ++k) M = __fmul_ru(M, m);
  }
  float v, S;
  HornerF32<L>::eval(a, d, st, x, ax, v, S);
  *val = v;
  const float rel = __fmul_ru((float)(2 * (2 * dsum + L + 4)), 0x1p-24f);
  *err = __fadd_ru(__fmul_ru(rel, S), __fmul_ru(__fmul_ru((float)(C + dsum), 0x1p-149f), M));
}

__device__ __forceinline__ void horner_f32(const float* a, int l, const int* deg, const float* x,
                                           float* val, float* err) {
  switch (l) {
    case 1: horner_f32_l<1>(a, deg, x, val, err); break;
    case 2: horner_f32_l<2>(a, deg, x, val, err); break;
    case 3: horner_f32_l<3>(a, deg, x, val, err); break;
    case 4: horner_f32_l<4>(a, deg, x, val, err); break;
    case 5: horner_f32_l<5>(a, deg, x, val, err); break;
    case 6: horner_f32_l<6>(a, deg, x, val, err); break;
    case 7: horner_f32_l<7>(a, deg, x, val, err); break;
    default: horner_f32_l<8>(a, deg, x, val, err); break;
  }
}

// The same nested Horner scheme in FP64 on the FP64 coefficients at an FP64
// point: |v - p(x)| <= 2 (2 dsum + l + 2) 2^-53 S + (C + dsum) 2^-1074 M.
template <int L>
struct HornerF64 {
  __device__ __forceinline__ static void eval(const double* a, const int* deg, const int* stride,
                                              const double* x, const double* ax, double& v,
                                              double& s) {
    v = 0.0;
    s = 0.0;
    for (int i = deg[0]; i >= 0; --i) {
      double vi, si;
      HornerF64<L - 1>::eval(a + i * stride[0], deg + 1, stride + 1, x + 1, ax + 1, vi, si);
      v = fma(v, x[0], vi);
      s = __fma_ru(s, ax[0], si);
    }
  }
};
template <>
struct HornerF64<1> {
  __device__ __forceinline__ static void eval(const double* a, const int* deg, const int*,
                                              const double* x, const double* ax, double& v,
                                              double& s) {
    v = 0.0;
    s = 0.0;
    for (int i = deg[0]; i >= 0; --i) {
      const double ai = __ldg(a + i);
      v = fma(v, x[0], ai);
      s = __fma_ru(s, ax[0], fabs(ai));
    }
  }
};

template <int L>
__device__ __forceinline__ void horner_f64_l(const double* a, const int* deg, const double* xin,
                                             double* val, double* err) {
  int d[L], st[L];
  double x[L], ax[L];
  int C = 1, dsum = 0;
  double M = 1.0;
#pragma unroll
  for (int r = L - 1; r >= 0; --r) {
    d[r] = deg[r];
    st[r] = C;
    C *= d[r] + 1;
    dsum += d[r];
    x[r] = xin[r];
    ax[r] = fabs(x[r]);
    const double m = fmax(1.0, ax[r]);
    for (int k = 0; k < d[r]; ++k) M = __dmul_ru(M, m);
  }
  double v, S;
  HornerF64<L>::eval(a, d, st, x, ax, v, S);
  *val = v;
  const double rel = __dmul_ru((double)(2 * (2 * dsum + L + 2)), 0x1p-53);
  *err = __dadd_ru(__dmul_ru(rel, S), __dmul_ru(__dmul_ru((double)(C + dsum), 0x1p-1074), M));
}

__device__ __forceinline__ void horner_f64(const double* a, int l, const int* deg, const double* x,
                                           double* val, double* err) {
  switch (l) {
    case 1: horner_f64_l<1>(a, deg, x, val, err); break;
    case 2: horner_f64_l<2>(a, deg, x, val, err); break;
    case 3: horner_f64_l<3>(a, deg, x, val, err); break;
    case 4: horner_f64_l<4>(a, deg, x, val, err); break;
    case 5: horner_f64_l<5>(a, deg, x, val, err); break;
    case 6: horner_f64_l<6>(a, deg, x, val, err); break;
    case 7: horner_f64_l<7>(a, deg, x, val, err); break;
    default: horner_f64_l<8>(a, deg, x, val, err); break;
  }
}

// candidate c of problem p: mode 0 a warm-start row (NaN first coordinate:
// none), mode 1 the point the solve returns; false if there is none
__device__ __forceinline__ bool eval_candidate(const Engine& E, int mode, int p, int c, double* x) {
  const ProbDesc* D = E.desc + p;
  const ProbState* S = E.state + p;
  const int l = D->l;
  if (mode == 0) {
    const double* w = E.warm + ((long long)p * E.n_warm + c) * PCBA_MAXD;
    if (isnan(w[0])) return false;
    for (int q = 0; q < l; ++q) x[q] = (double)__double2float_rn(w[q]);  // FP32 coordinates
    return true;
  }
  if (S->have_box) {
    for (int q = 0; q < l; ++q) {
      const double w = ldexp(D->hi[q] - D->lo[q], -S->best_level[q]);
      const double blo = D->lo[q] + w * (double)S->best_index[q];
      const double bhi = D->lo[q] + w * (double)(S->best_index[q] + 1u);
      x[q] = 0.5 * (blo + bhi);
    }
    return true;
  }
  if (S->from_warm) {
    for (int q = 0; q < l; ++q) x[q] = S->warm_x[q];
    return true;
  }
  return false;
}

#define PCBA_KILLERS 32

__global__ void __launch_bounds__(PCBA_TPB) k_eval(Engine E, int mode, void* results) {
  __shared__ double s_key[PCBA_MAX_CAND];
  __shared__ int s_id[PCBA_MAX_CAND];
  __shared__ double sx[PCBA_EVAL_CHUNK][PCBA_MAXD];
  __shared__ float sxf[PCBA_EVAL_CHUNK][PCBA_MAXD];
  __shared__ unsigned long long s_max[2];
  __shared__ int s_has[PCBA_EVAL_CHUNK];
  __shared__ int s_viol[PCBA_EVAL_CHUNK];
  __shared__ int s_kill[PCBA_KILLERS];
  __shared__ unsigned s_nkill;
  __shared__ int s_done;
  const int p = blockIdx.x;
  const ProbDesc* D = E.desc + p;
  ProbState* S = E.state + p;
  const int l = D->l;
  const double* base = E.mono + D->mono_off;
  const int total = D->alpha + D->beta;

  if (mode == 1) {
    // final check of one point, FP64
    if (threadIdx.x == 0) {
      s_has[0] = eval_candidate(E, 1, p, 0, sx[0]) ? 1 : 0;
      s_max[0] = 0ull;
      s_max[1] = 0ull;
    }
    __syncthreads();
    EvalOut* o = (EvalOut*)results + p;
    if (!s_has[0]) {
      if (threadIdx.x == 0) {
        o->cost = NAN; o->cost_err = NAN; o->max_g = NAN; o->max_abs_h = NAN; o->ok = 0;
      }
      return;
    }
    for (int q = threadIdx.x; q < total; q += PCBA_TPB) {
      const bool is_g = q < D->alpha;
      const double* a = is_g ? base + D->cp + (long long)q * D->cg
                             : base + D->cp + (long long)D->alpha * D->cg +
                                   (long long)(q - D->alpha) * D->ch;
      double val, err;
      horner_f64(a, l, is_g ? D->G : D->H, sx[0], &val, &err);
      atomicMax(&s_max[is_g ? 0 : 1], okey(__dadd_ru(is_g ? val : fabs(val), err)));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double pc, pe;
      horner_f64(base, l, D->P, sx[0], &pc, &pe);
      o->cost = pc;
      o->cost_err = pe;
      o->max_g = okey_dec_max(s_max[0]);
      o->max_abs_h = okey_dec_max(s_max[1]);
      o->ok = 1;
    }
    return;
  }

  // ---- mode 0: rank the candidates by an FP32 bound on their cost
  const int n_c = E.warm ? min(E.n_warm, PCBA_MAX_CAND) : 0;
  const float* mono32 = E.mono32 + D->mono_off;
  int n2 = 1;
  while (n2 < n_c) n2 <<= 1;
  for (int c = threadIdx.x; c < n2; c += PCBA_TPB) {
    double key = INFINITY;
    double x[PCBA_MAXD];
    if (c < n_c && eval_candidate(E, 0, p, c, x)) {
      float xf[PCBA_MAXD];
      for (int q = 0; q < l; ++q) xf[q] = (float)x[q];
      float v, e;
      horner_f32(mono32, l, D->P, xf, &v, &e);
      const float k = __fadd_ru(v, e);
      if (!isnan(k)) key = (double)k;
    }
    s_key[c] = key;
    s_id[c] = c < n_c ? c : 0x7fffffff;
  }
  if (threadIdx.x == 0) {
    s_nkill = 0u;
    s_done = 0;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += PCBA_TPB) {
        const int o = i ^ j;
        if (o > i) {
          const bool gt = s_key[i] > s_key[o] || (s_key[i] == s_key[o] && s_id[i] > s_id[o]);
          if (gt == ((i & k) == 0)) {
            const double tk = s_key[i]; s_key[i] = s_key[o]; s_key[o] = tk;
            const int ti = s_id[i]; s_id[i] = s_id[o]; s_id[o] = ti;
          }
        }
      }
      __syncthreads();
    }

  // ---- check them in rank order
  const float eq_tol = (float)E.params->eq_tol;
  int chosen = -1;  // thread 0: chunk slot of the chosen candidate
  for (int c0 = 0; c0 < n_c; c0 += PCBA_EVAL_CHUNK) {
    const int nc = min(PCBA_EVAL_CHUNK, n_c - c0);
    if (threadIdx.x < PCBA_EVAL_CHUNK) {
      const int c = threadIdx.x;
      int has = 0;
      if (c < nc && s_key[c0 + c] < INFINITY)
        has = eval_candidate(E, 0, p, s_id[c0 + c], sx[c]) ? 1 : 0;
      s_has[c] = has;
      s_viol[c] = 0;
      if (has)
        for (int q = 0; q < l; ++q) sxf[c][q] = (float)sx[c][q];
    }
    __syncthreads();
    const int nk = (int)min(s_nkill, (unsigned)PCBA_KILLERS);
    if (nk > 0) {
      for (int it = threadIdx.x; it < nc * nk; it += PCBA_TPB) {
        const int c = it / nk;
        const int q = s_kill[it - c * nk];
        if (!s_has[c] || s_viol[c]) continue;
        const bool is_g = q < D->alpha;
        const float* a = is_g ? mono32 + D->cp + (long long)q * D->cg
                              : mono32 + D->cp + (long long)D->alpha * D->cg +
                                    (long long)(q - D->alpha) * D->ch;
        float val, err;
        horner_f32(a, l, is_g ? D->G : D->H, sxf[c], &val, &err);
        if (!(__fadd_ru(is_g ? val : fabsf(val), err) <= (is_g ? 0.0f : eq_tol))) s_viol[c] = 1;
      }
      __syncthreads();
    }
    for (int it = threadIdx.x; it < nc * total; it += PCBA_TPB) {
      const int c = it / total;
      const int q = it - c * total;
      if (!s_has[c] || s_viol[c]) continue;
      const bool is_g = q < D->alpha;
      const float* a = is_g ? mono32 + D->cp + (long long)q * D->cg
                            : mono32 + D->cp + (long long)D->alpha * D->cg +
                                  (long long)(q - D->alpha) * D->ch;
      float val, err;
      horner_f32(a, l, is_g ? D->G : D->H, sxf[c], &val, &err);
      if (!(__fadd_ru(is_g ? val : fabsf(val), err) <= (is_g ? 0.0f : eq_tol))) {
        s_viol[c] = 1;
        s_kill[atomicAdd(&s_nkill, 1u) % PCBA_KILLERS] = q;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int c = 0; c < nc; ++c)
        if (s_has[c] && !s_viol[c]) { chosen = c; break; }
      s_done = chosen >= 0 || (c0 + nc < n_c && !(s_key[c0 + nc] < INFINITY));
    }
    __syncthreads();
    if (s_done) break;
  }
  if (threadIdx.x == 0) {
    double offer = INFINITY;
    if (chosen >= 0) {
      double pc, pe;
      horner_f64(base, l, D->P, sx[chosen], &pc, &pe);
      offer = __dadd_ru(pc, pe);
      if (!(offer < INFINITY)) chosen = -1;
    }
    const int found = chosen >= 0;
    S->from_warm = found;
    S->p_up_carry = found ? offer : INFINITY;
    S->seeded = found;
    S->seed_cost = found ? offer : INFINITY;
    for (int q = 0; q < PCBA_MAXD; ++q) {
      const double v = (found && q < l) ? sx[chosen][q] : NAN;
      if (found && q < l) S->warm_x[q] = v;
      S->seed_x[q] = v;
    }
  }
}

// Cost of problem p on a G x G grid over its first two axes (G nodes when
// l = 1; other axes at the box centre), node (i, j) at
// x_0 = lo_0 + i (hi_0 - lo_0) / (G - 1), x_1 likewise with j; written as
// log(c - min over the grid + 1e-3) to out[p * ld + col0 + i * G + j] (floats).
__global__ void __launch_bounds__(PCBA_TPB) k_cost_grid(Engine E, int G, float* out, int ld,
                                                        int col0) {
  __shared__ double s_c[PCBA_MAX_CAND];
  __shared__ double red[PCBA_TPB / 32];
  const int p = blockIdx.x;
  const ProbDesc* D = E.desc + p;
  const int l = D->l;
  const int nodes = l >= 2 ? G * G : G;
  const double* base = E.mono + D->mono_off;
  double mn = INFINITY;
  for (int node = threadIdx.x; node < nodes; node += PCBA_TPB) {
    const int i = l >= 2 ? node / G : node, j = l >= 2 ? node - i * G : 0;
    double x[PCBA_MAXD];
    for (int q = 0; q < l; ++q) x[q] = 0.5 * (D->lo[q] + D->hi[q]);
    x[0] = D->lo[0] + (D->hi[0] - D->lo[0]) * (double)i / (double)(G - 1);
    if (l >= 2) x[1] = D->lo[1] + (D->hi[1] - D->lo[1]) * (double)j / (double)(G - 1);
    double c, e;
    horner_f64(base, l, D->P, x, &c, &e);
    s_c[node] = c;
    mn = fmin(mn, c);
  }
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
  __syncthreads();
  mn = red[0];
  for (int w = 1; w < PCBA_TPB / 32; ++w) mn = fmin(mn, red[w]);
  for (int node = threadIdx.x; node < nodes; node += PCBA_TPB)
    out[(long long)p * ld + col0 + node] = (float)log(s_c[node] - mn + 1e-3);
}

// Candidate points of guided solves: candidate c of problem p is the guess of
// p (normalised coordinates, guess_dim axes) plus stencil row c, clamped to
// [-1, 1] and mapped to the box; axes beyond guess_dim take the box centre.
__global__ void k_candidates(Engine E, const float* guess, int guess_dim, const double* stencil,
                             int n_stencil, double* cand) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)E.np * n_stencil) return;
  const int p = (int)(t / n_stencil), c = (int)(t - (long long)p * n_stencil);
  const ProbDesc* D = E.desc + p;
  double* o = cand + t * PCBA_MAXD;
  for (int r = 0; r < PCBA_MAXD; ++r) {
    double x = 0.0;
    if (r < D->l) {
      double u = 0.0;
      if (r < guess_dim)
        u = (double)guess[(long long)p * guess_dim + r] + stencil[(long long)c * guess_dim + r];
      u = fmin(fmax(u, -1.0), 1.0);
      x = D->lo[r] + 0.5 * (u + 1.0) * (D->hi[r] - D->lo[r]);
    }
    o[r] = x;
  }
}
