// Point evaluation kernels of libpcba (sm_103a): the warm start (candidate
// points certified feasible in FP32 seed the incumbent p_up of Def. 4), the
// final FP64 check of the returned point (Alg. 1 line 12), and the helpers of
// the learned warm start (candidate stencil, FP32 monomials, cost grid).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "pcba_device.cuh"

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

// FP32 copy (round to nearest) of the linear-family constraint rows
// FP32 pairs of the linear rows: x = hi + lo to 2^-48 relative (x - hi is
// exact in FP64, lo its rounding to nearest FP32).
__global__ void k_rows32(const double* rows, float* out, long long nrows) {
  const long long n = nrows * PCBA_LIN_STRIDE;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / PCBA_LIN_STRIDE, j = i - q * PCBA_LIN_STRIDE;
    const double x = rows[i];
    const float hi = __double2float_rn(x);
    out[q * PCBA_LIN32_STRIDE + j] = hi;
    out[q * PCBA_LIN32_STRIDE + PCBA_LIN_STRIDE + j] = __double2float_rn(x - (double)hi);
  }
}

// Packed rows (w = 1 + K doubles each) to the padded FP64 layout
// (PCBA_LIN_STRIDE doubles, zeros after the first w).
__global__ void k_rows_unpack(const double* packed, double* rows, long long nrows, int w) {
  const long long n = nrows * PCBA_LIN_STRIDE;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / PCBA_LIN_STRIDE, j = i - q * PCBA_LIN_STRIDE;
    rows[i] = j < w ? packed[q * w + j] : 0.0;
  }
}

#define PCBA_EVAL_CHUNK 8
#define PCBA_MAX_CAND 1024
#define PCBA_CAND_TPB 512  // threads of k_cand_first

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
      const float af = a[i];
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

// horner_f32 for l = 2 and degree (N, N) known at compile time: the same
// operations in the same order (so the same value and bound, bit for bit),
// with the loops unrolled so that the coefficient loads are not each waited
// for in turn.
template <int N>
__device__ __forceinline__ void horner_f32_sq2(const float* a, const float* xin, float* val,
                                               float* err) {
  const float x0 = xin[0], x1 = xin[1];
  const float ax0 = fabsf(x0), ax1 = fabsf(x1);
  float M = 1.0f;
  const float m1 = fmaxf(1.0f, ax1), m0 = fmaxf(1.0f, ax0);
#pragma unroll
  for (int k = 0; k < N; ++k) M = __fmul_ru(M, m1);
#pragma unroll
  for (int k = 0; k < N; ++k) M = __fmul_ru(M, m0);
  float c[(N + 1) * (N + 1)];
#pragma unroll
  for (int j = 0; j < (N + 1) * (N + 1); ++j) c[j] = a[j];
  float v = 0.0f, S = 0.0f;
#pragma unroll
  for (int i = N; i >= 0; --i) {
    float vi = 0.0f, si = 0.0f;
#pragma unroll
    for (int j = N; j >= 0; --j) {
      const float af = c[i * (N + 1) + j];
      vi = fmaf(vi, x1, af);
      si = __fmaf_ru(si, ax1, fabsf(af));
    }
    v = fmaf(v, x0, vi);
    S = __fmaf_ru(S, ax0, si);
  }
  *val = v;
  constexpr int dsum = 2 * N, C = (N + 1) * (N + 1);
  const float rel = __fmul_ru((float)(2 * (2 * dsum + 2 + 4)), 0x1p-24f);
  *err = __fadd_ru(__fmul_ru(rel, S), __fmul_ru(__fmul_ru((float)(C + dsum), 0x1p-149f), M));
}

// horner_f32, with the unrolled form for l = 2 and equal degrees up to 8
__device__ __forceinline__ void horner_f32_any(const float* a, int l, const int* deg,
                                               const float* x, float* val, float* err) {
  if (l == 2 && deg[0] == deg[1]) {
    switch (deg[0]) {
      case 2: horner_f32_sq2<2>(a, x, val, err); return;
      case 3: horner_f32_sq2<3>(a, x, val, err); return;
      case 4: horner_f32_sq2<4>(a, x, val, err); return;
      case 6: horner_f32_sq2<6>(a, x, val, err); return;
      case 8: horner_f32_sq2<8>(a, x, val, err); return;
      default: break;
    }
  }
  horner_f32(a, l, deg, x, val, err);
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

// Linear families (pcba_create_linear): inequality q is g_q = c_q + sum_m
// w_qm s_m.  From the shared polynomials' values sv[m] at a point, each with
// |sv[m] - s_m(x)| <= se[m]:
//   FP32 (rows rounded to nearest FP32): the fused chain has K roundings and
//   the rows one each, so with A = |c| + sum |w_m| |sv_m|,
//     |val - g_q(x)| <= (2K + 2) 2^-24 A + (1 + 2^-20) sum |w_m| se_m + (2K + 2) 2^-149;
//   FP64 (exact rows): K roundings,
//     |val - g_q(x)| <= (K + 1) 2^-53 A + (1 + 2^-50) sum |w_m| se_m + (K + 1) 2^-1074.
__device__ __forceinline__ void lin_value_f32(const Engine& E, const ProbDesc* D, int q,
                                              const float* sv, const float* se, float* val,
                                              float* err) {
  const float* row = E.lin32 + (D->lin_off + q) * PCBA_LIN32_STRIDE;
  const int K = D->alpha;
  float v = row[0], A = fabsf(row[0]), Ee = 0.0f;
  for (int m = 0; m < K; ++m) {
    const float w = row[1 + m];
    v = fmaf(w, sv[m], v);
    A = __fmaf_ru(fabsf(w), fabsf(sv[m]), A);
    Ee = __fmaf_ru(fabsf(w), se[m], Ee);
  }
  const float kk = (float)(2 * K + 2);
  *val = v;
  *err = __fadd_ru(__fadd_ru(__fmul_ru(kk * 0x1p-24f, A), __fmul_ru(Ee, 1.0f + 0x1p-20f)),
                   kk * 0x1p-149f);
}
__device__ __forceinline__ void lin_value_f64(const Engine& E, const ProbDesc* D, int q,
                                              const double* sv, const double* se, double* val,
                                              double* err) {
  const double* row = E.lin64 + (D->lin_off + q) * PCBA_LIN_STRIDE;
  const int K = D->alpha;
  double v = row[0], A = fabs(row[0]), Ee = 0.0;
  for (int m = 0; m < K; ++m) {
    const double w = row[1 + m];
    v = fma(w, sv[m], v);
    A = __fma_ru(fabs(w), fabs(sv[m]), A);
    Ee = __fma_ru(fabs(w), se[m], Ee);
  }
  const double kk = (double)(K + 1);
  *val = v;
  *err = __dadd_ru(__dadd_ru(__dmul_ru(kk * 0x1p-53, A), __dmul_ru(Ee, 1.0 + 0x1p-50)),
                   kk * 0x1p-1074);
}
// Values and bounds of the K shared polynomials of a linear family at a point.
__device__ __forceinline__ void lin_shared_f64(const Engine& E, const ProbDesc* D, const double* x,
                                               double* sv, double* se) {
  const double* sh = E.mono + D->mono_off + D->cp;
  for (int m = 0; m < D->alpha; ++m) horner_f64(sh + (long long)m * D->cg, D->l, D->G, x, &sv[m], &se[m]);
}
__device__ __forceinline__ void lin_shared_f32(const Engine& E, const ProbDesc* D, const float* coef,
                                               const float* x, float* sv, float* se) {
  for (int m = 0; m < D->alpha; ++m)
    horner_f32_any(coef + (long long)m * D->cg, D->l, D->G, x, &sv[m], &se[m]);
}

#define PCBA_KILLERS 32

__global__ void __launch_bounds__(PCBA_TPB) k_eval(Engine E, int mode, void* results) {
  __shared__ double s_key[PCBA_MAX_CAND];
  __shared__ int s_id[PCBA_MAX_CAND];
  __shared__ double sx[PCBA_EVAL_CHUNK][PCBA_MAXD];
  __shared__ float sxf[PCBA_EVAL_CHUNK][PCBA_MAXD];
  __shared__ float s_lsv[PCBA_EVAL_CHUNK][PCBA_MAX_SHARED], s_lse[PCBA_EVAL_CHUNK][PCBA_MAX_SHARED];
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
  // constraints to check: every g_i and h_j, or the rows of a linear family
  const int total = D->lin ? D->nlin : D->alpha + D->beta;

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
    if (D->lin) {
      // the shared polynomials once, then every constraint from them
      __shared__ double s_sv[PCBA_MAX_SHARED], s_se[PCBA_MAX_SHARED];
      if (threadIdx.x == 0) lin_shared_f64(E, D, sx[0], s_sv, s_se);
      __syncthreads();
      for (int q = threadIdx.x; q < D->nlin; q += PCBA_TPB) {
        double val, err;
        lin_value_f64(E, D, q, s_sv, s_se, &val, &err);
        atomicMax(&s_max[0], okey(__dadd_ru(val, err)));
      }
    }
    for (int q = threadIdx.x; !D->lin && q < total; q += PCBA_TPB) {
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
  const float eq_tol = __double2float_rd(E.params->eq_tol);  // never above eq_tol
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
      if (has) {
        for (int q = 0; q < l; ++q) sxf[c][q] = (float)sx[c][q];
        if (D->lin) lin_shared_f32(E, D, mono32 + D->cp, sxf[c], s_lsv[c], s_lse[c]);
      }
    }
    __syncthreads();
    const int nk = (int)min(s_nkill, (unsigned)PCBA_KILLERS);
    if (nk > 0) {
      for (int it = threadIdx.x; it < nc * nk; it += PCBA_TPB) {
        const int c = it / nk;
        const int q = s_kill[it - c * nk];
        if (!s_has[c] || s_viol[c]) continue;
        const bool is_g = D->lin || q < D->alpha;
        float val, err;
        if (D->lin) {
          lin_value_f32(E, D, q, s_lsv[c], s_lse[c], &val, &err);
        } else {
          const float* a = is_g ? mono32 + D->cp + (long long)q * D->cg
                                : mono32 + D->cp + (long long)D->alpha * D->cg +
                                      (long long)(q - D->alpha) * D->ch;
          horner_f32(a, l, is_g ? D->G : D->H, sxf[c], &val, &err);
        }
        if (!(__fadd_ru(is_g ? val : fabsf(val), err) <= (is_g ? 0.0f : eq_tol))) s_viol[c] = 1;
      }
      __syncthreads();
    }
    for (int it = threadIdx.x; it < nc * total; it += PCBA_TPB) {
      const int c = it / total;
      const int q = it - c * total;
      if (!s_has[c] || s_viol[c]) continue;
      const bool is_g = D->lin || q < D->alpha;
      float val, err;
      if (D->lin) {
        lin_value_f32(E, D, q, s_lsv[c], s_lse[c], &val, &err);
      } else {
        const float* a = is_g ? mono32 + D->cp + (long long)q * D->cg
                              : mono32 + D->cp + (long long)D->alpha * D->cg +
                                    (long long)(q - D->alpha) * D->ch;
        horner_f32(a, l, is_g ? D->G : D->H, sxf[c], &val, &err);
      }
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
    double offer = INFINITY, perr = 0.0;
    if (chosen >= 0) {
      double pc, pe;
      horner_f64(base, l, D->P, sx[chosen], &pc, &pe);
      offer = __dadd_ru(pc, pe);
      perr = pe;
      if (!(offer < INFINITY)) chosen = -1;
    }
    const int found = chosen >= 0;
    S->from_warm = found;
    S->warm_err = found ? perr : 0.0;
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

// ---------------------------------------------------------------------------
// Warm start over many candidates: the same choice as k_eval mode 0 (the
// certified-feasible candidate with the lowest FP32 cost bound, ties to the
// lower index, its FP64 cost bound as p_up), computed as (1) every
// candidate's FP32 cost bound, (2) the candidates ranked by it, (3) the lowest
// feasible rank per problem, candidates dropped at their first violated
// bound, and (4) the FP64 cost bound of that candidate.
// ---------------------------------------------------------------------------
__global__ void k_cand_cost(Engine E, float* key) {
  const long long total = (long long)E.np * E.n_warm;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(t / E.n_warm), c = (int)(t - (long long)p * E.n_warm);
    const ProbDesc* D = E.desc + p;
    double x[PCBA_MAXD];
    float k = INFINITY;
    if (eval_candidate(E, 0, p, c, x)) {
      float xf[PCBA_MAXD];
      for (int q = 0; q < D->l; ++q) xf[q] = (float)x[q];
      float v, e;
      horner_f32(E.mono32 + D->mono_off, D->l, D->P, xf, &v, &e);
      const float kk = __fadd_ru(v, e);
      if (!isnan(kk)) k = kk;
    }
    key[t] = k;
  }
}

// Ranks the candidates of problem p by (FP32 cost bound, index): one block per
// problem, bitonic sort in shared memory (at most PCBA_MAX_CAND candidates);
// order[p][rank] = candidate index; first[p] is reset to INT_MAX.
__global__ void __launch_bounds__(PCBA_TPB) k_cand_rank(Engine E, const float* key, int* order,
                                                        int* first) {
  __shared__ float s_key[PCBA_MAX_CAND];
  __shared__ int s_id[PCBA_MAX_CAND];
  const int p = blockIdx.x;
  const int n_c = min(E.n_warm, PCBA_MAX_CAND);
  int n2 = 1;
  while (n2 < n_c) n2 <<= 1;
  for (int c = threadIdx.x; c < n2; c += PCBA_TPB) {
    s_key[c] = c < n_c ? key[(long long)p * E.n_warm + c] : INFINITY;
    s_id[c] = c < n_c ? c : 0x7fffffff;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += PCBA_TPB) {
        const int o = i ^ j;
        if (o > i) {
          const bool gt = s_key[i] > s_key[o] || (s_key[i] == s_key[o] && s_id[i] > s_id[o]);
          if (gt == ((i & k) == 0)) {
            const float tk = s_key[i]; s_key[i] = s_key[o]; s_key[o] = tk;
            const int ti = s_id[i]; s_id[i] = s_id[o]; s_id[o] = ti;
          }
        }
      }
      __syncthreads();
    }
  for (int c = threadIdx.x; c < n_c; c += PCBA_TPB) order[(long long)p * E.n_warm + c] = s_id[c];
  if (threadIdx.x == 0) first[p] = 0x7fffffff;
}

// The lowest rank whose candidate is certified feasible, per problem: one
// block per problem.  Warps take ranks in increasing order from a shared
// counter; a warp checks its candidate against 32 constraints at a time (lane
// i: constraint 32 t + i, FP32 Horner with its error bound, FP64 where that
// is undecided) and drops it at the first tile with a violated bound.  The
// tiles that dropped recent candidates (a ring of 4) are tried first:
// candidates of neighbouring cost tend to fail on the same constraints.  A
// rank is skipped once a lower one is known feasible, so the result is the
// minimum feasible rank whatever the order in which warps finish.  STAGE: the
// constraint coefficients (FP32) are first copied to shared memory.
// first[p] = that rank, or INT_MAX.
template <bool STAGE>
__global__ void __launch_bounds__(PCBA_CAND_TPB, 1) k_cand_first(Engine E, const float* key,
                                                              const int* order, int* first) {
  extern __shared__ float kcf[];
  __shared__ int s_next, s_best, s_kpos;
  __shared__ int s_killer[4];
  const int p = blockIdx.x;
  // gridDim.y blocks share a problem: block y takes ranks y, y + gridDim.y, ...
  // and all of them lower first[p] (set to INT_MAX by k_cand_rank)
  const int nb = gridDim.y, by = blockIdx.y;
  const ProbDesc* D = E.desc + p;
  const int l = D->l, alpha = D->alpha;
  const int total = D->lin ? D->nlin : D->alpha + D->beta;
  const int tiles = (total + 31) >> 5;
  const int n_c = min(E.n_warm, PCBA_MAX_CAND);
  const long long base = (long long)p * E.n_warm;
  const long long nf = (long long)alpha * D->cg + (long long)D->beta * D->ch;
  const float* src = E.mono32 + D->mono_off + D->cp;
  if (STAGE)
    for (long long t = threadIdx.x; t < nf; t += blockDim.x) kcf[t] = src[t];
  const float* coef = STAGE ? kcf : src;
  if (threadIdx.x == 0) {
    s_next = 0;
    s_best = 0x7fffffff;
    s_kpos = 0;
    for (int k = 0; k < 4; ++k) s_killer[k] = -1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const float eq_tol = __double2float_rd(E.params->eq_tol);  // never above eq_tol
  for (;;) {
    // lane 0 reads the shared state and broadcasts it, so that the warp stays
    // converged for its vote
    int rank = 0, stop = 0;
    if (lane == 0) {
      rank = atomicAdd(&s_next, 1) * nb + by;
      if (nb > 1 && rank < *(volatile int*)&s_best)
        atomicMin(&s_best, *(volatile int*)&first[p]);  // ranks found by the other blocks
      stop = rank >= n_c || rank >= *(volatile int*)&s_best;
    }
    rank = __shfl_sync(0xffffffffu, rank, 0);
    if (__shfl_sync(0xffffffffu, stop, 0)) break;
    const int c = order[base + rank];
    if (!(key[base + c] < INFINITY)) continue;  // no candidate point
    float xf[PCBA_MAXD];
    for (int r = 0; r < l; ++r) xf[r] = (float)E.warm[(base + c) * PCBA_MAXD + r];
    int kill[4];
    for (int k = 0; k < 4; ++k)
      kill[k] = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile int*)&s_killer[k] : 0, 0);
    // linear family: the shared polynomials at the point, once per candidate
    float lsv[PCBA_MAX_SHARED], lse[PCBA_MAX_SHARED];
    if (D->lin) lin_shared_f32(E, D, coef, xf, lsv, lse);
    bool bad = false;
    for (int step = 0; step < 4 + tiles && !bad; ++step) {
      int t;
      if (step < 4) {
        t = kill[step];
        bool dup = t < 0;
        for (int k = 0; k < step; ++k) dup = dup || kill[k] == t;
        if (dup) continue;
      } else {
        t = step - 4;
        if (t == kill[0] || t == kill[1] || t == kill[2] || t == kill[3]) continue;
      }
      const int q = t * 32 + lane;
      bool lane_bad = false;
      if (q < total && D->lin) {
        float val, err;
        lin_value_f32(E, D, q, lsv, lse, &val, &err);
        if (!(__fadd_ru(val, err) <= 0.0f)) {
          lane_bad = true;
          if (__fsub_rd(val, err) <= 0.0f) {
            // undecided in FP32: the shared polynomials and the row in FP64
            double xd[PCBA_MAXD], sv[PCBA_MAX_SHARED], se[PCBA_MAX_SHARED];
            for (int r = 0; r < l; ++r) xd[r] = (double)xf[r];
            lin_shared_f64(E, D, xd, sv, se);
            double v64, e64;
            lin_value_f64(E, D, q, sv, se, &v64, &e64);
            lane_bad = !(__dadd_ru(v64, e64) <= 0.0);
          }
        }
      } else if (q < total) {
        const bool is_g = q < alpha;
        const long long off = is_g ? (long long)q * D->cg
                                   : (long long)alpha * D->cg + (long long)(q - alpha) * D->ch;
        float val, err;
        horner_f32_any(coef + off, l, is_g ? D->G : D->H, xf, &val, &err);
        const float lim = is_g ? 0.0f : eq_tol;
        if (!(__fadd_ru(is_g ? val : fabsf(val), err) <= lim)) {
          lane_bad = true;
          if (__fsub_rd(is_g ? val : fabsf(val), err) <= lim) {
            // undecided in FP32: decide in FP64 on the FP64 coefficients at
            // the same (FP32) point
            double xd[PCBA_MAXD];
            for (int r = 0; r < l; ++r) xd[r] = (double)xf[r];
            double v64, e64;
            horner_f64(E.mono + D->mono_off + D->cp + off, l, is_g ? D->G : D->H, xd, &v64, &e64);
            lane_bad = !(__dadd_ru(is_g ? v64 : fabs(v64), e64) <= (is_g ? 0.0 : E.params->eq_tol));
          }
        }
      }
      if (__any_sync(0xffffffffu, lane_bad)) {
        bad = true;
        if (lane == 0) s_killer[atomicAdd(&s_kpos, 1) & 3] = t;
      }
    }
    if (!bad && lane == 0) {
      atomicMin(&s_best, rank);
      atomicMin(&first[p], rank);
    }
  }
}

// The first certified-feasible candidate in rank order seeds p_up with its
// FP64 cost bound.
__global__ void k_cand_pick(Engine E, const int* order, const int* first) {
  // one problem per block: the FP64 evaluation is a long chain of slow
  // dependent operations, best kept on SMs of its own
  const int p = blockIdx.x;
  if (p >= E.np || threadIdx.x != 0) return;
  const ProbDesc* D = E.desc + p;
  ProbState* S = E.state + p;
  const int n_c = min(E.n_warm, PCBA_MAX_CAND);
  const long long base = (long long)p * E.n_warm;
  const int br = first[p];
  const int l = D->l;
  double x[PCBA_MAXD];
  double offer = INFINITY, perr = 0.0;
  int found = 0;
  if (br < n_c && eval_candidate(E, 0, p, order[base + br], x)) {
    double pc, pe;
    horner_f64(E.mono + D->mono_off, l, D->P, x, &pc, &pe);
    offer = __dadd_ru(pc, pe);
    perr = pe;
    found = offer < INFINITY;
  }
  S->from_warm = found;
  S->warm_err = found ? perr : 0.0;
  S->p_up_carry = found ? offer : INFINITY;
  S->seeded = found;
  S->seed_cost = found ? offer : INFINITY;
  for (int q = 0; q < PCBA_MAXD; ++q) {
    const double v = (found && q < l) ? x[q] : NAN;
    if (found && q < l) S->warm_x[q] = v;
    S->seed_x[q] = v;
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

// pcba_eval_points_f32: one thread per point, the certification's FP32 Horner.
struct PointPoly {
  int l;
  int deg[PCBA_MAXD];
};
__global__ void k_eval_points_f32(const float* a, PointPoly q, const float* x, int n,
                                  int unrolled, float* val, float* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xf[PCBA_MAXD];
  for (int r = 0; r < q.l; ++r) xf[r] = x[(long long)i * q.l + r];
  float v, e;
  if (unrolled) horner_f32_any(a, q.l, q.deg, xf, &v, &e);
  else horner_f32(a, q.l, q.deg, xf, &v, &e);
  val[i] = v;
  err[i] = e;
}

// Candidate points of guided solves: candidate c of problem p is the guess of
// p (normalised coordinates, guess_dim axes) plus stencil row c, clamped to
// [-1, 1] and mapped to the box; axes beyond guess_dim take the box centre.
// refine = 1: the centre is the seed already chosen for the problem (its
// normalised coordinates), or the guess where no candidate was certified.
__global__ void k_candidates(Engine E, const float* guess, int guess_dim, const double* stencil,
                             int n_stencil, double* cand, int refine) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)E.np * n_stencil) return;
  const int p = (int)(t / n_stencil), c = (int)(t - (long long)p * n_stencil);
  const ProbDesc* D = E.desc + p;
  const ProbState* S = E.state + p;
  const bool from_seed = refine && S->seeded;
  double* o = cand + t * PCBA_MAXD;
  for (int r = 0; r < PCBA_MAXD; ++r) {
    double x = 0.0;
    if (r < D->l) {
      double u = 0.0;
      if (r < guess_dim) {
        const double centre =
            from_seed ? 2.0 * (S->seed_x[r] - D->lo[r]) / (D->hi[r] - D->lo[r]) - 1.0
                      : (double)guess[(long long)p * guess_dim + r];
        u = centre + stencil[(long long)c * guess_dim + r];
      }
      u = fmin(fmax(u, -1.0), 1.0);
      x = D->lo[r] + 0.5 * (u + 1.0) * (D->hi[r] - D->lo[r]);
    }
    o[r] = x;
  }
}
