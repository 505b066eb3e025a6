// Local polish of an incumbent (not in the paper).
//
// With equality constraints and a tight eq_tol, a box is certified feasible
// (Def. 4: every h_j stays within [-eq_tol, eq_tol] over the box) only once it
// is very small, so p_up stays infinite for many steps and Alg. 4 eliminates
// nothing: the list grows until the memory test stops the solve.  A certified
// feasible point found by other means gives p_up at once.  This kernel makes
// such a point: from the point a solve with a loose eq_tol returned, a
// log-barrier Newton method in FP64 on
//
//   min  p(x) - mu sum_i log(-g_i(x))   subject to  h_j(x) = 0,  x in the box,
//
// with mu lowered tenfold per level.  Each Newton step solves
//
//   [ H   J^T ] [ dx ]   [ -(grad p - mu sum_i grad g_i / g_i) ]
//   [ J    0  ] [ nu ] = [ -h                                  ]
//
// with H = hess p + mu sum_i grad g_i grad g_i^T / g_i^2 (the curvature terms
// of the constraints are left out, a Gauss-Newton barrier Hessian), then a
// backtracking search on the merit p - mu sum_i log(-g_i) + rho sum_j |h_j|
// that keeps every g_i < 0 and x in the box.  For a convex program the
// barrier point at mu is within (number of inequalities) * mu of the optimum,
// so the last level uses mu = gap / max(1, alpha).  At the end of every level
// the iterate rounded to FP32 coordinates (the coordinates the certification
// of a warm start uses) is kept if every g_i < 0 and sum_j |h_j| <= eq_tol / 2
// there; the last kept point is the output.  It is only a candidate: it lowers
// p_up only if the usual warm-start certification accepts it.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "pcba_device.cuh"

#define PCBA_POLISH_TPB 256

// Value, gradient and (HESS) Hessian of a dense monomial tensor a (row-major,
// last axis fastest; degrees deg[0..L), strides stride[0..L)) at x: nested
// Horner with forward-mode derivatives.  One Horner update q <- q x_0 + c,
// with the values before the update on the right, gives
//   dq/dx_0 <- dq/dx_0 x_0 + q,            dq/dx_s <- dq/dx_s x_0 + dc/dx_s,
//   d2q/dx_0^2 <- d2q/dx_0^2 x_0 + 2 dq/dx_0,
//   d2q/dx_0 dx_s <- d2q/dx_0 dx_s x_0 + dq/dx_s,
//   d2q/dx_s dx_t <- d2q/dx_s dx_t x_0 + d2c/dx_s dx_t        (s, t > 0).
// H is L x L row-major; only its entries (s, t) with s <= t are written.
template <int L, bool HESS>
struct PolyDiff {
  __device__ __forceinline__ static void eval(const double* a, const int* deg, const int* stride,
                                              const double* x, double& v, double* g, double* H) {
    v = 0.0;
#pragma unroll
    for (int s = 0; s < L; ++s) g[s] = 0.0;
    if (HESS) {
#pragma unroll
      for (int s = 0; s < L * L; ++s) H[s] = 0.0;
    }
    const double x0 = x[0];
    for (int i = deg[0]; i >= 0; --i) {
      double vi, gi[L - 1], Hi[HESS ? (L - 1) * (L - 1) : 1];
      PolyDiff<L - 1, HESS>::eval(a + (long long)i * stride[0], deg + 1, stride + 1, x + 1, vi, gi,
                                  Hi);
      if (HESS) {
#pragma unroll
        for (int s = 1; s < L; ++s)
#pragma unroll
          for (int t = s; t < L; ++t)
            H[s * L + t] = fma(H[s * L + t], x0, Hi[(s - 1) * (L - 1) + (t - 1)]);
#pragma unroll
        for (int s = 1; s < L; ++s) H[s] = fma(H[s], x0, g[s]);
        H[0] = fma(H[0], x0, 2.0 * g[0]);
      }
#pragma unroll
      for (int s = 1; s < L; ++s) g[s] = fma(g[s], x0, gi[s - 1]);
      g[0] = fma(g[0], x0, v);
      v = fma(v, x0, vi);
    }
  }
};
template <bool HESS>
struct PolyDiff<1, HESS> {
  __device__ __forceinline__ static void eval(const double* a, const int* deg, const int*,
                                              const double* x, double& v, double* g, double* H) {
    v = 0.0;
    g[0] = 0.0;
    if (HESS) H[0] = 0.0;
    const double x0 = x[0];
    for (int i = deg[0]; i >= 0; --i) {
      if (HESS) H[0] = fma(H[0], x0, 2.0 * g[0]);
      g[0] = fma(g[0], x0, v);
      v = fma(v, x0, a[i]);
    }
  }
};

// value only, nested Horner
template <int L>
struct PolyVal {
  __device__ __forceinline__ static double eval(const double* a, const int* deg, const int* stride,
                                                const double* x) {
    double v = 0.0;
    for (int i = deg[0]; i >= 0; --i)
      v = fma(v, x[0], PolyVal<L - 1>::eval(a + (long long)i * stride[0], deg + 1, stride + 1, x + 1));
    return v;
  }
};
template <>
struct PolyVal<1> {
  __device__ __forceinline__ static double eval(const double* a, const int* deg, const int*,
                                                const double* x) {
    double v = 0.0;
    for (int i = deg[0]; i >= 0; --i) v = fma(v, x[0], a[i]);
    return v;
  }
};

// block-wide sum of n doubles per thread; the sums land in vals of thread 0.
// red holds (PCBA_POLISH_TPB / 32) * n doubles.
__device__ __forceinline__ void polish_block_sum(double* vals, int n, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q < n; ++q) {
    double x = vals[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[w * n + q] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < n; ++q) {
      double x = 0.0;
      for (int ww = 0; ww < PCBA_POLISH_TPB / 32; ++ww) x += red[ww * n + q];
      vals[q] = x;
    }
  __syncthreads();
}

// index of (s, t), s <= t, in the packed upper triangle of an L x L matrix
__host__ __device__ constexpr int polish_tri(int L, int s, int t) {
  return s * L - s * (s - 1) / 2 + (t - s);
}

// Solves the KKT system by Gaussian elimination with partial pivoting (one
// thread).  acc: gradient [L] then the Hessian's packed upper triangle; hv,
// hg: h_j and grad h_j (beta rows of L).  shift is added to H's diagonal.
// Writes dx, and the largest |nu_j| to *numax; returns false if the system is
// singular or the solution not finite.
template <int L>
__device__ bool polish_kkt(const double* acc, const double* hv, const double* hg, int beta,
                           double shift, double* K, double* dx, double* numax) {
  const int n = L + beta, w = n + 1;
  for (int r = 0; r < n * w; ++r) K[r] = 0.0;
  for (int r = 0; r < L; ++r) {
    for (int c = 0; c < L; ++c)
      K[r * w + c] = acc[L + (r <= c ? polish_tri(L, r, c) : polish_tri(L, c, r))];
    K[r * w + r] += shift + 1e-12 * (1.0 + fabs(K[r * w + r]));
    K[r * w + n] = -acc[r];
  }
  for (int q = 0; q < beta; ++q) {
    for (int r = 0; r < L; ++r) {
      K[(L + q) * w + r] = hg[q * L + r];
      K[r * w + L + q] = hg[q * L + r];
    }
    K[(L + q) * w + n] = -hv[q];
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(K[r * w + c]) > fabs(K[piv * w + c])) piv = r;
    if (!(fabs(K[piv * w + c]) > 1e-300)) return false;
    if (piv != c)
      for (int k = 0; k < w; ++k) {
        const double t = K[c * w + k];
        K[c * w + k] = K[piv * w + k];
        K[piv * w + k] = t;
      }
    for (int r = c + 1; r < n; ++r) {
      const double f = K[r * w + c] / K[c * w + c];
      for (int k = c; k < w; ++k) K[r * w + k] -= f * K[c * w + k];
    }
  }
  double sol[L + PCBA_MAXD];
  for (int r = n - 1; r >= 0; --r) {
    double t = K[r * w + n];
    for (int k = r + 1; k < n; ++k) t -= K[r * w + k] * sol[k];
    sol[r] = t / K[r * w + r];
    if (!isfinite(sol[r])) return false;
  }
  double nm = 0.0;
  for (int q = 0; q < beta; ++q) nm = fmax(nm, fabs(sol[L + q]));
  *numax = nm;
  for (int r = 0; r < L; ++r) dx[r] = sol[r];
  return true;
}

// The cost is split into rows over its first K axes (row-major, so a row is
// a contiguous block of the tensor): with the outer monomial
// m(x) = prod_{r<K} x_r^{j_r} and the inner polynomial q of the row,
//   p_row = m q,  d/dx_r = dm/dx_r q (r < K),  d/dx_s = m dq/dx_s (s >= K),
//   d2/dx_r dx_t = d2m/dx_r dx_t q,  d2/dx_r dx_s = dm/dx_r dq/dx_s,
//   d2/dx_s dx_t = m d2q/dx_s dx_t,
// and the rows add up, so each thread handles whole rows.  pw, dpw, ddpw hold
// x_r^j and its first and second derivatives (17 per axis).
template <int L, int K, bool HESS>
__device__ __forceinline__ void cost_row(const double* a, const int* dP, const int* tP,
                                         const double* x, const double* pw, const double* dpw,
                                         const double* ddpw, int row, double& val, double* acc) {
  int j[K > 0 ? K : 1];
  int rem = row;
#pragma unroll
  for (int r = K - 1; r >= 0; --r) {
    j[r] = rem % (dP[r] + 1);
    rem /= dP[r] + 1;
  }
  const long long off = K > 0 ? (long long)row * tP[K > 0 ? K - 1 : 0] : 0;
  constexpr int NI = L - K;
  double P[K > 0 ? K : 1], Dv[K > 0 ? K : 1];
  double m = 1.0;
#pragma unroll
  for (int r = 0; r < K; ++r) {
    P[r] = pw[r * 17 + j[r]];
    Dv[r] = dpw[r * 17 + j[r]];
    m *= P[r];
  }
  if (!HESS) {
    val += m * PolyVal<NI>::eval(a + off, dP + K, tP + K, x + K);
    return;
  }
  double vq, gq[NI], Hq[NI * NI];
  PolyDiff<NI, true>::eval(a + off, dP + K, tP + K, x + K, vq, gq, Hq);
  val += m * vq;
#pragma unroll
  for (int r = 0; r < K; ++r) {
    double dm = Dv[r];
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (s != r) dm *= P[s];
    acc[r] += dm * vq;
#pragma unroll
    for (int s = 0; s < NI; ++s) acc[L + polish_tri(L, r, K + s)] += dm * gq[s];
#pragma unroll
    for (int t = r; t < K; ++t) {
      double d2 = t == r ? ddpw[r * 17 + j[r]] : Dv[r] * Dv[t];
#pragma unroll
      for (int s = 0; s < K; ++s)
        if (s != r && s != t) d2 *= P[s];
      acc[L + polish_tri(L, r, t)] += d2 * vq;
    }
  }
#pragma unroll
  for (int s = 0; s < NI; ++s) {
    acc[K + s] += m * gq[s];
#pragma unroll
    for (int t = s; t < NI; ++t) acc[L + polish_tri(L, K + s, K + t)] += m * Hq[s * NI + t];
  }
}

template <int L, bool HESS>
__device__ __forceinline__ void cost_row_any(int K, const double* a, const int* dP, const int* tP,
                                             const double* x, const double* pw, const double* dpw,
                                             const double* ddpw, int row, double& val,
                                             double* acc) {
  if constexpr (L == 1) {
    cost_row<1, 0, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc);
  } else {
    switch (K) {
      case 1: cost_row<L, 1, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc); break;
      case 2: if constexpr (L > 2) cost_row<L, 2, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc); break;
      case 3: if constexpr (L > 3) cost_row<L, 3, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc); break;
      case 4: if constexpr (L > 4) cost_row<L, 4, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc); break;
      case 5: if constexpr (L > 5) cost_row<L, 5, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc); break;
      case 6: if constexpr (L > 6) cost_row<L, 6, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc); break;
      default: if constexpr (L > 7) cost_row<L, 7, HESS>(a, dP, tP, x, pw, dpw, ddpw, row, val, acc); break;
    }
  }
}

// Slice i of a constraint polynomial along axis 0 (the terms with x_0^i):
// its value and (GRAD) gradient, x_0^i q_i(x_1..) and its derivatives, with
// pw / dpw the tables of x_0^j and j x_0^(j-1).  The slices of a polynomial
// add up to it; l = 1 has a single slice (the whole polynomial).
template <int L, bool GRAD>
__device__ __forceinline__ void poly_slice(const double* a, const int* deg, const int* stride,
                                           const double* x, const double* pw, const double* dpw,
                                           int i, double& v, double* g) {
  if constexpr (L == 1) {
    double Hd[1];
    if (GRAD) PolyDiff<1, false>::eval(a, deg, stride, x, v, g, Hd);
    else v = PolyVal<1>::eval(a, deg, stride, x);
  } else {
    const double* ai = a + (long long)i * stride[0];
    if (GRAD) {
      double vq, gq[L - 1], Hd[1];
      PolyDiff<L - 1, false>::eval(ai, deg + 1, stride + 1, x + 1, vq, gq, Hd);
      v = pw[i] * vq;
      g[0] = dpw[i] * vq;
#pragma unroll
      for (int s = 0; s < L - 1; ++s) g[1 + s] = pw[i] * gq[s];
    } else {
      v = pw[i] * PolyVal<L - 1>::eval(ai, deg + 1, stride + 1, x + 1);
    }
  }
}

// lanes per constraint: the slices along axis 0, rounded up to a power of two
__device__ __forceinline__ int polish_group(int L, int d0) {
  if (L == 1) return 1;
  int gs = 1;
  while (gs < d0 + 1) gs <<= 1;
  return gs;
}

// One block per problem; blocks of problems with l != L return at once (the
// host launches one instantiation per dimension present).  Work items of a
// block: the R rows of the cost (K outer axes, the fewest with R >= 32, at
// most l - 1), then, for every inequality and every equality, a group of
// lanes (a power of two) that evaluate its slices along axis 0 and add them
// with warp shuffles; the three segments start at multiples of 32 so that a
// warp never spans two of them, and the group's first lane takes the sum
// (short dependency chains: the latency of FP64 FMAs, not their rate, bounds
// this kernel).  Problems with
// more than PCBA_MAXD equality constraints, infeasible ones and ones without
// a point get a NaN row.  out: [np][PCBA_MAXD] doubles.
//
// One full evaluation at a point gives, summed over the block: the cost's
// gradient and Hessian, B1 = sum_i grad g_i / g_i and B2 = sum_i grad g_i
// grad g_i^T / g_i^2 (so that the barrier gradient and Gauss-Newton Hessian
// at any mu are grad p - mu B1 and hess p + mu B2), the merit pieces
// p, -sum_i log(-g_i), sum_j |h_j|, and h_j with its gradient.  The full step
// of every Newton iteration is evaluated this way (if it is accepted, the
// next iteration needs no other evaluation); shorter steps of the backtracking
// search evaluate values only.
template <int L>
__global__ void __launch_bounds__(PCBA_POLISH_TPB, 1)
    k_polish(Engine E, double* out, double mu0, double gap, double eq_tol, int iters) {
  constexpr int NS = L + L * (L + 1) / 2;  // gradient + packed Hessian
  constexpr int ND = 2 * NS + 3;           // cost part, barrier part, merit pieces
  __shared__ double sx[L], sxt[L], sdx[L], sbest[L];
  __shared__ double spw[L * 17], sdpw[L * 17], sddpw[L * 17];
  __shared__ double sred[(PCBA_POLISH_TPB / 32) * ND];
  __shared__ double sdata[2][ND];
  __shared__ double shv[2][PCBA_MAXD], shg[2][PCBA_MAXD * L];
  __shared__ double sK[(L + PCBA_MAXD) * (L + PCBA_MAXD + 1)];
  __shared__ double s_m[3];
  __shared__ double s_rho, s_rel;
  __shared__ int s_ok, s_stop, s_best, s_has, s_okd[2];
  const int p = blockIdx.x;
  const ProbDesc* D = E.desc + p;
  if (D->l != L) return;
  const ProbState* S = E.state + p;
  const int alpha = D->alpha, beta = D->beta;
  const double* base = E.mono + D->mono_off;
  const double* gbase = base + D->cp;
  const double* hbase = gbase + (long long)alpha * D->cg;
  int dP[L], dG[L], dH[L], tP[L], tG[L], tH[L];
#pragma unroll
  for (int r = 0; r < L; ++r) {
    dP[r] = D->P[r];
    dG[r] = D->G[r];
    dH[r] = D->H[r];
  }
  tP[L - 1] = tG[L - 1] = tH[L - 1] = 1;
#pragma unroll
  for (int r = L - 2; r >= 0; --r) {
    tP[r] = tP[r + 1] * (dP[r + 1] + 1);
    tG[r] = tG[r + 1] * (dG[r + 1] + 1);
    tH[r] = tH[r + 1] * (dH[r + 1] + 1);
  }
  int K = 0, R = 1;
  while (K < L - 1 && R < 32) R *= dP[K++] + 1;
  const int gG = polish_group(L, dG[0]), gH = polish_group(L, dH[0]);
  const int seg_g = (R + 31) & ~31;
  const int seg_h = seg_g + ((alpha * gG + 31) & ~31);
  const int items = seg_h + ((beta * gH + 31) & ~31);
  double* res = out + (long long)p * PCBA_MAXD;
  if (threadIdx.x == 0) {
    double x0[PCBA_MAXD];
    s_has = S->status != PCBA_INFEASIBLE && beta <= PCBA_MAXD && eval_candidate(E, 1, p, 0, x0);
    for (int q = 0; q < L; ++q) sx[q] = x0[q];
    s_best = 0;
    for (int q = 0; q < PCBA_MAXD; ++q) res[q] = NAN;
  }
  __syncthreads();
  if (!s_has) return;

  // x_r^j, j x_r^(j-1), j (j-1) x_r^(j-2) for the outer axes of the cost rows
  // (axis 0 among them whenever l > 1, which the constraint slices use)
  auto powers = [&](const double* xv) {
    for (int t = threadIdx.x; t < K * 17; t += PCBA_POLISH_TPB) {
      const int r = t / 17, jj = t - r * 17;
      const double x = xv[r];
      double pj = 1.0, pj1 = 0.0, pj2 = 0.0;
      for (int k = 0; k < jj; ++k) {
        pj2 = pj2 * x + 2.0 * pj1;
        pj1 = pj1 * x + pj;
        pj *= x;
      }
      spw[t] = pj;
      sdpw[t] = pj1;
      sddpw[t] = pj2;
    }
    __syncthreads();
  };
  // values only: s_m = (p, -sum log(-g_i), sum |h_j|) at xv; s_ok = every g_i < 0
  auto merit = [&](const double* xv) {
    powers(xv);
    double m[3] = {0.0, 0.0, 0.0};
    int feas = 1;
    for (int q = threadIdx.x; q < items; q += PCBA_POLISH_TPB) {
      if (q < seg_g) {
        if (q < R) cost_row_any<L, false>(K, base, dP, tP, xv, spw, sdpw, sddpw, q, m[0], nullptr);
      } else {
        const bool is_g = q < seg_h;
        const int gs = is_g ? gG : gH, u = q - (is_g ? seg_g : seg_h);
        const int c = u / gs, sl = u - c * gs;
        const bool live = c < (is_g ? alpha : beta) && sl <= (is_g ? dG[0] : dH[0]);
        double v = 0.0;
        if (live) {
          double gd[1];
          if (is_g)
            poly_slice<L, false>(gbase + (long long)c * D->cg, dG, tG, xv, spw, sdpw, sl, v, gd);
          else
            poly_slice<L, false>(hbase + (long long)c * D->ch, dH, tH, xv, spw, sdpw, sl, v, gd);
        }
        for (int o = gs >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (sl == 0 && c < (is_g ? alpha : beta)) {
          if (!is_g) m[2] += fabs(v);
          else if (v < 0.0) m[1] -= log(-v);
          else feas = 0;
        }
      }
    }
    feas = __syncthreads_and(feas);
    polish_block_sum(m, 3, sred);
    if (threadIdx.x == 0) {
      s_m[0] = m[0];
      s_m[1] = m[1];
      s_m[2] = m[2];
      s_ok = feas;
    }
    __syncthreads();
  };
  // full evaluation at xv into sdata[d], shv[d], shg[d], s_okd[d]
  auto evaluate = [&](const double* xv, int d) {
    powers(xv);
    double acc[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) acc[q] = 0.0;
    int feas = 1;
    for (int q = threadIdx.x; q < items; q += PCBA_POLISH_TPB) {
      if (q < seg_g) {
        if (q < R) cost_row_any<L, true>(K, base, dP, tP, xv, spw, sdpw, sddpw, q, acc[2 * NS], acc);
      } else {
        const bool is_g = q < seg_h;
        const int gs = is_g ? gG : gH, u = q - (is_g ? seg_g : seg_h);
        const int c = u / gs, sl = u - c * gs;
        const bool live = c < (is_g ? alpha : beta) && sl <= (is_g ? dG[0] : dH[0]);
        double v = 0.0, g[L];
#pragma unroll
        for (int r = 0; r < L; ++r) g[r] = 0.0;
        if (live) {
          if (is_g)
            poly_slice<L, true>(gbase + (long long)c * D->cg, dG, tG, xv, spw, sdpw, sl, v, g);
          else
            poly_slice<L, true>(hbase + (long long)c * D->ch, dH, tH, xv, spw, sdpw, sl, v, g);
        }
        for (int o = gs >> 1; o > 0; o >>= 1) {
          v += __shfl_xor_sync(0xffffffffu, v, o);
#pragma unroll
          for (int r = 0; r < L; ++r) g[r] += __shfl_xor_sync(0xffffffffu, g[r], o);
        }
        if (sl == 0 && c < (is_g ? alpha : beta)) {
          if (is_g) {
            if (v < 0.0) {
              acc[2 * NS + 1] -= log(-v);
              const double inv = 1.0 / v;
#pragma unroll
              for (int s2 = 0; s2 < L; ++s2) {
                acc[NS + s2] += g[s2] * inv;
#pragma unroll
                for (int t = s2; t < L; ++t)
                  acc[NS + L + polish_tri(L, s2, t)] += g[s2] * g[t] * inv * inv;
              }
            } else {
              feas = 0;
            }
          } else {
            acc[2 * NS + 2] += fabs(v);
            shv[d][c] = v;
#pragma unroll
            for (int r = 0; r < L; ++r) shg[d][c * L + r] = g[r];
          }
        }
      }
    }
    feas = __syncthreads_and(feas);
    polish_block_sum(acc, ND, sred);
    if (threadIdx.x == 0) {
      for (int q = 0; q < ND; ++q) sdata[d][q] = acc[q];
      s_okd[d] = feas;
    }
    __syncthreads();
  };

  int cur = 0;
  evaluate(sx, cur);
  if (!s_okd[cur]) return;  // the start point must be strictly inside every g_i < 0
  double mu = mu0 * fmax(1.0, fabs(sdata[cur][2 * NS]));
  const double mu_end = fmin(mu, gap / fmax(1.0, (double)alpha));
  double rho = 10.0;
  for (int lev = 0; lev < 24; ++lev) {
    // centring tolerance on the Newton step: loose on the way, tight at the end
    const double tol = mu <= mu_end ? 1e-11 : 1e-7;
    for (int it = 0; it < iters; ++it) {
      bool moved = false, stop = false;
      // Newton step; if its line search fails, once more with H shifted to
      // diagonal dominance (Gershgorin), which makes the step a descent one
      for (int attempt = 0; attempt < 2 && !moved && !stop; ++attempt) {
        if (threadIdx.x == 0) {
          const double* dc = sdata[cur];
          double acc[NS];
          for (int q = 0; q < L; ++q) acc[q] = dc[q] - mu * dc[NS + q];
          for (int q = L; q < NS; ++q) acc[q] = dc[q] + mu * dc[NS + q];
          double shift = 0.0;
          if (attempt == 1)
            for (int r = 0; r < L; ++r) {
              double off = 0.0;
              for (int c = 0; c < L; ++c)
                if (c != r)
                  off += fabs(acc[L + (r <= c ? polish_tri(L, r, c) : polish_tri(L, c, r))]);
              shift = fmax(shift, off - acc[L + polish_tri(L, r, r)]);
            }
          double numax = 0.0, xm = 0.0, step = 0.0;
          const bool ok = polish_kkt<L>(acc, shv[cur], shg[cur], beta, shift, sK, sdx, &numax);
          for (int r = 0; r < L; ++r) {
            if (!ok) sdx[r] = 0.0;
            step = fmax(step, fabs(sdx[r]));
            xm = fmax(xm, fabs(sx[r]));
          }
          if (ok) rho = fmax(rho, 2.0 * numax + 1.0);
          s_rho = rho;
          s_stop = !ok || step <= tol * (1.0 + xm);
          s_rel = step / (1.0 + xm);
          for (int q = 0; q < L; ++q) sxt[q] = fmin(fmax(sx[q] + sdx[q], D->lo[q]), D->hi[q]);
        }
        __syncthreads();
        rho = s_rho;
        const double rel = s_rel;
        if (s_stop) {
          stop = true;
          break;
        }
        const double* dc = sdata[cur];
        const double phi0 = dc[2 * NS] + mu * dc[2 * NS + 1] + rho * dc[2 * NS + 2];
        // the full step, evaluated in full
        evaluate(sxt, 1 - cur);
        const double* dn = sdata[1 - cur];
        if (s_okd[1 - cur] && dn[2 * NS] + mu * dn[2 * NS + 1] + rho * dn[2 * NS + 2] <= phi0) {
          if (threadIdx.x == 0)
            for (int q = 0; q < L; ++q) sx[q] = sxt[q];
          cur = 1 - cur;
          moved = true;
          __syncthreads();
          break;
        }
        // shorter steps, values only
        double t = 0.5;
        for (int ls = 1; ls < 30 && t * rel > 1e-15; ++ls, t *= 0.5) {
          if (threadIdx.x == 0)
            for (int q = 0; q < L; ++q) sxt[q] = fmin(fmax(sx[q] + t * sdx[q], D->lo[q]), D->hi[q]);
          __syncthreads();
          merit(sxt);
          if (s_ok && s_m[0] + mu * s_m[1] + rho * s_m[2] <= phi0) {
            moved = true;
            break;
          }
        }
        if (moved) {
          if (threadIdx.x == 0)
            for (int q = 0; q < L; ++q) sx[q] = sxt[q];
          __syncthreads();
          evaluate(sx, cur);
        }
      }
      if (!moved) break;
    }
    // keep the FP32-rounded iterate if it is strictly feasible with margin
    if (threadIdx.x == 0) {
      int inbox = 1;
      for (int q = 0; q < L; ++q) {
        sxt[q] = (double)__double2float_rn(sx[q]);
        inbox &= sxt[q] >= D->lo[q] && sxt[q] <= D->hi[q];
      }
      s_stop = !inbox;
    }
    __syncthreads();
    if (!s_stop) {
      merit(sxt);
      if (threadIdx.x == 0 && s_ok && s_m[2] <= 0.5 * eq_tol && isfinite(s_m[0])) {
        for (int q = 0; q < L; ++q) sbest[q] = sxt[q];
        s_best = 1;
      }
      __syncthreads();
    }
    if (mu <= mu_end) break;
    mu = fmax(0.1 * mu, mu_end);
  }
  if (threadIdx.x == 0 && s_best)
    for (int q = 0; q < PCBA_MAXD; ++q) res[q] = q < L ? sbest[q] : 0.0;
}
