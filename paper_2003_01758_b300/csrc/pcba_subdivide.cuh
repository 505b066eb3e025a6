// Subdivision kernels of libpcba (sm_103a): Alg. 2 + Alg. 3 for many problems
// at once.  k2_subdivide loads parent patches directly; k2_subdivide_tma
// stages them in shared memory with bulk tensor copies.  Both bisect every
// item in direction r (de Casteljau at 1/2 on every fibre, Sec. II-E), bound
// every child patch by the min and max of its coefficients (Thm. 1) into
// per-child records, and in FP32 mode carry each patch's error bound and mark
// patches whose bound changes a decision (for k_refresh).
//
// Included by pcba_kernels.cuh after its small exact helpers (dev_binom,
// addrn, mulrn).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "pcba_device.cuh"

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

// FP32 re-centring of a dense constraint patch at a bisection.  The patch is
// stored as residuals r relative to an FP32 offset o.  With s = r_0 (its first
// stored coefficient): o + s = o' + t exactly (TwoSum, Knuth), d = fl(s - t),
// and the parent's residuals are shifted to fl(r - d) before the de Casteljau
// triangle, so the children are stored relative to o'.  Then
// o' + fl(r - d) = o + r - (d - (s - t)) + (fl(r - d) - (r - d)): the patch
// error grows by at most u |d| (1 + 2u) + u m' (m' = max |fl(r - d)|), which
// scales with the patch's range, not with its magnitude.
struct Recentre {
  float o, d;
};
__device__ __forceinline__ Recentre recentre(float o, float s) {
  const float on = __fadd_rn(o, s);
  const float bv = __fsub_rn(on, o);
  const float t = __fadd_rn(__fsub_rn(o, __fsub_rn(on, bv)), __fsub_rn(s, bv));
  return Recentre{on, __fsub_rn(s, t)};
}

// FP32 bounds of a re-centred child: the parent bound e, the shift d, the
// triangle over residuals of magnitude m (n levels), then [o + min - e,
// o + max + e] with directed rounding, the stored values o + min / o + max
// (round to nearest, for the mark) and the mark floor.
struct ChildBound {
  float ec, lo, hi, smin, smax, floor;
};
__device__ __forceinline__ ChildBound child_bound(float ep, float m, float d, int n, float o,
                                                  float mn, float mx) {
  ChildBound b;
  const float fn = (float)n;
  b.ec = __fadd_ru(__fadd_ru(__fadd_ru(fabsf(ep), __fmul_ru(m, (fn + 1.0f + 0x1p-10f) * 0x1p-24f)),
                             __fmul_ru(fabsf(d), 0x1p-24f * (1.0f + 0x1p-20f))),
                   (fn + 2.0f) * 0x1p-149f);
  b.lo = __fadd_rd(o, __fsub_rd(mn, b.ec));
  b.hi = __fadd_ru(o, __fadd_ru(mx, b.ec));
  b.smin = __fadd_rn(o, mn);
  b.smax = __fadd_rn(o, mx);
  // a refresh stores residuals rounded to FP32 (~u max |r| / 2) and adds the
  // FP64 conversion bound, which grows with the power-basis weights (up to
  // ~3^12 |value| 2^-45 for degree 12 on [-1,1]): below 8 u max |r| +
  // 2^-30 |value| a refresh would not pay
  b.floor = __fadd_ru(__fmul_ru(fmaxf(fabsf(mn), fabsf(mx)), 8.0f * 0x1p-24f),
                      __fmul_ru(fmaxf(fabsf(b.smin), fabsf(b.smax)), 0x1p-30f));
  return b;
}

// Thread i walks every fibre of constraint patch i (column i of a
// coefficient-major [C][pad] block); the left child overwrites the parent.
// The de Casteljau triangle (see split_fibre) is evaluated in place: after
// level k, q[0] is left_k and q[N-k] is right_(N-k), and both are stored at
// once, so only the N+1 working values stay in registers.  Writing left_k over
// the parent's coefficient k is safe: it was loaded before the first level.
// FP32 (RIG): every parent coefficient is first shifted by d (the patch's
// re-centring, see constraint_part), and the left child's coefficient 0 is
// stored too.
template <typename T, int N, bool RIG>
__device__ __forceinline__ void constraint_fibres(T* src, T* dR, size_t pad, int C, int stride,
                                                  int i, FibAcc<T>& a, T d = T(0)) {
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
      for (int j = 0; j <= N; ++j) {
        q[j] = addrn(q[j], -d);
        a.m = fmax(a.m, fabs(q[j]));
      }
      colL[0] = q[0];
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

// One cost fibre into shared staging buffers (same in-place triangle).  The
// extremes are kept in the patch's own type (a min or max of stored values is
// exact in it): in FP32 this keeps the long per-fibre chains off the FP64 units.
template <typename T, int N>
__device__ __forceinline__ void cost_fibre(const T* src, T* sL, T* sR, int base, int stride,
                                           T (&v)[5]) {
  T q[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    q[j] = src[base + j * stride];
    v[4] = max(v[4], abs(q[j]));
  }
  sL[base] = q[0];
  sR[base + N * stride] = q[N];
  v[0] = max(v[0], -q[0]);
  v[1] = max(v[1], q[0]);
  v[2] = max(v[2], -q[N]);
  v[3] = max(v[3], q[N]);
#pragma unroll
  for (int k = 1; k <= N; ++k) {
#pragma unroll
    for (int j = 0; j <= N - k; ++j) q[j] = mulrn(addrn(q[j], q[j + 1]), T(0.5));
    sL[base + k * stride] = q[0];
    sR[base + (N - k) * stride] = q[N - k];
    v[0] = max(v[0], -q[0]);
    v[1] = max(v[1], q[0]);
    v[2] = max(v[2], -q[N - k]);
    v[3] = max(v[3], q[N - k]);
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

// With NFIX > 0 every patch of the batch has degree NFIX along every axis: the
// kernel is built for that degree only (a smaller body for the instruction
// cache); NFIX = 0 dispatches on n at run time.
template <int NMAX, int NFIX, typename F>
__device__ __forceinline__ void dispatch_fixed(int n, F&& f) {
  if constexpr (NFIX > 0) {
    (void)n;
    f(std::integral_constant<int, NFIX>{});
  } else {
    dispatch_degree<NMAX>(n, f);
  }
}

__device__ __forceinline__ int axis_stride(const int* deg, int l, int r) {
  int s = 1;
  for (int q = r + 1; q < l; ++q) s *= deg[q] + 1;
  return s;
}


// FP32 error bounds are stored with a mark in the sign bit, set when the bound
// itself changes a decision of Def. 3 for this patch: the stored values (min s,
// max s, offset included) would decide it (infeasible, feasible, or inside
// the equality window) but the enclosure [lo, hi] does not.  The magnitude is
// the bound; k_refresh recomputes marked patches.  floor: about what a refresh
// could reach (its rounding of the stored values and the FP64 conversion
// bound) times 8; a patch whose bound is below it is left alone.
__device__ __forceinline__ float mark_err(float e, float smin, float smax, float lo, float hi,
                                          int fam, float eqt, float floor) {
  if (e <= floor) return e;
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
  int p, kL, kR;       // problem, logical positions of the children
  unsigned sL, sR;     // their physical slots
  uint4* list;
  unsigned* count;
  unsigned cap;
};

// A mark: problem, logical child position, physical slot (the refresh runs
// beside the compaction, which moves map entries), family | patch << 2.
__device__ __forceinline__ uint4 make_mark(int p, int k, unsigned slot, int fam, int ip) {
  return make_uint4((unsigned)p, (unsigned)k, slot, (unsigned)fam | ((unsigned)ip << 2));
}

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
    if (q < m.cap) m.list[q] = make_mark(m.p, m.kL, m.sL, fam, ip);
  }
  if (mR) {
    const unsigned q = base + __popc(bl) + __popc(br & below);
    if (q < m.cap) m.list[q] = make_mark(m.p, m.kR, m.sR, fam, ip);
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

// Layout of the cost patch along the bisection axis r: coefficient count,
// degree, stride of the axis, fibre count, block of one outer index, offset
// in the item.  The TMA kernel loads it with the per-problem context, before
// the wait for the unit's copies, so its reads overlap that wait.
struct CostGeom {
  int cp, n, stride, nf, blk;
  long long off;
};
__device__ __forceinline__ CostGeom cost_geom(const ProbDesc* D, int r) {
  CostGeom g;
  g.cp = D->cp;
  g.n = D->P[r];
  g.stride = axis_stride(D->P, D->l, r);
  g.nf = g.cp / (g.n + 1);
  g.blk = (g.n + 1) * g.stride;
  g.off = D->off_cost;
  return g;
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
template <typename T, int NMAX, int NFIX = 0>
__device__ void cost_part(const CostGeom& cg, const char* head, char* parent, char* right,
                          ChildRec* recL, ChildRec* recR, T* stage, const MarkCtx& mk,
                          double cost_thr) {
  const int lane = threadIdx.x & 31;
  const int cp = cg.cp, n = cg.n, stride = cg.stride, nf = cg.nf, blk = cg.blk;
  const T* src = (const T*)(head + cg.off);
  T* dstL = (T*)(parent + cg.off);
  T* dstR = (T*)(right + cg.off);
  T* sL = stage;
  T* sR = stage + cp;
  double O = 0.0, ep = 0.0;
  if constexpr (sizeof(T) == 4) {
    O = *(const double*)(head + 32);
    ep = (double)*(const float*)(head + 40);
  }
  T vt[5] = {T(-INFINITY), T(-INFINITY), T(-INFINITY), T(-INFINITY), T(0)};
  for (int f = lane; f < nf; f += 32) {
    const int o = f / stride;
    const int base = o * blk + (f - o * stride);
    dispatch_fixed<NMAX, NFIX>(n, [&](auto nc) {
      cost_fibre<T, decltype(nc)::value>(src, sL, sR, base, stride, vt);
    });
  }
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vt[q] = max(vt[q], __shfl_xor_sync(0xffffffffu, vt[q], o));
  double v[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) v[q] = (double)vt[q];
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
      recL->perr = __float_as_uint((float)efs[0]);
      recR->perr = __float_as_uint((float)efs[1]);
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
    Recentre rc{0.0f, 0.0f};
    float* opp = nullptr;
    if constexpr (RIG) {
      opp = (float*)(parent + (fam ? D->off_oh : D->off_og));
      rc = recentre(opp[i], (float)src[i]);  // src[i]: coefficient 0 of patch i
    }
    dispatch_degree<NMAX>(n, [&](auto nc) {
      constraint_fibres<T, decltype(nc)::value, RIG>(src, dR, pad, C, stride, i, a, T(rc.d));
    });
    T loL, hiL, loR, hiR;
    if constexpr (RIG) {
      float* ep = (float*)(parent + (fam ? D->off_eh : D->off_eg));
      float* er = (float*)(right + (fam ? D->off_eh : D->off_eg));
      const ChildBound bL = child_bound(ep[i], (float)a.m, rc.d, n, rc.o, (float)a.minL,
                                        (float)a.maxL);
      const ChildBound bR = child_bound(ep[i], (float)a.m, rc.d, n, rc.o, (float)a.minR,
                                        (float)a.maxR);
      loL = bL.lo;
      hiL = bL.hi;
      loR = bR.lo;
      hiR = bR.hi;
      const float eL = mark_err(bL.ec, bL.smin, bL.smax, loL, hiL, fam, eqt, bL.floor);
      const float eR = mark_err(bR.ec, bR.smin, bR.smax, loR, hiR, fam, eqt, bR.floor);
      ep[i] = eL;
      er[i] = eR;
      opp[i] = rc.o;
      ((float*)(right + (fam ? D->off_oh : D->off_og)))[i] = rc.o;
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


// Work unit = (problem, parent item k, tile t).  Tile 0 also splits the cost
// patch (warp 0) and the box; every tile splits up to PCBA_TPB constraint
// patches, 32 per warp.  Warps never wait for each other inside a unit: each
// warp publishes its bound maxima with fire-and-forget atomics into the two
// child records; p_up is computed from the finished records by k_pup.
//
// Each block takes one contiguous range of units, so consecutive units mostly
// belong to one problem; the problem's descriptor and step state are copied to
// shared memory once per problem.
// Physical slot of the right child of logical parent k: the k-th free slot
// popped from the stack (top first), then slots never used before.
__device__ __forceinline__ unsigned right_slot(const Engine& E, long long slot_off, int k,
                                               int ftop, int hw) {
  return k < ftop ? E.fstack[slot_off + ftop - 1 - k] : (unsigned)(hw + (k - ftop));
}

template <typename T, int NMAX>
__global__ void __launch_bounds__(PCBA_TPB) k2_subdivide(Engine E) {
  if (blockIdx.x == 0 && threadIdx.x == 0) E.plan->kr_par = E.plan->steps_global & 1;  // for k_refresh
  extern __shared__ __align__(16) unsigned char k2stage[];
  __shared__ __align__(16) ProbDesc sD;
  __shared__ int sK, sR, sFtop, sHw;
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
        sFtop = E.state[p].ftop;
        sHw = E.state[p].hw;
      }
      __syncthreads();
    }
    const ProbDesc* D = &sD;
    const int K = sK, r = sR, tiles = D->tiles;
    const unsigned local = u - pbeg;
    const int k = (int)(local / (unsigned)tiles);
    const int t = (int)(local - (unsigned)k * tiles);
    const unsigned pslot = E.map[D->slot_off + k];
    const unsigned rslot = right_slot(E, D->slot_off, k, sFtop, sHw);
    char* parent = E.arena + D->list_off + (size_t)pslot * D->item_bytes;
    char* right = E.arena + D->list_off + (size_t)rslot * D->item_bytes;
    ChildRec* recL = E.rec + D->slot_off + k;
    ChildRec* recR = E.rec + D->slot_off + k + K;
    const MarkCtx mk{p, k, k + K, pslot, rslot, E.marks + (size_t)mpar * E.mark_cap,
                     &E.plan->mark_count[mpar], E.mark_cap};
    if (t == 0 && warp == 0) {
      cost_part<T, NMAX>(cost_geom(D, r), parent, parent, right, recL, recR, (T*)k2stage, mk,
                         cost_thr);
      if (lane == 0) {
        E.map[D->slot_off + k + K] = rslot;
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

// A warp work unit u = (problem p, parent item k, column group g), resolved by
// the lane that issues its copies and kept in the stage's header, together
// with the physical slots of the parent and of the right child, so that the
// warp that computes it reads everything from shared memory.
struct WarpUnit {
  int p, k, g, fam, x;
  unsigned pslot, rslot;
  int pad;
};

// Per-problem values the issuing lane needs, reloaded when the problem changes.
struct IssueCtx {
  int p;
  unsigned beg, end;
  int tiles, groups_g, groups_h, K, ftop, hw;
  long long slot_off;
};

__device__ __forceinline__ WarpUnit resolve_unit(const Engine& E, unsigned u, IssueCtx& c) {
  if (u >= c.end || u < c.beg) {
    const int p = find_problem(E.k2_pre, E.np, u);
    const ProbDesc* D = E.desc + p;
    const ProbState* S = E.state + p;
    c.p = p;
    c.beg = E.k2_pre[p];
    c.end = E.k2_pre[p + 1];
    c.tiles = D->tiles;
    c.groups_g = D->groups_g;
    c.groups_h = D->groups_h;
    c.slot_off = D->slot_off;
    c.K = S->K;
    c.ftop = S->ftop;
    c.hw = S->hw;
  }
  const unsigned local = u - c.beg;
  WarpUnit w;
  w.p = c.p;
  w.k = (int)(local / (unsigned)c.tiles);
  w.g = (int)(local - (unsigned)w.k * c.tiles);
  if (w.g < c.groups_g) {
    w.fam = 0;
    w.x = w.g * 32;
  } else if (w.g < c.groups_g + c.groups_h) {
    w.fam = 1;
    w.x = (w.g - c.groups_g) * 32;
  } else {
    w.fam = -1;  // cost-only unit of a problem without constraints
    w.x = 0;
  }
  w.pslot = E.map[c.slot_off + w.k];
  w.rslot = right_slot(E, c.slot_off, w.k, c.ftop, c.hw);
  w.pad = 0;
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
  const char* item = E.arena + D->list_off + (size_t)w.pslot * D->item_bytes;
  const unsigned hb = w.g == 0 ? head_bytes(D, (unsigned)sizeof(T)) : 0u;
  if (w.fam < 0) {
    mbar_arrive_expect_tx(bar, hb);
    bulk_load(head, item, hb, bar);
    return;
  }
  const int C = w.fam ? D->ch : D->cg;
  unsigned bytes = (unsigned)C * 32u * (unsigned)sizeof(T) + hb;
  if (sizeof(T) == 4) bytes += 256u;
  mbar_arrive_expect_tx(bar, bytes);
  if (hb) bulk_load(head, item, hb, bar);
  const char* tm = (const char*)E.tmaps + ((size_t)w.p * 2 + w.fam) * 128;
  tma_load_3d(stage, tm, w.x, 0, (int)w.pslot, bar);
  if (sizeof(T) == 4) {
    // the group's 32 error bounds, then its 32 offsets
    bulk_load(estage, item + (w.fam ? D->off_eh : D->off_eg) + (size_t)w.x * 4, 128u, bar);
    bulk_load(estage + 32, item + (w.fam ? D->off_oh : D->off_og) + (size_t)w.x * 4, 128u, bar);
  }
}

// Fibres of one column (lane) of a staged [C][32] block: loads from shared
// memory, children stored straight to global memory (coalesced across lanes).
//
// The triangle keeps its sums unhalved: level k holds 2^k times the de
// Casteljau values, and each child coefficient is scaled by 2^-k only when it
// is stored.  Scaling by a power of two commutes with round-to-nearest outside
// the subnormal and overflow ranges, so every stored value equals the halved
// triangle's bit for bit there; in the subnormal range the unhalved sums lose
// nothing (the FP32 bound's 2^-149 term per level covers the final scaling).
// Two fibres are processed together for instruction-level parallelism.
template <typename T, int N, bool RIG, int NF>
__device__ __forceinline__ void staged_fibre_group(const T* sl, T* gL, T* gR, size_t pad,
                                                   size_t st, int blk, int stride, int f,
                                                   FibAcc<T>& a, T d) {
  int c0[NF];
  T q[NF][N + 1];
#pragma unroll
  for (int h = 0; h < NF; ++h) {
    const int ff = f + h;
    const int o = ff / stride;
    c0[h] = o * blk + (ff - o * stride);
    const T* sc = sl + c0[h] * 32;
#pragma unroll
    for (int j = 0; j <= N; ++j) q[h][j] = sc[j * stride * 32];
  }
#pragma unroll
  for (int h = 0; h < NF; ++h) {
    if constexpr (RIG) {
      // FP32: the re-centring shift (see recentre); left_0 is stored shifted
#pragma unroll
      for (int j = 0; j <= N; ++j) {
        q[h][j] = addrn(q[h][j], -d);
        a.m = fmax(a.m, fabs(q[h][j]));
      }
      gL[(size_t)c0[h] * pad] = q[h][0];
    }
    // (FP64: left_0 = f_0 already sits in the parent slot the left child overwrites)
    gR[(size_t)c0[h] * pad + N * st] = q[h][N];
    a.minL = fmin(a.minL, q[h][0]);
    a.maxL = fmax(a.maxL, q[h][0]);
    a.minR = fmin(a.minR, q[h][N]);
    a.maxR = fmax(a.maxR, q[h][N]);
  }
  T scale = T(1);
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    scale = scale * T(0.5);
#pragma unroll
    for (int j = 0; j <= N - k; ++j)
#pragma unroll
      for (int h = 0; h < NF; ++h) q[h][j] = addrn(q[h][j], q[h][j + 1]);
#pragma unroll
    for (int h = 0; h < NF; ++h) {
      const T l = mulrn(q[h][0], scale);
      const T r = mulrn(q[h][N - k], scale);
      gL[(size_t)c0[h] * pad + k * st] = l;
      gR[(size_t)c0[h] * pad + (N - k) * st] = r;
      a.minL = fmin(a.minL, l);
      a.maxL = fmax(a.maxL, l);
      a.minR = fmin(a.minR, r);
      a.maxR = fmax(a.maxR, r);
    }
  }
}

template <typename T, int N, bool RIG>
__device__ __forceinline__ void staged_fibres(const T* stage, T* gL, T* gR, size_t pad, int C,
                                              int stride, int lane, FibAcc<T>& a, T d = T(0)) {
  const int nf = C / (N + 1);
  const int blk = (N + 1) * stride;
  const size_t st = (size_t)stride * pad;
  const T* sl = stage + lane;
  int f = 0;
#pragma unroll 1
  for (; f + 1 < nf; f += 2)
    staged_fibre_group<T, N, RIG, 2>(sl, gL, gR, pad, st, blk, stride, f, a, d);
  if (f < nf) staged_fibre_group<T, N, RIG, 1>(sl, gL, gR, pad, st, blk, stride, f, a, d);
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
template <typename T, int NMAX, int NFIX = 0>
__global__ void __launch_bounds__(256) k2_subdivide_tma(Engine E, int stages, int stage_elems,
                                                        int cpmax) {
  if (blockIdx.x == 0 && threadIdx.x == 0) E.plan->kr_par = E.plan->steps_global & 1;  // for k_refresh
  constexpr bool RIG = sizeof(T) == 4;
  extern __shared__ __align__(128) unsigned char k2t_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  // per warp: stages x (stage_elems T + 32 floats + head), then 2*cpmax T of cost
  // staging; head = box, cost meta and cost patch of the parent (group 0),
  // with the unit's WarpUnit header in its last 32 bytes
  const size_t head_cap = ((size_t)64 + (size_t)cpmax * sizeof(T) + 32 + 127) / 128 * 128;
  const size_t stage_bytes = (size_t)stage_elems * sizeof(T) + PCBA_ESTAGE_BYTES + head_cap;
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
  IssueCtx ic;
  ic.beg = 1u;
  ic.end = 0u;
  // prologue
  for (int j = 0; j < J && j < stages; ++j) {
    if (lane == 0) {
      const WarpUnit w = resolve_unit(E, first + (unsigned)j * wpb, ic);
      unsigned char* st = wb + (size_t)j * stage_bytes;
      unsigned char* head = st + (size_t)stage_elems * sizeof(T) + PCBA_ESTAGE_BYTES;
      *(WarpUnit*)(head + head_cap - 32) = w;
      issue_unit<T>(E, w, (T*)st, (float*)(st + (size_t)stage_elems * sizeof(T)), head, &bars[j]);
    }
  }
  __syncwarp();
  // per-problem context, reloaded only when the unit's problem changes
  int cx_p = -1, cx_K = 0, cx_r = 0;
  CostGeom cx_cost{};
  char* cx_list = nullptr;
  long long cx_ib = 0, cx_slot = 0;
  // family fields of the unit's family (units of one problem are ordered
  // inequality groups first, then equality groups)
  int cx_fam = -1, cx_cnt = 0, cx_C = 0, cx_n = 0, cx_stride = 1;
  size_t cx_pad = 0;
  long long cx_off = 0, cx_offe = 0, cx_offo = 0;
  for (int j = 0; j < J; ++j) {
    const int s = j % stages;
    const unsigned parity = (unsigned)(j / stages) & 1u;
    unsigned char* st = wb + (size_t)s * stage_bytes;
    const T* stage = (const T*)st;
    const float* estage = (const float*)(st + (size_t)stage_elems * sizeof(T));
    const WarpUnit w =
        *(const WarpUnit*)(st + (size_t)stage_elems * sizeof(T) + PCBA_ESTAGE_BYTES + head_cap - 32);
    const ProbDesc* D = E.desc + w.p;
    if (w.p != cx_p) {
      const ProbState* S = E.state + w.p;
      cx_p = w.p;
      cx_K = S->K;
      cx_r = S->r;
      cx_list = E.arena + D->list_off;
      cx_ib = D->item_bytes;
      cx_slot = D->slot_off;
      cx_fam = -1;
      cx_cost = cost_geom(D, cx_r);
    }
    if (w.fam >= 0 && w.fam != cx_fam) {
      const int fam = w.fam;
      const int* deg = fam ? D->H : D->G;
      cx_fam = fam;
      cx_cnt = fam ? D->beta : D->alpha;
      cx_C = fam ? D->ch : D->cg;
      cx_pad = fam ? D->bpad : D->apad;
      cx_off = fam ? D->off_h : D->off_g;
      cx_offe = fam ? D->off_eh : D->off_eg;
      cx_offo = fam ? D->off_oh : D->off_og;
      cx_n = deg[cx_r];
      cx_stride = axis_stride(deg, D->l, cx_r);
    }
    const int K = cx_K, r = cx_r;
    const unsigned rslot = w.rslot;
    char* parent = cx_list + (size_t)w.pslot * cx_ib;
    char* right = cx_list + (size_t)rslot * cx_ib;
    ChildRec* recL = E.rec + cx_slot + w.k;
    ChildRec* recR = E.rec + cx_slot + w.k + K;
    const MarkCtx mk{w.p, w.k, w.k + K, w.pslot, rslot, E.marks + (size_t)mpar * E.mark_cap,
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
      const unsigned char* head = st + (size_t)stage_elems * sizeof(T) + PCBA_ESTAGE_BYTES;
      cost_part<T, NMAX, NFIX>(cx_cost, (const char*)head, parent, right, recL, recR, cost_stage,
                               mk, cost_thr);
      if (lane == 0) {
        E.map[cx_slot + w.k + K] = rslot;
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
      const int cnt = cx_cnt;
      const size_t pad = cx_pad;
      const int C = cx_C;
      const long long off = cx_off;
      const int n = cx_n;
      const int stride = cx_stride;
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
        // FP32: re-centre on the staged coefficient 0 of this lane's patch
        Recentre rc{0.0f, 0.0f};
        if constexpr (RIG) rc = recentre(estage[32 + lane], (float)stage[lane]);
        dispatch_fixed<NMAX, NFIX>(n, [&](auto nc) {
          staged_fibres<T, decltype(nc)::value, RIG>(stage, gL, gR, pad, C, stride, lane, a,
                                                     T(rc.d));
        });
        T loL, hiL, loR, hiR;
        if constexpr (RIG) {
          const ChildBound bL = child_bound(estage[lane], (float)a.m, rc.d, n, rc.o,
                                            (float)a.minL, (float)a.maxL);
          const ChildBound bR = child_bound(estage[lane], (float)a.m, rc.d, n, rc.o,
                                            (float)a.minR, (float)a.maxR);
          loL = bL.lo;
          hiL = bL.hi;
          loR = bR.lo;
          hiR = bR.hi;
          const float eL = mark_err(bL.ec, bL.smin, bL.smax, loL, hiL, fam, eqt, bL.floor);
          const float eR = mark_err(bR.ec, bR.smin, bR.smax, loR, hiR, fam, eqt, bR.floor);
          ((float*)(parent + cx_offe))[i] = eL;
          ((float*)(right + cx_offe))[i] = eR;
          ((float*)(parent + cx_offo))[i] = rc.o;
          ((float*)(right + cx_offo))[i] = rc.o;
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
      const WarpUnit wn = resolve_unit(E, first + (unsigned)(j + stages) * wpb, ic);
      unsigned char* head = st + (size_t)stage_elems * sizeof(T) + PCBA_ESTAGE_BYTES;
      *(WarpUnit*)(head + head_cap - 32) = wn;
      issue_unit<T>(E, wn, (T*)st, (float*)(st + (size_t)stage_elems * sizeof(T)), head, &bars[s]);
    }
    __syncwarp();
  }
  // every issued unit was consumed above: no copy is in flight at exit
}

