// Subdivision and bounds of linear-family problems (pcba_create_linear).
//
// The inequalities of such a problem are g_i = c_i + sum_m w_im s_m with K
// shared polynomials s_m.  The Bernstein transform is linear and maps a
// constant to that constant on every coefficient (Sec. II-D, Eq. (BF)), so
// on every box the coefficients of g_i are c_i + sum_m w_im b_mj, b_m the
// patch of s_m: an item stores the K patches b_m, and each constraint's
// min / max coefficient (Alg. 3) is computed from them when the box is
// bounded.  A constraint whose bound proves g_i <= 0 on a box is cleared from
// the item's activity bits: the Bernstein coefficients of a sub-box are convex
// combinations of those of the box (Sec. II-E), so its range stays inside
// [min, max] of the box and the constraint holds on every descendant.  Only
// active constraints are evaluated, and most are decided by an interval
// bound from the ranges of the shared patches before any coefficient loop.
//
// Rigour in FP32.  A shared patch is stored as FP32 residuals r_mj relative to
// an FP64 offset O_m (re-centred on the middle of its range at every
// bisection, as the cost patch), with a bound e_m: |O_m + r_mj - b_mj| <= e_m.
// Near an obstacle's boundary the terms c_i, ||F||^2 and 2 o_i . F are large
// and cancel, so the constant part kappa_i = c_i + sum_m w_im O_m is formed in
// FP64 from the FP64 row (error <= 2^-50 A64, A64 = |c| + sum_m |w_m| |O_m|,
// for K <= 4) and rounded to FP32; the FP32 work only carries residuals.
// With A = |kappa| + sum_m |w_m| max_j |r_mj| (the child's residuals), the
// computed coefficient v_j = fma(w_K-1, r_K-1,j, ... fma(w_0, r_0j, kappa))
// differs from the exact c_i + sum_m w_im b_mj by at most
//     K u A (1 + u)^K            the K roundings of the fused chain,
//   + 2.02 u A                   rounding of kappa and of w to FP32,
//   + (1 + 1.01 u) sum |w_m| e_m stored-patch errors,
//   + 2^-50 A64                  the FP64 constant term,
// and the interval bound kappa + sum_m min/max(w_m mn_m, w_m mx_m) (mn_m, mx_m
// the exact extremes of the stored residuals) by at most 2K u A plus the same
// other terms; subnormal results add at most 2^-149 each.  So
//     E = (2K + 3) u A + (1 + 2^-20) sum |w_m| e_m + 2^-50 A64 + (2K + 2) 2^-149,
// computed with upward rounding, bounds both, and [min_j v_j - E, max_j v_j + E]
// encloses the exact coefficient range of the constraint on the box.  (FP64
// mode stores plain patches, O_m = 0, and is plain arithmetic as the paper's.)
//
// Work unit = (problem, parent item, chunk of PCBA_LIN_WORDS activity words),
// one warp each.  Every unit subdivides the K shared patches of its parent in
// shared memory (from the copy of this step's parity); chunk 0 also writes the
// children's patches (to the other copy), splits the cost patch and the box
// and updates the slot map.  A unit compacts the active constraints of its
// chunk, bounds each on both children and writes the children's activity
// words; the bound maxima go to the child records with one atomic per warp.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "pcba_device.cuh"

// Bytes of shared memory one warp of k2_subdivide_lin uses.
template <typename T, int K>
__host__ __device__ constexpr size_t lin_warp_bytes(int cgmax, int cpmax) {
  return (((size_t)K * cgmax + 8 * (size_t)cgmax + 2 * (size_t)cpmax) * sizeof(T) +
          32 * PCBA_LIN_WORDS * sizeof(unsigned short) + 2 * PCBA_LIN_WORDS * sizeof(unsigned) +
          15) / 16 * 16;
}

// One fibre of shared patch m: parent coefficients base + j * stride of src,
// children written to coefficient-major [C][4] buffers at slot m.
template <typename T, int N>
__device__ __forceinline__ void lin_fibre(const T* src, T* dL, T* dR, int base, int stride,
                                          int m) {
  T q[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) q[j] = src[base + j * stride];
  dL[(size_t)base * 4 + m] = q[0];
  dR[(size_t)(base + N * stride) * 4 + m] = q[N];
#pragma unroll
  for (int k = 1; k <= N; ++k) {
#pragma unroll
    for (int j = 0; j <= N - k; ++j) q[j] = mulrn(addrn(q[j], q[j + 1]), T(0.5));
    dL[(size_t)(base + k * stride) * 4 + m] = q[0];
    dR[(size_t)(base + (N - k) * stride) * 4 + m] = q[N - k];
  }
}

// Directed sums of the FP32 bounds; FP64 mode is plain arithmetic (E = 0).
__device__ __forceinline__ float add_up(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ double add_up(double a, double b) { return a + b; }
__device__ __forceinline__ float sub_dn(float a, float b) { return __fsub_rd(a, b); }
__device__ __forceinline__ double sub_dn(double a, double b) { return a - b; }

__device__ __forceinline__ float lin_wmax(float v) {
  return okey32_dec(__reduce_max_sync(0xffffffffu, okey32(v)));
}
__device__ __forceinline__ float lin_wmin(float v) {
  return okey32_dec(__reduce_min_sync(0xffffffffu, okey32(v)));
}
__device__ __forceinline__ double lin_wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double lin_wmin(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Coefficient range of c + sum_m w_m s_mj over the C coefficients of one
// child (coefficient-major, 4 slots per coefficient).
// (Two partial extremes per bound, for independent dependency chains.)
template <typename T, int K>
__device__ __forceinline__ T lin_coef(const T* s, T c, const T (&w)[K]) {
  T v = c;
#pragma unroll
  for (int m = 0; m < K; ++m) v = fma(w[m], s[m], v);
  return v;
}
template <typename T, int K>
__device__ __forceinline__ void lin_full_range(const T* sc, int C, T c, const T (&w)[K], T& lo,
                                               T& hi) {
  T lo0 = T(INFINITY), hi0 = T(-INFINITY), lo1 = T(INFINITY), hi1 = T(-INFINITY);
  int j = 0;
#pragma unroll 2
  for (; j + 1 < C; j += 2) {
    const T v0 = lin_coef<T, K>(sc + (size_t)j * 4, c, w);
    const T v1 = lin_coef<T, K>(sc + (size_t)(j + 1) * 4, c, w);
    lo0 = min(lo0, v0);
    hi0 = max(hi0, v0);
    lo1 = min(lo1, v1);
    hi1 = max(hi1, v1);
  }
  if (j < C) {
    const T v0 = lin_coef<T, K>(sc + (size_t)j * 4, c, w);
    lo0 = min(lo0, v0);
    hi0 = max(hi0, v0);
  }
  lo = min(lo0, lo1);
  hi = max(hi0, hi1);
}
// Both children at once (the same constraint on the two halves of a box).
template <typename T, int K>
__device__ __forceinline__ void lin_full_range2(const T* sl, const T* sr, int C, T c,
                                                const T (&w)[K], T& loL, T& hiL, T& loR,
                                                T& hiR) {
  T a0 = T(INFINITY), b0 = T(-INFINITY), a1 = T(INFINITY), b1 = T(-INFINITY);
#pragma unroll 2
  for (int j = 0; j < C; ++j) {
    const T v0 = lin_coef<T, K>(sl + (size_t)j * 4, c, w);
    const T v1 = lin_coef<T, K>(sr + (size_t)j * 4, c, w);
    a0 = min(a0, v0);
    b0 = max(b0, v0);
    a1 = min(a1, v1);
    b1 = max(b1, v1);
  }
  loL = a0;
  hiL = b0;
  loR = a1;
  hiR = b1;
}

// NFIX > 0: every patch of the batch has degree NFIX along every axis (a
// smaller kernel body); 0: any degree up to 16.
//
// Work units per item (ProbState::lin_tiles, set when the step is planned):
// while a problem's list is short its items are split into one unit per chunk
// of PCBA_LIN_WORDS activity words (near the root most constraints are still
// active); later one unit takes the whole item and skips the chunks whose
// summary bit is clear without reading them.
template <typename T, int K, int NFIX>
__global__ void __launch_bounds__(256, 3) k2_subdivide_lin(Engine E, int cgmax, int cpmax) {
  constexpr bool RIG = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char kls[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = kls + (size_t)warp * lin_warp_bytes<T, K>(cgmax, cpmax);
  T* sP = (T*)wb;                                   // parent patches [K][C]
  T* sC = sP + (size_t)K * cgmax;                   // children [2][C][4]
  T* cstage = sC + (size_t)8 * cgmax;               // cost staging [2][cp]
  unsigned short* sIdx = (unsigned short*)(cstage + (size_t)2 * cpmax);
  unsigned* sMw = (unsigned*)(sIdx + 32 * PCBA_LIN_WORDS);  // child words [2][LIN_WORDS]
  const unsigned units = E.plan->k2_units;
  const int par = E.plan->steps_global & 1;  // copy read this step; children go to par ^ 1
  const double cost_thr = E.params->opt_tol * (1.0 / 64.0);
  constexpr float u24 = 0x1p-24f;
  // per-problem context, reloaded when the unit's problem changes
  int cx_p = -1, cx_K = 0, cx_r = 0, cx_ftop = 0, cx_hw = 0, cx_chunks = 1, cx_tiles = 1;
  unsigned cx_beg = 0, cx_end = 0;
  const ProbDesc* D = nullptr;
  // units are fetched in batches from a counter (reset before every step), so
  // that the few heavy units - items with many active constraints - spread
  // over the whole GPU instead of lengthening one block's range
  for (;;) {
  unsigned ubeg = 0;
  if (lane == 0) ubeg = atomicAdd(&E.plan->lin_next, (unsigned)PCBA_LIN_BATCH);
  ubeg = __shfl_sync(0xffffffffu, ubeg, 0);
  if (ubeg >= units) break;
  const unsigned uend = min(units, ubeg + (unsigned)PCBA_LIN_BATCH);
  for (unsigned u = ubeg; u < uend; ++u) {
    if (u < cx_beg || u >= cx_end || cx_p < 0) {
      cx_p = find_problem(E.k2_pre, E.np, u);
      cx_beg = E.k2_pre[cx_p];
      cx_end = E.k2_pre[cx_p + 1];
      D = E.desc + cx_p;
      const ProbState* S = E.state + cx_p;
      cx_K = S->K;
      cx_r = S->r;
      cx_ftop = S->ftop;
      cx_hw = S->hw;
      cx_chunks = D->lin_chunks;
      cx_tiles = S->lin_tiles;
    }
    const int p = cx_p, Kl = cx_K, r = cx_r, chunks = cx_chunks, tiles = cx_tiles;
    const unsigned local = u - cx_beg;
    const int k = (int)(local / (unsigned)tiles);
    const int t = (int)(local - (unsigned)k * tiles);
    // the chunks of this unit
    const int c_beg = tiles == 1 ? 0 : t, c_end = tiles == 1 ? chunks : t + 1;
    const long long slot_off = D->slot_off;
    const unsigned pslot = E.map[slot_off + k];
    const unsigned rslot = right_slot(E, slot_off, k, cx_ftop, cx_hw);
    char* list = E.arena + D->list_off;
    char* parent = list + (size_t)pslot * D->item_bytes;
    char* right = list + (size_t)rslot * D->item_bytes;
    ChildRec* recL = E.rec + slot_off + k;
    ChildRec* recR = E.rec + slot_off + k + Kl;
    const int C = D->cg, apad = D->apad, l = D->l, mwords = D->mwords;
    const int n = D->G[r];
    const int stride = axis_stride(D->G, l, r);
    const int nf = C / (n + 1);
    const int blk = (n + 1) * stride;
    const MarkCtx mk{p, k, k + Kl, E.marks + (size_t)par * E.mark_cap, &E.plan->mark_count[par],
                     E.mark_cap};
    unsigned* pmask = (unsigned*)(parent + D->off_mask);
    unsigned* rmask = (unsigned*)(right + D->off_mask);
    // summaries: bit c of the parent's says whether chunk c has an active
    // constraint; the children's are written to the other word (kept only
    // for up to 64 chunks; beyond that every chunk is read)
    const bool summ = chunks <= 64;
    unsigned long long* sumL = (unsigned long long*)(parent + D->off_sum) + (par ^ 1);
    unsigned long long* sumR = (unsigned long long*)(right + D->off_sum) + (par ^ 1);
    const unsigned long long range =
        summ ? ((c_end >= 64 ? ~0ull : ((1ull << c_end) - 1ull)) & ~((1ull << c_beg) - 1ull)) : 0ull;
    const unsigned long long psum =
        summ ? *((const unsigned long long*)(parent + D->off_sum) + par) : ~0ull;
    const unsigned long long live = summ ? (psum & range) : ~0ull;
    // the unit holding chunk 0 writes the children's shared patches whenever
    // any chunk of the item is live
    const bool need_shared = c_beg == 0 ? psum != 0ull : live != 0ull;
    // chunk 0 splits the cost patch and the box, and updates the slot map
    auto split_cost_and_box = [&]() {
      cost_part<T, 16, NFIX>(cost_geom(D, r), parent, parent, right, recL, recR, cstage, mk,
                             cost_thr);
      if (lane == 0) {
        E.map[slot_off + k + Kl] = rslot;
        unsigned* iL = (unsigned*)parent;
        unsigned* iR = (unsigned*)right;
        for (int s = 0; s < l; ++s) iR[s] = iL[s];
        const unsigned v = iL[r];
        iL[r] = 2u * v;
        iR[r] = 2u * v + 1u;
      }
    };
    // the children's words of a chunk with no active constraint: zero (the
    // left child shares the parent's, already zero)
    auto clear_right = [&](int c0, int c1) {
      const int wb0 = c0 * PCBA_LIN_WORDS, wb1 = min(c1 * PCBA_LIN_WORDS, mwords);
      for (int q = wb0 + lane; q < wb1; q += 32) rmask[q] = 0u;
    };
    if (!need_shared) {
      // no active constraint in this unit's chunks (nor, for chunk 0, in the
      // item): the shared patches are not needed any more
      clear_right(c_beg, c_end);
      if (lane == 0 && summ) {
        if (tiles == 1) {
          *sumL = 0ull;
          *sumR = 0ull;
        } else {
          atomicAnd(sumL, ~range);
          atomicAnd(sumR, ~range);
        }
      }
      if (c_beg == 0) split_cost_and_box();
      __syncwarp();
      continue;
    }
    // ---- the parent's shared patches into shared memory
    const T* gsrc = (const T*)(parent + D->off_g + par * D->copy_g);
    const char* pmeta = parent + D->off_eg + par * D->copy_e;  // FP32: errors, then offsets
    float em[K];   // stored error bounds (FP32)
    float am[K];   // max |parent residual| per patch (FP32)
    double Om[K];  // FP64 offsets of the parent's stored patches (FP32; 0 in FP64)
#pragma unroll
    for (int m = 0; m < K; ++m) {
      float a = 0.0f;
      for (int j = lane; j < C; j += 32) {
        const T v = gsrc[(size_t)j * apad + m];
        sP[(size_t)m * C + j] = v;
        if constexpr (RIG) a = fmaxf(a, fabsf((float)v));
      }
      if constexpr (RIG) {
        am[m] = lin_wmax(a);
        em[m] = fabsf(((const float*)pmeta)[m]);
        Om[m] = ((const double*)(pmeta + 4LL * apad))[m];
      } else {
        am[m] = 0.0f;
        em[m] = 0.0f;
        Om[m] = 0.0;
      }
    }
    __syncwarp();
    // ---- de Casteljau at 1/2 on every fibre of every shared patch (Sec. II-E)
    T* sL = sC;
    T* sR = sC + (size_t)4 * cgmax;
    for (int f = lane; f < K * nf; f += 32) {
      const int m = f / nf;
      const int fi = f - m * nf;
      const int o = fi / stride;
      const int base = o * blk + (fi - o * stride);
      dispatch_fixed<16, NFIX>(n, [&](auto nc) {
        lin_fibre<T, decltype(nc)::value>(sP + (size_t)m * C, sL, sR, base, stride, m);
      });
    }
    __syncwarp();
    // ---- extremes of the children's patches, and their error bounds
    T mn[2][K], mx[2][K];
    float Mabs[2][K], ec[K];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T* sc = c ? sR : sL;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        T a = T(INFINITY), b = T(-INFINITY);
        for (int j = lane; j < C; j += 32) {
          const T v = sc[(size_t)j * 4 + m];
          a = min(a, v);
          b = max(b, v);
        }
        mn[c][m] = lin_wmin(a);
        mx[c][m] = lin_wmax(b);
        if constexpr (RIG)
          Mabs[c][m] = fmaxf(fabsf((float)mn[c][m]), fabsf((float)mx[c][m]));
        else
          Mabs[c][m] = 0.0f;
      }
    }
#pragma unroll
    for (int m = 0; m < K; ++m) {
      if constexpr (RIG) {
        const float fn = (float)n;
        ec[m] = __fadd_ru(__fadd_ru(em[m], __fmul_ru(am[m], fn * u24)), fn * 0x1p-149f);
      } else {
        ec[m] = 0.0f;
      }
    }
    // ---- chunk 0: the children's shared patches, the cost patch, box and map
    if (c_beg == 0) {
      T* dL = (T*)(parent + D->off_g + (par ^ 1) * D->copy_g);
      T* dR = (T*)(right + D->off_g + (par ^ 1) * D->copy_g);
      if constexpr (RIG) {
        // FP32: each child patch re-centred on the middle of its range, as the
        // cost patch: stored r' = fl(r - mid) (error <= u |r'|, and r' lies in
        // [fl(mn - mid), fl(mx - mid)] since rounding is monotone), offset
        // O' = O + mid in FP64 (error <= 2^-53 |O'|)
        float mid[2][K];
        float enew[2][K];
        double On[2][K];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int m = 0; m < K; ++m) {
            const float md = __fmul_rn(__fadd_rn((float)mn[c][m], (float)mx[c][m]), 0.5f);
            const float Mr = fmaxf(fabsf(__fsub_rn((float)mn[c][m], md)),
                                   fabsf(__fsub_rn((float)mx[c][m], md)));
            mid[c][m] = md;
            On[c][m] = Om[m] + (double)md;
            const float eo = __double2float_ru(__dmul_ru(fabs(On[c][m]), 0x1p-52));
            enew[c][m] = __fadd_ru(__fadd_ru(__fadd_ru(ec[m], __fmul_ru(Mr, u24)), 0x1p-149f), eo);
          }
        for (int e = lane; e < C * K; e += 32) {
          const int j = e / K;
          const int m = e - j * K;
          float mL = mid[0][0], mR = mid[1][0];
#pragma unroll
          for (int q = 1; q < K; ++q)
            if (m == q) { mL = mid[0][q]; mR = mid[1][q]; }
          dL[(size_t)j * apad + m] = __fsub_rn((float)sL[(size_t)j * 4 + m], mL);
          dR[(size_t)j * apad + m] = __fsub_rn((float)sR[(size_t)j * 4 + m], mR);
        }
        if (lane < K) {
          float eL = enew[0][0], eR = enew[1][0];
          double oL = On[0][0], oR = On[1][0];
#pragma unroll
          for (int m = 1; m < K; ++m)
            if (lane == m) { eL = enew[0][m]; eR = enew[1][m]; oL = On[0][m]; oR = On[1][m]; }
          char* mL = parent + D->off_eg + (par ^ 1) * D->copy_e;
          char* mR = right + D->off_eg + (par ^ 1) * D->copy_e;
          ((float*)mL)[lane] = eL;
          ((float*)mR)[lane] = eR;
          ((double*)(mL + 4LL * apad))[lane] = oL;
          ((double*)(mR + 4LL * apad))[lane] = oR;
        }
      } else {
        for (int e = lane; e < C * K; e += 32) {
          const int j = e / K;
          const int m = e - j * K;
          dL[(size_t)j * apad + m] = sL[(size_t)j * 4 + m];
          dR[(size_t)j * apad + m] = sR[(size_t)j * 4 + m];
        }
      }
      split_cost_and_box();
    }
    T gmax[2] = {T(-INFINITY), T(-INFINITY)}, gmin[2] = {T(-INFINITY), T(-INFINITY)};
    bool mark[2] = {false, false};
    unsigned nfull = 0;      // coefficient-range evaluations of this lane
    unsigned npairs = 0;     // (child, active constraint) bounds of this unit
    const int Kw = K;
    unsigned long long bitsL = 0ull, bitsR = 0ull;  // children's non-empty chunks here
    for (int cc = c_beg; cc < c_end; ++cc) {
      if (summ && !((live >> cc) & 1ull)) {
        clear_right(cc, cc + 1);
        continue;
      }
      // ---- the active constraints of chunk cc, compacted
      const int w0 = cc * PCBA_LIN_WORDS;
      const int nw = min(PCBA_LIN_WORDS, mwords - w0);
      unsigned* pm = pmask + w0;
      unsigned* rm = rmask + w0;
      __syncwarp();  // the previous chunk's readers of sIdx and sMw are done
      const unsigned word = lane < nw ? pm[lane] : 0u;
      const unsigned cnt = __popc(word);
      unsigned incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned na = __shfl_sync(0xffffffffu, incl, 31);
      if (na == 0) {
        if (lane < nw) rm[lane] = 0u;
        continue;
      }
      {
        unsigned pos = incl - cnt, bits = word;
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1u;
          sIdx[pos++] = (unsigned short)(lane * 32 + b);
        }
      }
      if (lane < 2 * PCBA_LIN_WORDS) sMw[lane] = 0u;
      __syncwarp();
      npairs += 2u * na;
      for (unsigned q = lane; q < na; q += 32) {
        const int li = sIdx[q];
        const long long row = (D->lin_off + (long long)w0 * 32 + li) * PCBA_LIN_STRIDE;
        T cc, w[K];
        float E64 = 0.0f;  // FP32: bound of the FP64 rounding of the constant term
        if constexpr (RIG) {
          const float4 r0 = *(const float4*)(E.lin32 + row);
          const float4 r1 = *(const float4*)(E.lin32 + row + 4);
          const float rr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
  #pragma unroll
          for (int m = 0; m < K; ++m) w[m] = rr[1 + m];
          // the constant term c_i + sum_m w_im O_m of the coefficients relative
          // to the parent's offsets, in FP64 from the FP64 row: the large terms
          // cancel here, exactly enough, and the FP32 part only carries the
          // residuals (of the order of the box's range)
          const double* rw = E.lin64 + row;
          double kap = rw[0], a64 = fabs(rw[0]);
  #pragma unroll
          for (int m = 0; m < K; ++m) {
            kap = fma(rw[1 + m], Om[m], kap);
            a64 = fma(fabs(rw[1 + m]), fabs(Om[m]), a64);
          }
          cc = (float)kap;
          E64 = __double2float_ru(__dmul_ru(a64, 0x1p-50));
        } else {
          const double* rw = E.lin64 + row;
          cc = rw[0];
  #pragma unroll
          for (int m = 0; m < K; ++m) w[m] = rw[1 + m];
        }
        // E of the comment at the top of this file (0 in FP64 mode), and the
        // interval bound from the ranges of the shared patches, per child
        float Ee[2] = {0.0f, 0.0f}, Er[2] = {0.0f, 0.0f};
        T lo[2], hi[2], Et[2];
  #pragma unroll
        for (int c = 0; c < 2; ++c) {
          float Eb = 0.0f;
          if constexpr (RIG) {
            float A = fabsf((float)cc), ee = 0.0f;
  #pragma unroll
            for (int m = 0; m < K; ++m) {
              A = __fmaf_ru(fabsf((float)w[m]), Mabs[c][m], A);
              ee = __fmaf_ru(fabsf((float)w[m]), ec[m], ee);
            }
            const float kk = (float)(2 * Kw + 2);
            Er[c] = __fmul_ru((kk + 1.0f) * u24, A);
            Ee[c] = ee;
            Eb = __fadd_ru(__fadd_ru(__fadd_ru(Er[c], __fmul_ru(ee, 1.0f + 0x1p-20f)), E64),
                           kk * 0x1p-149f);
          }
          Et[c] = T(Eb);
          T a = cc, b = cc;
  #pragma unroll
          for (int m = 0; m < K; ++m) {
            const T x = w[m] * mn[c][m], y = w[m] * mx[c][m];
            a += min(x, y);
            b += max(x, y);
          }
          lo[c] = a;
          hi[c] = b;
        }
        // undecided by the interval: the coefficient range itself (Alg. 3)
        const bool needL = !(add_up(hi[0], Et[0]) <= T(0)) && !(sub_dn(lo[0], Et[0]) > T(0));
        const bool needR = !(add_up(hi[1], Et[1]) <= T(0)) && !(sub_dn(lo[1], Et[1]) > T(0));
        if (needL && needR) {
          lin_full_range2<T, K>(sL, sR, C, cc, w, lo[0], hi[0], lo[1], hi[1]);
          nfull += 2;
        } else if (needL) {
          lin_full_range<T, K>(sL, C, cc, w, lo[0], hi[0]);
          nfull += 1;
        } else if (needR) {
          lin_full_range<T, K>(sR, C, cc, w, lo[1], hi[1]);
          nfull += 1;
        }
  #pragma unroll
        for (int c = 0; c < 2; ++c) {
          const T up = add_up(hi[c], Et[c]), dn = sub_dn(lo[c], Et[c]);
          const bool sat = up <= T(0);
          const bool inf = dn > T(0);
          if (!sat) {
            atomicOr(&sMw[c * PCBA_LIN_WORDS + (li >> 5)], 1u << (li & 31));
            gmax[c] = max(gmax[c], up);
            gmin[c] = max(gmin[c], dn);
          }
          if constexpr (RIG) {
            // the bound changed a decision the stored coefficients make: mark
            // the child's shared patches for a refresh if their errors are the
            // larger part of the bound
            const bool flip = (hi[c] <= T(0)) != sat || (lo[c] > T(0)) != inf;
            if (flip && Ee[c] > Er[c]) mark[c] = true;
          }
        }
      }

      __syncwarp();
      if (lane < nw) {
        pm[lane] = sMw[lane];                      // left child: in place (this unit's words)
        rm[lane] = sMw[PCBA_LIN_WORDS + lane];     // right child
      }
      const bool keepL = __any_sync(0xffffffffu, lane < nw && sMw[lane] != 0u);
      const bool keepR = __any_sync(0xffffffffu, lane < nw && sMw[PCBA_LIN_WORDS + lane] != 0u);
      if (cc < 64) {
        if (keepL) bitsL |= 1ull << cc;
        if (keepR) bitsR |= 1ull << cc;
      }
    }
    // ---- the children's summaries for this unit's chunks
    if (lane == 0 && summ) {
      if (tiles == 1) {
        *sumL = bitsL;
        *sumR = bitsR;
      } else {
        const unsigned long long tb = 1ull << t;
        if (bitsL) atomicOr(sumL, tb); else atomicAnd(sumL, ~tb);
        if (bitsR) atomicOr(sumR, tb); else atomicAnd(sumR, ~tb);
      }
    }
    // ---- bound maxima of the children, counters, refresh marks
    if (npairs > 0) {
      const unsigned full = __reduce_add_sync(0xffffffffu, nfull);
      if (lane == 0) {
        atomicAdd(&E.plan->lin_pairs, (unsigned long long)npairs);
        atomicAdd(&E.plan->lin_full, (unsigned long long)full);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T gx = lin_wmax(gmax[c]);
        const T gn = lin_wmax(gmin[c]);
        ChildRec* rc = c ? recR : recL;
        if (lane == 0 && gx > T(-INFINITY)) {
          atomicMax(&rc->gmaxmax, okey((double)gx));
          atomicMax(&rc->gminmax, okey((double)gn));
        }
      }
    }
    if constexpr (RIG) {
      const bool bl = __any_sync(0xffffffffu, mark[0]);
      const bool br = __any_sync(0xffffffffu, mark[1]);
      append_marks(mk, bl && lane < K, br && lane < K, 0, lane);
    }
    __syncwarp();
  }
  }
}
