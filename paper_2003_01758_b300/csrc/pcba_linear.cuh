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
// and cancel, so the constant part kappa_i = c_i + sum_m w_im O_m is formed to
// about 48 bits and then rounded to FP32; the FP32 work only carries
// residuals.  It takes no FP64 operation (B300 issues FP64 at a small
// fraction of the FP32 rate): c, w and O are each split into two FP32 values
// (x = hi + lo to 2^-48 |x|), w_hi O_hi is formed exactly as p + e (fused
// multiply-add), c_hi + sum p_m is summed error-free (TwoSum, Knuth), and the
// small terms (c_lo, e, w_hi O_lo, w_lo O_hi, the TwoSum errors) in plain FP32.
// With A64 = |c| + sum_m |w_m| |O_m| the splits and the dropped w_lo O_lo cost
// at most (1 + 5K) 2^-48 A64 and the sum of the small terms (each at most
// 2^-24 A64 in size, (K + 3) 2^-24 A64 together, 4K roundings) at most
// 4K (K + 3) 2^-48 A64, so for K <= 4 the error before the final rounding is
// below 134 2^-48 A64 < 2^-40 A64; products and sums that underflow add at
// most (8K + 2) 2^-149.
// With A = |kappa| + sum_m |w_m| max_j |r_mj| (the child's residuals), the
// computed coefficient v_j = fma(w_K-1, r_K-1,j, ... fma(w_0, r_0j, kappa))
// differs from the exact c_i + sum_m w_im b_mj by at most
//     K u A (1 + u)^K            the K roundings of the fused chain,
//   + 2.02 u A                   rounding of kappa and of w to FP32,
//   + (1 + 1.01 u) sum |w_m| e_m stored-patch errors,
//   + 2^-40 A64 + (8K+2) 2^-149  the two-float constant term,
// and the interval bound kappa + sum_m min/max(w_m mn_m, w_m mx_m) (mn_m, mx_m
// the exact extremes of the stored residuals) by at most 2K u A plus the same
// other terms; subnormal results add at most 2^-149 each.  So
//     E = (2K + 3) u A + (1 + 2^-20) sum |w_m| e_m + 2^-40 A64 + (10K + 4) 2^-149,
// computed with upward rounding, bounds both, and [min_j v_j - E, max_j v_j + E]
// encloses the exact coefficient range of the constraint on the box.  (FP64
// mode stores plain patches, O_m = 0, and is plain arithmetic as the paper's.)
//
// Two kernels per bisection step:
//   k2_lin_split   one warp per parent item (items fetched in batches from a
//                  counter): splits the cost patch and the K shared patches
//                  (de Casteljau at 1/2, Sec. II-E) into the two children, a
//                  lane per fibre, re-centres every FP32 child patch on the
//                  middle of its range, and stores per child and patch the
//                  extremes of the stored values (with their error bound and
//                  offset), the box and the slot map; the cost bounds go to
//                  the child records.  The children's shared patches go to the
//                  copy of the other parity, so the parent's stay readable.
//                  An item whose live chunks (chunks of PCBA_LIN_WORDS
//                  activity words with an active constraint; at most 8) hold
//                  at most PCBA_LIN_LIGHT_MAX active constraints is bounded
//                  here from the children still staged in shared memory; the
//                  live chunks of the other items are grouped into windows of
//                  about PCBA_LIN_WIN active constraints; a single window is
//                  bounded here, several are queued as (item, window).
//   k2_lin_bound   one warp per queued (item, window): stages both children and
//                  bounds the window's constraints as the split kernel does.
// Bounding a window compacts its active constraints and bounds each on both
// children from the stored extremes (interval bound) or, where that is
// undecided, from the children's coefficients; it writes the children's
// activity words and its chunks' summary bits, and publishes the bound maxima
// with one atomic per warp.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "pcba_device.cuh"


// Per-patch metadata of a linear item, one block per copy (copy_e bytes apart):
//   FP32: error bound f32[apad] | offset f64[apad] | min f32[apad] | max f32[apad]
//   FP64: min f64[apad] | max f64[apad]
// (min and max are those of the stored values of each shared patch).
template <typename T>
struct LinMeta {
  __device__ __forceinline__ static float* err(char* m, int) { return (float*)m; }
  __device__ __forceinline__ static double* off(char* m, int a) { return (double*)(m + 4LL * a); }
  __device__ __forceinline__ static T* mn(char* m, int a) {
    return sizeof(T) == 4 ? (T*)(m + 12LL * a) : (T*)m;
  }
  __device__ __forceinline__ static T* mx(char* m, int a) {
    return sizeof(T) == 4 ? (T*)(m + 16LL * a) : (T*)(m + 8LL * a);
  }
};

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


// ---------------------------------------------------------------------------
// k2_lin_split: one warp per parent item
// ---------------------------------------------------------------------------

// NP coefficients of one position of NP patches stored coefficient-major
// (patch m at p[m]): one 16-byte (FP32) or two (FP64) loads when NP > 1.
template <typename T, int NP>
__device__ __forceinline__ void lin_load(const T* p, T (&v)[NP]) {
  if constexpr (NP == 1) {
    v[0] = p[0];
  } else if constexpr (sizeof(T) == 4) {
    const float4 a = *(const float4*)p;
    const float t[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int m = 0; m < NP; ++m) v[m] = t[m];
  } else {
    const double2 a = *(const double2*)p;
    const double2 b = *(const double2*)(p + 2);
    const double t[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
    for (int m = 0; m < NP; ++m) v[m] = t[m];
  }
}
template <typename T, int NP>
__device__ __forceinline__ void lin_store(T* p, const T (&v)[NP]) {
  if constexpr (NP == 1) {
    p[0] = v[0];
  } else if constexpr (sizeof(T) == 4) {
    float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int m = 0; m < NP; ++m) t[m] = v[m];
    *(float4*)p = make_float4(t[0], t[1], t[2], t[3]);
  } else {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int m = 0; m < NP; ++m) t[m] = v[m];
    *(double2*)p = make_double2(t[0], t[1]);
    *(double2*)(p + 2) = make_double2(t[2], t[3]);
  }
}

// Copies n1 elements of T from s1 to d1 and n2 from s2 to d2 (global to
// shared memory, all four 16-byte aligned) in 16-byte pieces, a lane's loads
// issued before its stores (U at a time); one warp.
template <typename T, int U>
__device__ __forceinline__ void lin_copy2(T* d1, const T* s1, int n1, T* d2, const T* s2, int n2,
                                          int lane) {
  constexpr int V = 16 / (int)sizeof(T);
  const int a = n1 / V, b = n2 / V, n = a + b;
  const float4* x1 = (const float4*)s1;
  const float4* x2 = (const float4*)s2;
  // the ragged ends (fewer than V elements each, lanes 0.. and 8..) are read
  // with the first pieces
  const int r1 = n1 - a * V, r2 = n2 - b * V;
  T t = T(0);
  if (lane < r1) t = s1[a * V + lane];
  else if (lane >= 8 && lane - 8 < r2) t = s2[b * V + lane - 8];
  for (int e0 = lane; e0 < n; e0 += 32 * U) {
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + 32 * u;
      if (e < n) v[u] = e < a ? x1[e] : x2[e - a];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + 32 * u;
      if (e < n) {
        if (e < a) ((float4*)d1)[e] = v[u];
        else ((float4*)d2)[e - a] = v[u];
      }
    }
  }
  if (lane < r1) d1[a * V + lane] = t;
  else if (lane >= 8 && lane - 8 < r2) d2[b * V + lane - 8] = t;
}

// One mark (problem, logical child position, physical slot, family, patch)
// for k_refresh.
__device__ __forceinline__ void lin_mark(const Engine& E, int mpar, int p, int slot,
                                         unsigned phys, int fam, int ip) {
  const unsigned q = atomicAdd(&E.plan->mark_count[mpar], 1u);
  if (q < E.mark_cap) E.marks[(size_t)mpar * E.mark_cap + q] = make_mark(p, slot, phys, fam, ip);
}


// ---------------------------------------------------------------------------
// k2_lin_bound: one warp per (parent item, chunk of activity words)
// ---------------------------------------------------------------------------

// Windows one item may form: every chunk with more active constraints than a
// window takes is cut into word ranges while this many fit (so that an item
// with all of 4096 constraints active, at the root, gives 64 windows of 64
// rather than whole chunks of 256 that one warp would walk alone).  A cut
// chunk gives at most 4 windows (a word holds at most 32 of a window's 64),
// any other at most one, and items with summaries have at most 64 chunks, so
// 4 x 64 entries never overflow.
#define PCBA_LIN_MAXWIN 256
static_assert(PCBA_LIN_MAXWIN >= 4 * 64 && PCBA_LIN_WIN >= 64,
              "the window list of an item holds every window it can form");

// Per-warp buffers of the constraint bounds, after the staged patches.
struct LinScratch {
  unsigned char* sCh;     // the children's metadata (a LinChildren), 256 bytes
  unsigned* sMw;          // the children's words of a window, [2][64]
  int* sWi;               // the window's word indices, [64] (two per lane)
  unsigned* sWin;         // the windows of an item, [PCBA_LIN_MAXWIN]
  unsigned short* sIdx;   // compacted constraints, [PCBA_LIN_IDX]
  unsigned short* sCnt;   // active constraints per live chunk, [64]
  unsigned char* sChunk;  // the live chunks, [64]
};
__host__ __device__ constexpr size_t lin_scratch_bytes() {
  return 256 + 4 * 128 + 4 * 64 + 4 * PCBA_LIN_MAXWIN + 2 * PCBA_LIN_IDX + 2 * 64 + 64;
}
// base: 16-byte aligned
__device__ __forceinline__ LinScratch lin_scratch(unsigned char* base) {
  LinScratch s;
  s.sCh = base;
  s.sMw = (unsigned*)(base + 256);
  s.sWi = (int*)(s.sMw + 128);
  s.sWin = (unsigned*)(s.sWi + 64);
  s.sIdx = (unsigned short*)(s.sWin + PCBA_LIN_MAXWIN);
  s.sCnt = s.sIdx + PCBA_LIN_IDX;
  s.sChunk = (unsigned char*)(s.sCnt + 64);
  return s;
}

// Bytes of shared memory one warp of k2_lin_bound uses: both children's
// shared patches ([C][4] each), then the constraint buffers.
template <typename T>
__host__ __device__ constexpr size_t lin_bound_warp_bytes(int cgmax) {
  return (8 * (size_t)cgmax * sizeof(T) + 15) / 16 * 16 + lin_scratch_bytes();
}

// A window, as lane q's two word slots q and q + 32: each slot's word index
// wi (-1: none), value wv and summary bit cb (0 without summaries).  Two
// forms (chunk t0 in bits 0..15):
//   bit 31 clear: bit j of bits 16..30 says chunk t0 + j belongs to it (at
//     most PCBA_LIN_WCHUNKS chunks); slot s takes word s % 8 of its
//     (s / 8)-th chunk;
//   bit 31 set: words a .. b-1 of chunk t0 (a in bits 16..18, b in bits
//     19..22), for a chunk with more active constraints than one window
//     takes; slot q (of lane q) takes word a + q.
#define PCBA_LIN_WCHUNKS 8
__device__ __forceinline__ unsigned lin_word_window(int t0, int a, int b) {
  return (unsigned)t0 | ((unsigned)a << 16) | ((unsigned)b << 19) | 0x80000000u;
}
__device__ __forceinline__ void lin_window_words(const ProbDesc* D, const unsigned* pmask,
                                                 unsigned win, bool summ, int (&wi)[2],
                                                 unsigned (&wv)[2], unsigned long long (&cb)[2]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    wi[h] = -1;
    wv[h] = 0u;
    cb[h] = 0ull;
  }
  if (win & 0x80000000u) {
    const int t = (int)(win & 0xFFFFu), a = (int)((win >> 16) & 7u), b = (int)((win >> 19) & 15u);
    const int w = t * PCBA_LIN_WORDS + a + lane;
    if (lane < b - a && w < D->mwords) {
      wi[0] = w;
      wv[0] = pmask[w];
      cb[0] = summ ? 1ull << t : 0ull;
    }
    return;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int sl = lane + 32 * h;
    unsigned m = (win >> 16) & 0x7FFFu;
    for (int i = 0; i < (sl >> 3); ++i) m &= m - 1u;
    if (m != 0u) {
      const int t = (int)(win & 0xFFFFu) + __ffs(m) - 1;
      const int w = t * PCBA_LIN_WORDS + (sl & 7);
      if (w < D->mwords) {
        wi[h] = w;
        wv[h] = pmask[w];
        cb[h] = summ ? 1ull << t : 0ull;
      }
    }
  }
}

// Range of cc + sum_m w_m s_mj over the coefficients j = j0, j0 + G, ... of
// one child staged in shared memory ([C][4]); two partial extremes per bound.
template <typename T, int K>
__device__ __forceinline__ void lin_range(const T* s, int C, T cc, const T (&w)[K], int j0, int G,
                                          T& lo, T& hi) {
  T lo0 = T(INFINITY), hi0 = T(-INFINITY), lo1 = T(INFINITY), hi1 = T(-INFINITY);
  int j = j0;
#pragma unroll 2
  for (; j + G < C; j += 2 * G) {
    T a[K], b[K];
    lin_load<T, K>(s + (size_t)j * 4, a);
    lin_load<T, K>(s + (size_t)(j + G) * 4, b);
    T v0 = cc, v1 = cc;
#pragma unroll
    for (int m = 0; m < K; ++m) {
      v0 = fma(w[m], a[m], v0);
      v1 = fma(w[m], b[m], v1);
    }
    lo0 = min(lo0, v0);
    hi0 = max(hi0, v0);
    lo1 = min(lo1, v1);
    hi1 = max(hi1, v1);
  }
  if (j < C) {
    T a[K];
    lin_load<T, K>(s + (size_t)j * 4, a);
    T v0 = cc;
#pragma unroll
    for (int m = 0; m < K; ++m) v0 = fma(w[m], a[m], v0);
    lo0 = min(lo0, v0);
    hi0 = max(hi0, v0);
  }
  lo = min(lo0, lo1);
  hi = max(hi0, hi1);
}

// Both children's metadata (kept in shared memory, written by lane c K + g
// for child c and shared patch g): extremes of the stored values of each
// shared patch and, in FP32, their error bounds and offsets (the FP64 offset
// O split into FP32 values, O = Oh + Ol to 2^-48 |O|).  At most 256 bytes.
template <typename T, int K>
struct LinChildren {
  T mn[2][K], mx[2][K];
  float Mabs[2][K], ec[2][K];
  float Oh[2][K], Ol[2][K];
};
static_assert(sizeof(LinChildren<double, PCBA_MAX_SHARED>) <= 256, "metadata area of a warp");

// An FP64 value as two FP32 values, x = hi + lo to 2^-48 |x| (x - hi is
// exact in FP64).
__device__ __forceinline__ void lin_split_f64(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

// An upper bound of |x| 2^-52 (so of the rounding error of an FP64 sum
// whose result is x) from x's exponent field alone, without an FP64
// instruction: |x| < 2^(E - 1022) for the biased exponent E.  At most twice
// |x| 2^-52 when that is above 2^-126, +inf for a non-finite x.
__device__ __forceinline__ float lin_f64_ulp_bound(double x) {
  const int fe = max(((__double2hiint(x) >> 20) & 0x7ff) - 947, 1);
  return fe >= 255 ? INFINITY : __int_as_float(fe << 23);
}

// -x when neg, by the sign bit (no FP64 instruction).
__device__ __forceinline__ double lin_neg_if(double x, bool neg) {
  return __hiloint2double(__double2hiint(x) ^ (neg ? (int)0x80000000 : 0), __double2loint(x));
}

// The constant term kappa = c + sum_m w_m O_m of a constraint's coefficients
// relative to a child's offsets, in FP32 operations only (the two-float
// scheme of the comment at the top of this file): hv / lv are the row's FP32
// pairs (c, w_0 .. w_K-1).  kap is the result rounded to FP32, ekap a bound
// of its error before that rounding (2^-40 A64 + (8K + 2) 2^-149).
template <int K>
__device__ __forceinline__ void lin_kappa(const float* hv, const float* lv, const float (&Oh)[K],
                                          const float (&Ol)[K], float& kap, float& ekap) {
  float s = hv[0];        // c_hi + sum p_m, carried error-free with the TwoSum errors
  float sm = lv[0];       // the small terms
  float A = fabsf(hv[0]);  // A64 from the high parts, rounded up
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const float wh = hv[1 + m], wl = lv[1 + m];
    const float p = __fmul_rn(wh, Oh[m]);
    const float e = __fmaf_rn(wh, Oh[m], -p);  // wh Oh = p + e exactly
    const float t = __fadd_rn(s, p);           // TwoSum: s + p = t + er exactly
    const float bv = __fsub_rn(t, s);
    const float er = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    s = t;
    const float cross = __fadd_rn(__fmul_rn(wh, Ol[m]), __fmul_rn(wl, Oh[m]));
    sm = __fadd_rn(sm, __fadd_rn(__fadd_rn(e, er), cross));
    A = __fmaf_ru(fabsf(wh), fabsf(Oh[m]), A);
  }
  kap = __fadd_rn(s, sm);
  // the high parts understate A64 by at most a factor (1 + 2^-24)^2, well
  // inside the margin of 134 2^-48 < 2^-40
  ekap = __fadd_ru(__fmul_ru(A, 0x1p-40f), (float)(8 * K + 2) * 0x1p-149f);
}

// A window of up to 64 of parent item k's activity words (problem p, list
// length Kl): lane q holds two word slots (q and q + 32), each the index wi
// of one of the item's words (-1: none), its value word and its chunk's
// summary bit cbit (0 without summaries).  The window holds at most
// PCBA_LIN_IDX active constraints (a single chunk at most PCBA_LIN_WORDS x 32,
// several at most PCBA_LIN_WIN, a light item at most PCBA_LIN_LIGHT_MAX).
// They are compacted and bounded on both children (items left / right in
// slots slotL / slotR, shared patches staged at sL / sR, [C][4]); the
// children's words and their chunks' summary bits are written and the bound
// maxima go to the child records.  One warp; sIdx, sMw (the children's
// words, 2 x 64) and sWi (the 64 word indices) are its buffers.
static_assert(PCBA_LIN_WORDS * 32 <= PCBA_LIN_IDX && PCBA_LIN_WIN <= PCBA_LIN_IDX &&
                  PCBA_LIN_LIGHT_MAX <= PCBA_LIN_IDX,
              "a window's active constraints fit the compaction buffer");
template <typename T, int K>
__device__ void lin_window(const Engine& E, const ProbDesc* D, int p, int k, int Kl,
                           const int (&wi)[2], const unsigned (&word)[2],
                           const unsigned long long (&cbit)[2], char* left, char* right,
                           unsigned slotL, unsigned slotR,
                           const T* sL, const T* sR, const LinChildren<T, K>& ch,
                           unsigned short* sIdx, unsigned* sMw, int* sWi, int par) {
  constexpr bool RIG = sizeof(T) == 4;
  constexpr float u24 = 0x1p-24f;
  const int lane = threadIdx.x & 31;
  const long long slot_off = D->slot_off;
  const int C = D->cg;
  unsigned* pm = (unsigned*)(left + D->off_mask);  // the parent's words, in place
  unsigned* rm = (unsigned*)(right + D->off_mask);
  unsigned long long* sumL = (unsigned long long*)(left + D->off_sum) + (par ^ 1);
  unsigned long long* sumR = (unsigned long long*)(right + D->off_sum) + (par ^ 1);
  const unsigned w0 = wi[0] >= 0 ? word[0] : 0u, w1 = wi[1] >= 0 ? word[1] : 0u;
  const unsigned cnt = __popc(w0) + __popc(w1);
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned na = __shfl_sync(0xffffffffu, incl, 31);
  if (na == 0) {
    // no active constraint here: the children's words are zero (the left
    // child shares the parent's, already zero)
    if (wi[0] >= 0) rm[wi[0]] = 0u;
    if (wi[1] >= 0) rm[wi[1]] = 0u;
    return;
  }
  __syncwarp();  // earlier readers of the buffers are done
  sWi[lane] = wi[0];
  sWi[32 + lane] = wi[1];
#pragma unroll
  for (int i = 0; i < 4; ++i) sMw[32 * i + lane] = 0u;  // [child][slot]
  T gmax[2] = {T(-INFINITY), T(-INFINITY)}, gmin[2] = {T(-INFINITY), T(-INFINITY)};
  bool mark[2] = {false, false};
  unsigned nfull = 0;  // coefficient-range evaluations of this lane
  const int Kw = K;
  // lanes per constraint: G lanes share one constraint's coefficients when
  // the window has few (G a power of 2, na G <= 32, at most 8)
  const int G = na > 16 ? 1 : (na > 8 ? 2 : (na > 4 ? 4 : 8));
  const int gsub = lane & (G - 1);
  const unsigned per = 32u / (unsigned)G;
  // vertex incumbents: each child's corner values of its active constraints
  // (the corner coefficient is the constraint's value there, Sec. II-D)
  const bool vtx_on = E.params->vertex != 0;
  int jc[4] = {0, 0, 0, 0};
  T vmax[2][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (vtx_on) jc[q] = corner_index(D->G, D->l, q);
    vmax[0][q] = vmax[1][q] = T(-INFINITY);
  }
  {
    unsigned pos = incl - cnt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      unsigned bits = h ? w1 : w0;
      while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        sIdx[pos++] = (unsigned short)((lane + 32 * h) * 32 + b);
      }
    }
  }
  __syncwarp();
  for (unsigned q0 = 0; q0 < na; q0 += per) {
    // (the lanes past the last constraint repeat the first one and drop it)
    const unsigned q = q0 + (unsigned)lane / (unsigned)G;
    const bool act = q < na;
    const int li = sIdx[act ? q : 0u];
    const long long row = D->lin_off + (long long)sWi[li >> 5] * 32 + (li & 31);
    T w[K], cc[2];
    float E64[2] = {0.0f, 0.0f};  // FP32: bound of the error of the constant term
    if constexpr (RIG) {
      // the row's FP32 pairs (the slots past K + 1 are zero and not read)
      const float* r32 = E.lin32 + row * PCBA_LIN32_STRIDE;
      float hv[8], lv[8];
      {
        const float4 h0 = *(const float4*)r32, l0 = *(const float4*)(r32 + PCBA_LIN_STRIDE);
        hv[0] = h0.x; hv[1] = h0.y; hv[2] = h0.z; hv[3] = h0.w;
        lv[0] = l0.x; lv[1] = l0.y; lv[2] = l0.z; lv[3] = l0.w;
        if constexpr (K >= 4) {
          const float4 h1 = *(const float4*)(r32 + 4);
          const float4 l1 = *(const float4*)(r32 + PCBA_LIN_STRIDE + 4);
          hv[4] = h1.x; hv[5] = h1.y; hv[6] = h1.z; hv[7] = h1.w;
          lv[4] = l1.x; lv[5] = l1.y; lv[6] = l1.z; lv[7] = l1.w;
        }
      }
#pragma unroll
      for (int m = 0; m < K; ++m) w[m] = hv[1 + m];
      // the constant term c_i + sum_m w_im O_m of each child's coefficients
      // relative to its offsets: the large terms cancel here, and the FP32
      // part only carries the residuals (of the order of the box's range)
#pragma unroll
      for (int c = 0; c < 2; ++c) lin_kappa<K>(hv, lv, ch.Oh[c], ch.Ol[c], cc[c], E64[c]);
    } else {
      const double* rw = E.lin64 + row * PCBA_LIN_STRIDE;
#pragma unroll
      for (int m = 0; m < K; ++m) w[m] = (T)rw[1 + m];
      cc[0] = cc[1] = (T)rw[0];
    }
    // E of the comment at the top of this file (0 in FP64 mode), and the
    // interval bound from the ranges of the stored patches, per child
    float Ee[2] = {0.0f, 0.0f}, Er[2] = {0.0f, 0.0f};
    T lo[2], hi[2], Et[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float Eb = 0.0f;
      if constexpr (RIG) {
        float A = fabsf((float)cc[c]), ee = 0.0f;
#pragma unroll
        for (int m = 0; m < K; ++m) {
          A = __fmaf_ru(fabsf((float)w[m]), ch.Mabs[c][m], A);
          ee = __fmaf_ru(fabsf((float)w[m]), ch.ec[c][m], ee);
        }
        const float kk = (float)(2 * Kw + 2);
        Er[c] = __fmul_ru((kk + 1.0f) * u24, A);
        Ee[c] = ee;
        Eb = __fadd_ru(__fadd_ru(__fadd_ru(Er[c], __fmul_ru(ee, 1.0f + 0x1p-20f)), E64[c]),
                       kk * 0x1p-149f);
      }
      Et[c] = T(Eb);
      T x0 = cc[c], x1 = cc[c];
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const T x = w[m] * ch.mn[c][m], y = w[m] * ch.mx[c][m];
        x0 += min(x, y);
        x1 += max(x, y);
      }
      lo[c] = x0;
      hi[c] = x1;
    }
    // undecided by the interval: the coefficient range itself (Alg. 3), the
    // G lanes of the constraint taking every G-th coefficient
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const bool need = !(add_up(hi[c], Et[c]) <= T(0)) && !(sub_dn(lo[c], Et[c]) > T(0));
      T rl = T(INFINITY), rh = T(-INFINITY);
      if (need) lin_range<T, K>(c ? sR : sL, C, cc[c], w, gsub, G, rl, rh);
      for (int o = 1; o < G; o <<= 1) {
        rl = min(rl, __shfl_xor_sync(0xffffffffu, rl, o));
        rh = max(rh, __shfl_xor_sync(0xffffffffu, rh, o));
      }
      if (need) {
        lo[c] = rl;
        hi[c] = rh;
        if (act && gsub == 0) ++nfull;
      }
    }
    if (vtx_on && act && gsub == 0) {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T a[K];
          lin_load<T, K>((c ? sR : sL) + (size_t)jc[q] * 4, a);
          T v = cc[c];
#pragma unroll
          for (int m = 0; m < K; ++m) v = fma(w[m], a[m], v);
          vmax[c][q] = max(vmax[c][q], add_up(v, Et[c]));
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!act || gsub != 0) continue;
      const T up = add_up(hi[c], Et[c]), dn = sub_dn(lo[c], Et[c]);
      const bool sat = up <= T(0);
      const bool inf = dn > T(0);
      if (!sat) {
        atomicOr(&sMw[c * 64 + (li >> 5)], 1u << (li & 31));
        gmax[c] = max(gmax[c], up);
        gmin[c] = max(gmin[c], dn);
      }
      if constexpr (RIG) {
        // the bound changed a decision the stored coefficients make: mark
        // the child's shared patches for a refresh if their errors are
        // the larger part of the bound
        const bool flip = (hi[c] <= T(0)) != sat || (lo[c] > T(0)) != inf;
        if (flip && Ee[c] > Er[c]) mark[c] = true;
      }
    }
  }
  unsigned long long kl = 0ull, kr = 0ull;
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (wi[h] >= 0) {
      const unsigned vl = sMw[lane + 32 * h], vr = sMw[64 + lane + 32 * h];
      pm[wi[h]] = vl;  // left child: in place (this window's words)
      rm[wi[h]] = vr;  // right child
      // the summary bits of the chunks that keep an active constraint
      if (vl != 0u) kl |= cbit[h];
      if (vr != 0u) kr |= cbit[h];
    }
  const unsigned long long keepL =
      ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(kl >> 32)) << 32) |
      __reduce_or_sync(0xffffffffu, (unsigned)kl);
  const unsigned long long keepR =
      ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(kr >> 32)) << 32) |
      __reduce_or_sync(0xffffffffu, (unsigned)kr);
  if (lane == 0) {
    if (keepL) atomicOr(sumL, keepL);
    if (keepR) atomicOr(sumR, keepR);
    atomicAdd(&E.plan->lin_pairs, 2ull * na);
  }
  if (vtx_on) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T m = lin_wmax(vmax[c][q]);
        if (lane == 0 && m > T(-INFINITY)) {
          const float mf = sizeof(T) == 4 ? (float)m : __double2float_ru((double)m);
          atomicMax(&E.rec[slot_off + k + (c ? Kl : 0)].vtxg[q], okey32(mf));
        }
      }
  }
  const unsigned full = __reduce_add_sync(0xffffffffu, nfull);
  if (lane == 0) atomicAdd(&E.plan->lin_full, (unsigned long long)full);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T gx = lin_wmax(gmax[c]);
    const T gn = lin_wmax(gmin[c]);
    ChildRec* rc = E.rec + slot_off + k + (c ? Kl : 0);
    if (lane == 0 && gx > T(-INFINITY)) {
      if constexpr (RIG) {
        atomicMax(&rc->gmaxmax, okey_f32((float)gx));
        atomicMax(&rc->gminmax, okey_f32((float)gn));
      } else {
        atomicMax(&rc->gmaxmax, okey((double)gx));
        atomicMax(&rc->gminmax, okey((double)gn));
      }
    }
  }
  if constexpr (RIG) {
    const MarkCtx mk{p, k, k + Kl, slotL, slotR, E.marks + (size_t)par * E.mark_cap,
                     &E.plan->mark_count[par], E.mark_cap};
    // one mark per child for all its shared patches (family PCBA_FAM_LIN),
    // the first window to ask for it sets bit 32 of the child record's perr
    // (the split kernel wrote the error bits below it this step)
    bool ml = __any_sync(0xffffffffu, mark[0]), mr = __any_sync(0xffffffffu, mark[1]);
    if (lane == 0) {
      constexpr unsigned long long bit = 1ull << 32;
      if (ml) ml = !(atomicOr(&E.rec[slot_off + k].perr, bit) & bit);
      if (mr) mr = !(atomicOr(&E.rec[slot_off + k + Kl].perr, bit) & bit);
    }
    append_marks(mk, lane == 0 && ml, lane == 0 && mr, PCBA_FAM_LIN, 0);
  }
  __syncwarp();
}

// Bytes of shared memory one warp of k2_lin_split uses: the parent's shared
// patches and their two children (coefficient-major, 4 slots per
// coefficient), the parent's cost patch and its two children, then the
// compacted constraint indices and the children's activity words of one chunk.
template <typename T>
__host__ __device__ constexpr size_t lin_split_warp_bytes(int cgmax, int cpmax) {
  return ((3 * (size_t)cpmax + 12 * (size_t)cgmax) * sizeof(T) + 15) / 16 * 16 +
         lin_scratch_bytes();
}

// Extremes of the two children of one patch group (the cost, or one shared
// patch) and the largest |parent value|, accumulated per lane.
template <typename T>
struct LinAcc {
  T mnL, mxL, mnR, mxR, am;
  __device__ __forceinline__ void init() {
    mnL = mnR = T(INFINITY);
    mxL = mxR = T(-INFINITY);
    am = T(0);
  }
  __device__ __forceinline__ void merge(const LinAcc& o) {
    mnL = min(mnL, o.mnL);
    mxL = max(mxL, o.mxL);
    mnR = min(mnR, o.mnR);
    mxR = max(mxR, o.mxR);
    am = max(am, o.am);
  }
};

// One fibre (N + 1 values at src[j * sst], children to dL / dR at the same
// positions): the de Casteljau triangle at 1/2 (Sec. II-E) in registers.
template <typename T, int N>
__device__ __forceinline__ void lin_fibre(const T* src, T* dL, T* dR, int sst, LinAcc<T>& a) {
  T q[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    q[j] = src[j * sst];
    a.am = max(a.am, abs(q[j]));
  }
  dL[0] = q[0];
  dR[N * sst] = q[N];
  a.mnL = min(a.mnL, q[0]);
  a.mxL = max(a.mxL, q[0]);
  a.mnR = min(a.mnR, q[N]);
  a.mxR = max(a.mxR, q[N]);
#pragma unroll
  for (int k = 1; k <= N; ++k) {
#pragma unroll
    for (int j = 0; j <= N - k; ++j) q[j] = mulrn(addrn(q[j], q[j + 1]), T(0.5));
    dL[k * sst] = q[0];
    dR[(N - k) * sst] = q[N - k];
    a.mnL = min(a.mnL, q[0]);
    a.mxL = max(a.mxL, q[0]);
    a.mnR = min(a.mnR, q[N - k]);
    a.mxR = max(a.mxR, q[N - k]);
  }
}

// NFIX > 0: every patch of the batch has degree NFIX along every axis (a
// smaller kernel body); 0: any degree up to 16.
// Resident blocks per SM the register allocation of the two kernels aims at
// (128 registers: with two word slots per lane, a third block's 80 registers
// made the split kernel spill more than its extra warps gained).
#ifndef PCBA_LIN_SPLIT_BLOCKS
#define PCBA_LIN_SPLIT_BLOCKS 2
#endif
#ifndef PCBA_LIN_BOUND_BLOCKS
#define PCBA_LIN_BOUND_BLOCKS 2
#endif

template <typename T, int K, int NFIX>
__global__ void __launch_bounds__(256, PCBA_LIN_SPLIT_BLOCKS) k2_lin_split(Engine E, int cgmax, int cpmax) {
  pdl_begin();
  if (blockIdx.x == 0 && threadIdx.x == 0) E.plan->kr_par = E.plan->steps_global & 1;
  constexpr bool RIG = sizeof(T) == 4;
  constexpr float u24 = 0x1p-24f;
  extern __shared__ __align__(16) unsigned char kls[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the shared patches first: their 16-byte vector loads need the warp's
  // (16-byte aligned) base, whatever the cost patch's size
  T* sp = (T*)(kls + (size_t)warp * lin_split_warp_bytes<T>(cgmax, cpmax));  // [C][4]
  T* spL = sp + 4 * (size_t)cgmax;
  T* spR = spL + 4 * (size_t)cgmax;
  T* sc = spR + 4 * (size_t)cgmax;  // parent cost patch and its children
  T* scL = sc + cpmax;
  T* scR = scL + cpmax;
  const LinScratch ls = lin_scratch(
      (unsigned char*)sp + ((3 * (size_t)cpmax + 12 * (size_t)cgmax) * sizeof(T) + 15) / 16 * 16);
  // the children's metadata, warp-uniform: read by broadcast from shared memory
  LinChildren<T, K>& ch = *reinterpret_cast<LinChildren<T, K>*>(ls.sCh);
  const unsigned items = E.plan->kr_units;
  const int par = E.plan->steps_global & 1;  // copy read this step; children go to par ^ 1
  // an FP32 e exceeds opt_tol / 64 exactly when it exceeds this
  const float cost_thr32 = __double2float_rd(E.params->opt_tol * (1.0 / 64.0));
  const bool vtx = E.params->vertex != 0;
  int cx_p = -1, cx_K = 0, cx_r = 0, cx_ftop = 0, cx_hw = 0;
  unsigned cx_beg = 0, cx_end = 0;
  const ProbDesc* D = nullptr;
  // items are fetched from a counter (reset before every step), one at a
  // time unless there are many per resident warp: a step ends when its last
  // warp does, so batches that leave some warps one batch more than others
  // cost a whole batch of latency
  const unsigned bsz =
      items < 16u * gridDim.x * (blockDim.x >> 5) ? 1u : (unsigned)PCBA_LIN_BATCH;
  for (;;) {
    unsigned ubeg = 0;
    if (lane == 0) ubeg = atomicAdd(&E.plan->lin_next2, bsz);
    ubeg = __shfl_sync(0xffffffffu, ubeg, 0);
    if (ubeg >= items) break;
    const unsigned uend = min(items, ubeg + bsz);
    for (unsigned u = ubeg; u < uend; ++u) {
      if (u < cx_beg || u >= cx_end || cx_p < 0) {
        cx_p = find_problem_warp(E.kr_pre, E.np, u, lane);
        cx_beg = E.kr_pre[cx_p];
        cx_end = E.kr_pre[cx_p + 1];
        D = E.desc + cx_p;
        const ProbState* S = E.state + cx_p;
        cx_K = S->K;
        cx_r = S->r;
        cx_ftop = S->ftop;
        cx_hw = S->hw;
      }
      const int p = cx_p, Kl = cx_K, r = cx_r, k = (int)(u - cx_beg);
      const long long slot_off = D->slot_off;
      const unsigned pslot = E.map[slot_off + k];
      const unsigned rslot = right_slot(E, slot_off, k, cx_ftop, cx_hw);
      char* list = E.arena + D->list_off;
      char* parent = list + (size_t)pslot * D->item_bytes;
      char* right = list + (size_t)rslot * D->item_bytes;
      ChildRec* recL = E.rec + slot_off + k;
      ChildRec* recR = E.rec + slot_off + k + Kl;
      const int l = D->l, cp = D->cp, C = D->cg;
      // the parent's box index along axis lane - 16 (read early: the
      // children's are written with the cost records)
      const unsigned ivw = lane >= 16 && lane < 16 + l ? ((const unsigned*)parent)[lane - 16] : 0u;
      // ---- stage the parent (coalesced).  Every read of the parent is issued
      // before the first use of one: its summary, header, the shared patches'
      // metadata and the patches themselves (read whatever the summary says,
      // unused when it is empty)
      const unsigned long long psum0 =
          D->lin_chunks <= 64 ? *((const unsigned long long*)(parent + D->off_sum) + par) : ~0ull;
      T* pc = (T*)(parent + D->off_cost);
      T* rc = (T*)(right + D->off_cost);
      const T* gs = (const T*)(parent + D->off_g + par * D->copy_g);
      char* pm = parent + D->off_eg + par * D->copy_e;
      double Oc = 0.0, Om[K];
      float ecost = 0.0f, em[K];
#pragma unroll
      for (int m = 0; m < K; ++m) {
        Om[m] = 0.0;
        em[m] = 0.0f;
      }
      if constexpr (RIG) {
        Oc = *(const double*)(parent + 32);
        ecost = *(const float*)(parent + 40);
#pragma unroll
        for (int m = 0; m < K; ++m) {
          em[m] = fabsf(LinMeta<T>::err(pm, 4)[m]);
          Om[m] = LinMeta<T>::off(pm, 4)[m];
        }
      }
      lin_copy2<T, 4>(sc, pc, cp, sp, gs, 4 * C, lane);
      // shared patches only while a constraint is active in the item
      const bool any = psum0 != 0ull;
      __syncwarp();
      // ---- every fibre of the cost patch and of the shared patches, a lane each
      const int nc = D->P[r], stc = axis_stride(D->P, l, r), nfc = cp / (nc + 1);
      const int blkc = (nc + 1) * stc;
      const int ns = D->G[r], sts = axis_stride(D->G, l, r), nfs = C / (ns + 1);
      const int blks = (ns + 1) * sts;
      const int ntask = nfc + (any ? K * nfs : 0);
      LinAcc<T> acc[K + 1];
#pragma unroll
      for (int g = 0; g <= K; ++g) acc[g].init();
      // (one code path for every task: the fibre's extremes are merged into
      // its group's accumulator afterwards)
      for (int task = lane; task < ntask; task += 32) {
        int grp = 0, base, sst, n = nc;
        const T* src = sc;
        T *dL = scL, *dR = scR;
        if (task < nfc) {
          const int o = task / stc;
          base = o * blkc + (task - o * stc);
          sst = stc;
        } else {
          const int t2 = task - nfc;
          const int m = t2 / nfs;
          const int f = t2 - m * nfs;
          const int o = f / sts;
          base = (o * blks + (f - o * sts)) * 4 + m;
          sst = 4 * sts;
          grp = 1 + m;
          n = ns;
          src = sp;
          dL = spL;
          dR = spR;
        }
        LinAcc<T> t;
        t.init();
        dispatch_fixed<16, NFIX>(n, [&](auto c) {
          lin_fibre<T, decltype(c)::value>(src + base, dL + base, dR + base, sst, t);
        });
#pragma unroll
        for (int g = 0; g <= K; ++g)
          if (g == grp) acc[g].merge(t);
      }
      // ---- extremes per patch group, over the warp
#pragma unroll
      for (int g = 0; g <= K; ++g) {
        acc[g].mnL = lin_wmin(acc[g].mnL);
        acc[g].mxL = lin_wmax(acc[g].mxL);
        acc[g].mnR = lin_wmin(acc[g].mnR);
        acc[g].mxR = lin_wmax(acc[g].mxR);
        acc[g].am = lin_wmax(acc[g].am);
      }
      __syncwarp();
      // ---- cost children: re-centred on the middle of each child's range
      // (FP32), error bound grown by n (max |parent| 2^-24 + 2^-149) for the
      // triangle and by max |stored| 2^-24 + 2^-149 + 2^-52 |O'| (rounded up
      // to a power of two) for the re-centring; the bounds go to the child
      // records
      T shc[2] = {T(0), T(0)};
      if constexpr (RIG) {
        shc[0] = __fmul_rn(__fadd_rn(acc[0].mnL, acc[0].mxL), 0.5f);
        shc[1] = __fmul_rn(__fadd_rn(acc[0].mnR, acc[0].mxR), 0.5f);
      }
      for (int j = lane; j < cp; j += 32) {
        pc[j] = addrn(scL[j], -shc[0]);
        rc[j] = addrn(scR[j], -shc[1]);
      }
      // the cost records, lane 2 v + c for child c and value v: 0 the lower
      // bound, 1 the upper bound, 2 + q the cost at corner q (vertex
      // incumbents).  Every lane forms the child's offset and error bound,
      // then one upward FP64 sum with them (the lower bound is the negated
      // sum of the negated terms), so the warp issues each FP64 instruction
      // of the records once.  Lane 16 + s: the children's box index along
      // axis s, and (s = 0) the right child's slot.
      if (lane < 12) {
        const int c = lane & 1, v = lane >> 1;
        const T cmn = c ? acc[0].mnR : acc[0].mnL, cmx = c ? acc[0].mxR : acc[0].mxL;
        const T* st = c ? scR : scL;
        ChildRec* rec = c ? recR : recL;
        if constexpr (RIG) {
          if (v < (vtx ? 6 : 2)) {
            const float e1 = __fadd_ru(__fadd_ru(ecost, __fmul_ru(acc[0].am, (float)nc * u24)),
                                       (float)nc * 0x1p-149f);
            const float sh = c ? shc[1] : shc[0];
            const float smin = __fsub_rn(cmn, sh);
            const float smax = __fsub_rn(cmx, sh);
            const float Mr = fmaxf(fabsf(smin), fabsf(smax));
            const double On = Oc + (double)sh;
            const float e2 = __fadd_ru(__fadd_ru(__fadd_ru(e1, __fmul_ru(Mr, u24)), 0x1p-149f),
                                       lin_f64_ulp_bound(On));
            // the stored value at corner v - 2 is exactly the re-centred
            // child coefficient written above
            const float b = v == 0 ? __fsub_ru(e2, smin)
                            : v == 1 ? __fadd_ru(smax, e2)
                                     : __fadd_ru(__fsub_rn(st[corner_index(D->P, l, v - 2)], sh), e2);
            const double y = __dadd_ru(lin_neg_if(On, v == 0), (double)b);
            if (v == 0) {
              rec->pmin = okey(lin_neg_if(y, true));
            } else if (v == 1) {
              char* it = c ? right : parent;
              *(double*)(it + 32) = On;
              *(float*)(it + 40) = e2;
              rec->pmax = okey(y);
              rec->perr = __float_as_uint(e2);
              if (e2 > cost_thr32) lin_mark(E, par, p, c ? k + Kl : k, c ? rslot : pslot, 2, 0);
            } else {
              rec->vtxc[v - 2] = __double2float_ru(y);
            }
          }
        } else if (v == 0) {
          rec->pmin = okey((double)cmn);
          rec->pmax = okey((double)cmx);
          if (vtx) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              rec->vtxc[q] = __double2float_ru((double)st[corner_index(D->P, l, q)]);
          }
        }
      } else if (lane >= 16 && lane < 16 + l) {
        const int s = lane - 16;
        ((unsigned*)right)[s] = s == r ? 2u * ivw + 1u : ivw;
        if (s == r) ((unsigned*)parent)[s] = 2u * ivw;
        if (s == 0) E.map[slot_off + k + Kl] = rslot;
      }
      // ---- shared children, re-centred likewise, to the other copy, with
      // their metadata (error bound, offset, extremes of the stored values)
      if (any) {
        T sh[2][K];
#pragma unroll
        for (int g = 0; g < K; ++g) {
          sh[0][g] = RIG ? T(__fmul_rn(__fadd_rn((float)acc[1 + g].mnL, (float)acc[1 + g].mxL), 0.5f))
                         : T(0);
          sh[1][g] = RIG ? T(__fmul_rn(__fadd_rn((float)acc[1 + g].mnR, (float)acc[1 + g].mxR), 0.5f))
                         : T(0);
        }
        T* gL = (T*)(parent + D->off_g + (par ^ 1) * D->copy_g);
        T* gR = (T*)(right + D->off_g + (par ^ 1) * D->copy_g);
        for (int e = lane; e < 4 * C; e += 32) {
          const int m = e & 3;
          T a0 = T(0), a1 = T(0);
#pragma unroll
          for (int g = 0; g < K; ++g)
            if (g == m) {
              a0 = sh[0][g];
              a1 = sh[1][g];
            }
          if (m < K) {
            // the stored values, kept staged for the constraint bounds below
            const T vl = addrn(spL[e], -a0), vr = addrn(spR[e], -a1);
            gL[e] = vl;
            gR[e] = vr;
            spL[e] = vl;
            spR[e] = vr;
          }
        }
        // the children's metadata, lane c K + g for child c and shared patch
        // g (the FP64 offset arithmetic once per value), then broadcast: it
        // is also what the bound of the constraints below uses
        {
          T mn0 = T(0), mx0 = T(0), shv = T(0);
          float amv = 0.0f, emv = 0.0f;
          double omv = 0.0;
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int g = 0; g < K; ++g)
              if (lane == c * K + g) {
                mn0 = c ? acc[1 + g].mnR : acc[1 + g].mnL;
                mx0 = c ? acc[1 + g].mxR : acc[1 + g].mxL;
                shv = sh[c][g];
                amv = (float)acc[1 + g].am;
                emv = em[g];
                omv = Om[g];
              }
          T vmn = mn0, vmx = mx0;
          float vM = 0.0f, vec = 0.0f, vOh = 0.0f, vOl = 0.0f;
          double vO = 0.0;
          if constexpr (RIG) {
            if (lane < 2 * K) {
              const float e1 = __fadd_ru(__fadd_ru(emv, __fmul_ru(amv, (float)ns * u24)),
                                         (float)ns * 0x1p-149f);
              const float smin = __fsub_rn((float)mn0, (float)shv);
              const float smax = __fsub_rn((float)mx0, (float)shv);
              vM = fmaxf(fabsf(smin), fabsf(smax));
              vO = omv + (double)shv;
              lin_split_f64(vO, vOh, vOl);
              vec = __fadd_ru(__fadd_ru(__fadd_ru(e1, __fmul_ru(vM, u24)), 0x1p-149f),
                              lin_f64_ulp_bound(vO));
              vmn = T(smin);
              vmx = T(smax);
            }
          }
          if (lane < 2 * K) {
            const int c = lane / K, g = lane - c * K;
            char* cm = (c ? right : parent) + D->off_eg + (par ^ 1) * D->copy_e;
            if constexpr (RIG) {
              LinMeta<T>::err(cm, 4)[g] = vec;
              LinMeta<T>::off(cm, 4)[g] = vO;
            }
            LinMeta<T>::mn(cm, 4)[g] = vmn;
            LinMeta<T>::mx(cm, 4)[g] = vmx;
            ch.mn[c][g] = vmn;
            ch.mx[c][g] = vmx;
            ch.Mabs[c][g] = vM;
            ch.ec[c][g] = vec;
            ch.Oh[c][g] = vOh;
            ch.Ol[c][g] = vOl;
          }
        }
        __syncwarp();
      }
      // ---- the constraints.  The children's summaries start empty (each
      // window sets the bits of its chunks that keep an active constraint)
      // and their words of chunks without one are zero.  An item whose live
      // chunks (at most PCBA_LIN_WCHUNKS) hold at most PCBA_LIN_LIGHT_MAX
      // active constraints is bounded here, from the children still staged.
      // The live chunks of the other items are grouped into windows (at most
      // PCBA_LIN_WCHUNKS chunks within 16 consecutive ones, at most PCBA_LIN_WIN active
      // constraints unless a single chunk); a single window stays here,
      // several are queued for k2_lin_bound (those the full queue refuses
      // stay here too).
      {
        const int chunks = D->lin_chunks, mwords = D->mwords;
        const bool summ = chunks <= 64;  // (more chunks keep no summaries: all are read)
        const unsigned long long psum = summ ? psum0 : 0ull;
        if (lane == 0 && summ) {
          *((unsigned long long*)(parent + D->off_sum) + (par ^ 1)) = 0ull;
          *((unsigned long long*)(right + D->off_sum) + (par ^ 1)) = 0ull;
        }
        const unsigned* pmask = (const unsigned*)(parent + D->off_mask);
        unsigned* rmask = (unsigned*)(right + D->off_mask);
        if (summ)
          for (int q = lane; q < mwords; q += 32)
            if (!((psum >> (q / PCBA_LIN_WORDS)) & 1ull)) rmask[q] = 0u;
        __syncwarp();
        const int nlive = summ ? __popcll(psum) : chunks;
        // what this warp bounds itself: mode 1 the light window (lane words
        // lwi / lwv / lcb), 2 the windows in ls.sWin not queued (a single
        // one, or those the full queue refused), 3 the single-chunk windows
        // the queue refused
        int mode = 0, nwin = 0, nq = 0;
        unsigned qb = 0u;
        int lwi[2] = {-1, -1};
        unsigned lwv[2] = {0u, 0u};
        unsigned long long lcb[2] = {0ull, 0ull};
        if (nlive > 0 && summ && nlive <= PCBA_LIN_WCHUNKS) {
          // word slot s (q and q + 32 of lane q): word s % 8 of the (s / 8)-th
          // live chunk
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = (lane + 32 * h) >> 3;
            if (j < nlive) {
              unsigned long long m = psum;
              for (int i2 = 0; i2 < j; ++i2) m &= m - 1ull;
              const int t = __ffsll((long long)m) - 1;
              const int w = t * PCBA_LIN_WORDS + (lane & 7);
              if (w < mwords) {
                lwi[h] = w;
                lwv[h] = pmask[w];
                lcb[h] = 1ull << t;
              }
            }
          }
          if (__reduce_add_sync(0xffffffffu, (unsigned)(__popc(lwv[0]) + __popc(lwv[1]))) <=
              PCBA_LIN_LIGHT_MAX)
            mode = 1;
        }
        if (nlive > 0 && summ && mode == 0) {
          // the live chunks in order and their active constraints
          for (int t = lane; t < 64; t += 32)
            if ((psum >> t) & 1ull)
              ls.sChunk[__popcll(psum & ((1ull << t) - 1ull))] = (unsigned char)t;
          __syncwarp();
          for (int j0 = 0; j0 < nlive; j0 += 4) {
            const int j = j0 + (lane >> 3);
            unsigned c = 0u;
            if (j < nlive) {
              const int w = ls.sChunk[j] * PCBA_LIN_WORDS + (lane & 7);
              if (w < mwords) c = __popc(pmask[w]);
            }
            c += __shfl_xor_sync(0xffffffffu, c, 1);
            c += __shfl_xor_sync(0xffffffffu, c, 2);
            c += __shfl_xor_sync(0xffffffffu, c, 4);
            if ((lane & 7) == 0 && j < nlive) ls.sCnt[j] = (unsigned short)c;
          }
          __syncwarp();
          // the windows, formed greedily by lane 0; a chunk with more than
          // PCBA_LIN_WIN active constraints is cut into ranges of its words
          // (while the window list has room)
          if (lane == 0) {
            int j = 0;
            while (j < nlive) {
              const int t0 = ls.sChunk[j];
              if (ls.sCnt[j] > PCBA_LIN_WIN && nwin + PCBA_LIN_WORDS <= PCBA_LIN_MAXWIN) {
                int a = 0;
                unsigned cw = 0u;
                for (int b = 0; b < PCBA_LIN_WORDS; ++b) {
                  const int w = t0 * PCBA_LIN_WORDS + b;
                  const unsigned c = w < mwords ? (unsigned)__popc(pmask[w]) : 0u;
                  if (b > a && cw + c > (unsigned)PCBA_LIN_WIN) {
                    ls.sWin[nwin++] = lin_word_window(t0, a, b);
                    a = b;
                    cw = 0u;
                  }
                  cw += c;
                }
                ls.sWin[nwin++] = lin_word_window(t0, a, PCBA_LIN_WORDS);
                ++j;
                continue;
              }
              unsigned mask = 1u, cw = ls.sCnt[j];
              int nch = 1;
              ++j;
              while (j < nlive && nch < PCBA_LIN_WCHUNKS && ls.sChunk[j] - t0 < 15 &&
                     cw + ls.sCnt[j] <= (unsigned)PCBA_LIN_WIN) {
                mask |= 1u << (ls.sChunk[j] - t0);
                cw += ls.sCnt[j];
                ++nch;
                ++j;
              }
              ls.sWin[nwin++] = (unsigned)t0 | (mask << 16);
            }
          }
          nwin = __shfl_sync(0xffffffffu, nwin, 0);
          __syncwarp();
          // several windows: all go to the bound kernel's warps (a heavy
          // item's windows would otherwise run one after another here)
          nq = nwin > 1 ? nwin : 0;
          if (lane == 0 && nq > 0) qb = atomicAdd(&E.plan->lin_qcount, (unsigned)nq);
          qb = __shfl_sync(0xffffffffu, qb, 0);
          for (int i2 = lane; i2 < nq; i2 += 32) {
            const unsigned q = qb + (unsigned)i2;
            if (q < E.lin_qcap) E.lin_queue[q] = make_uint4(u, ls.sWin[i2], (unsigned)p, (unsigned)k);
          }
          mode = 2;
        }
        if (nlive > 0 && !summ) {
          // no summaries: every chunk is a window of its own, queued
          if (lane == 0) qb = atomicAdd(&E.plan->lin_qcount, (unsigned)chunks);
          qb = __shfl_sync(0xffffffffu, qb, 0);
          for (int t = lane; t < chunks; t += 32)
            if (qb + (unsigned)t < E.lin_qcap)
              E.lin_queue[qb + (unsigned)t] =
                  make_uint4(u, (unsigned)t | (1u << 16), (unsigned)p, (unsigned)k);
          mode = 3;
        }
        for (int i2 = 0; mode != 0; ++i2) {
          int wi[2] = {lwi[0], lwi[1]};
          unsigned wv[2] = {lwv[0], lwv[1]};
          unsigned long long cb[2] = {lcb[0], lcb[1]};
          if (mode == 1) {
            if (i2 > 0) break;
          } else if (mode == 2) {
            while (i2 < nq && qb + (unsigned)i2 < E.lin_qcap) ++i2;  // queued
            if (i2 >= nwin) break;
            lin_window_words(D, pmask, ls.sWin[i2], true, wi, wv, cb);
          } else {
            while (i2 < chunks && qb + (unsigned)i2 < E.lin_qcap) ++i2;
            if (i2 >= chunks) break;
            lin_window_words(D, pmask, (unsigned)i2 | (1u << 16), false, wi, wv, cb);
          }
          lin_window<T, K>(E, D, p, k, Kl, wi, wv, cb, parent, right, pslot, rslot, spL, spR, ch, ls.sIdx,
                           ls.sMw, ls.sWi, par);
        }
      }
      __syncwarp();  // the staging buffers are reused by the next item
    }
  }
}

// Heavy items' live chunks, queued by k2_lin_split as (item, window): the
// children are staged from memory.
template <typename T, int K>
__global__ void __launch_bounds__(256, PCBA_LIN_BOUND_BLOCKS) k2_lin_bound(Engine E, int cgmax) {
  pdl_begin();
  constexpr bool RIG = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char klb[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* sS = (T*)(klb + (size_t)warp * lin_bound_warp_bytes<T>(cgmax));  // children [2][C][4]
  const LinScratch ls =
      lin_scratch((unsigned char*)sS + (8 * (size_t)cgmax * sizeof(T) + 15) / 16 * 16);
  LinChildren<T, K>& ch = *reinterpret_cast<LinChildren<T, K>*>(ls.sCh);
  const unsigned units = min(E.plan->lin_qcount, E.lin_qcap);
  const int par = E.plan->steps_global & 1;  // the children's data is in copy par ^ 1
  const unsigned bsz =
      units < 16u * gridDim.x * (blockDim.x >> 5) ? 1u : (unsigned)PCBA_LIN_BATCH;
  unsigned cur = 0xFFFFFFFFu;  // the item whose children are staged
  int p = 0, k = 0, Kl = 0;
  const ProbDesc* D = nullptr;
  char *left = nullptr, *right = nullptr;
  unsigned sLs = 0u, sRs = 0u;  // their physical slots
  for (;;) {
    unsigned ubeg = 0;
    if (lane == 0) ubeg = atomicAdd(&E.plan->lin_next, bsz);
    ubeg = __shfl_sync(0xffffffffu, ubeg, 0);
    if (ubeg >= units) break;
    const unsigned uend = min(units, ubeg + bsz);
    for (unsigned q = ubeg; q < uend; ++q) {
      const uint4 ent = E.lin_queue[q];  // (item, window, problem, index in the list)
      // an item's windows are queued one after another: the next window of
      // the same item reuses the staged children
      if (ent.x != cur) {
        cur = ent.x;
        p = (int)ent.z;
        D = E.desc + p;
        k = (int)ent.w;
        Kl = E.state[p].K;
        char* list = E.arena + D->list_off;
        sLs = E.map[D->slot_off + k];
        sRs = E.map[D->slot_off + k + Kl];
        left = list + (size_t)sLs * D->item_bytes;
        right = list + (size_t)sRs * D->item_bytes;
        const int C = D->cg;
        __syncwarp();  // the previous unit's readers of the staging buffers are done
        // the children's shared patches, and their metadata (lane c K + g)
        lin_copy2<T, 2>(sS, (const T*)(left + D->off_g + (par ^ 1) * D->copy_g), 4 * C,
                        sS + 4 * (size_t)cgmax,
                        (const T*)(right + D->off_g + (par ^ 1) * D->copy_g), 4 * C, lane);
        if (lane < 2 * K) {
          const int c = lane / K, g = lane - c * K;
          char* mc = (c ? right : left) + D->off_eg + (par ^ 1) * D->copy_e;
          const T vmn = LinMeta<T>::mn(mc, 4)[g];
          const T vmx = LinMeta<T>::mx(mc, 4)[g];
          float vM = 0.0f, vec = 0.0f, vOh = 0.0f, vOl = 0.0f;
          if constexpr (RIG) {
            vM = fmaxf(fabsf((float)vmn), fabsf((float)vmx));
            vec = LinMeta<T>::err(mc, 4)[g];
            lin_split_f64(LinMeta<T>::off(mc, 4)[g], vOh, vOl);
          }
          ch.mn[c][g] = vmn;
          ch.mx[c][g] = vmx;
          ch.Mabs[c][g] = vM;
          ch.ec[c][g] = vec;
          ch.Oh[c][g] = vOh;
          ch.Ol[c][g] = vOl;
        }
      }
      int wi[2];
      unsigned wv[2];
      unsigned long long cb[2];
      lin_window_words(D, (const unsigned*)(left + D->off_mask), ent.y, D->lin_chunks <= 64, wi,
                       wv, cb);
      __syncwarp();
      lin_window<T, K>(E, D, p, k, Kl, wi, wv, cb, left, right, sLs, sRs, sS, sS + 4 * (size_t)cgmax, ch,
                       ls.sIdx, ls.sMw, ls.sWi, par);
    }
  }
}
