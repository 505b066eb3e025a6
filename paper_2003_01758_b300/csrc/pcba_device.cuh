// Device-side data structures and small helpers of libpcba (sm_103a).
//
// The list of items (Sec. III-B) of every problem lives in one device arena.
// One item is one contiguous block of item_bytes (a multiple of 256):
//
//   [0, 32)            box: dyadic index per axis (u32[l]); the level per axis
//                      is shared by all items of a problem and kept in its state
//   [32, 48)           cost meta (FP32 mode): f64 offset O, f32 error bound e_p
//   off_cost           cost patch B_p, cp values of T (FP32: stored = value - O)
//   off_eg, off_eh     FP32 mode: error bound per inequality / equality patch, then
//                      (dense families) the patch's FP32 offset o (off_og = off_eg +
//                      4 max(apad, 32), off_oh likewise): stored = value - o
//   off_g              inequality patches, coefficient-major: [cg][apad] of T,
//                      so patch i is the column i ("constraint-minor")
//   off_h              equality patches, [ch][bpad] of T
//
// A linear-family item (pcba_create_linear) stores the K shared patches in the
// inequality block twice (copy_g apart; their error bounds twice, copy_e
// apart): a bisection step reads the copy of its parity and writes the
// children into the other one, so that the several work units of one parent
// can all read it while the left child takes its slot.  After the patches,
// off_sum holds two 64-bit summaries (bit t: chunk t of the activity bits is
// not empty; same alternation) and off_mask one activity bit per constraint
// (mwords words).  An item whose summary is empty - every constraint proven
// to hold on its box - no longer carries its shared patches.
//
// Constraint-minor storage makes every load and store of the subdivision
// kernel unit-stride across the threads of a warp for every bisection
// direction: thread i owns patch i and walks its fibres.
//
// The list order of the paper (children of parent k at positions k and k+K,
// Alg. 2; holes filled from the top, Alg. 5) is kept as a map from logical
// position to physical item slot.  A left child stays in its parent's slot, a
// right child takes a free slot (popped from a per-problem stack, or a slot
// never used before), and Eliminate moves map entries instead of items; the
// slots of eliminated children are pushed back.  At most 2K slots are in use
// during a step, so the memory test 2K <= M is unchanged.
#pragma once

#include <cstdint>

#define PCBA_TPB 256
#define PCBA_MAXD 8
#define PCBA_NONE 0xFFFFFFFFu
#define PCBA_RUNNING 10
#define PCBA_TRACE_PER_DIM 40
#define PCBA_LIN_WORDS 8     // activity words (256 constraints) per linear subdivision unit
#define PCBA_LIN_STRIDE 8    // doubles per linear constraint row (c, w_0 .. w_K-1)
#define PCBA_ESTAGE_BYTES 256  // TMA subdivision stage: 32 FP32 error bounds, then 32 offsets
#define PCBA_FAM_LIN 3        // refresh mark: every shared patch of a linear-family item
#define PCBA_LIN32_STRIDE 16  // floats per FP32 row: the FP64 row rounded, then the remainders
#define PCBA_LIN_BATCH 4     // units a warp of the linear subdivision kernel fetches at once
#ifndef PCBA_LIN_LIGHT_MAX
#define PCBA_LIN_LIGHT_MAX 64  // an item with <= 4 live chunks and at most this many active
                               // constraints is bounded by the split kernel
#endif
#ifndef PCBA_LIN_WIN
#define PCBA_LIN_WIN 64      // active constraints per queued window (unless a single chunk)
#endif
#define PCBA_LIN_IDX 256     // compaction buffer of a warp (constraints per pass)

struct ProbDesc {
  int l;
  int cp, cg, ch;            // coefficients per patch of p, g, h
  int alpha, beta;           // constraint counts
  int apad, bpad;            // padded to multiples of 32
  int tiles_g, tiles_h, tiles;  // subdivision work units per item
  int form_bernstein;        // 1: inputs already Bernstein patches
  int move_chunks;           // compaction work units per item
  int groups_g, groups_h;    // 32-patch column groups per family (TMA subdivision)
  int P[PCBA_MAXD], G[PCBA_MAXD], H[PCBA_MAXD];
  double lo[PCBA_MAXD], hi[PCBA_MAXD];
  long long item_bytes;      // stride of the list
  long long payload_bytes;   // algorithmic bytes of one item (no padding)
  long long off_cost, off_eg, off_eh, off_g, off_h;
  long long off_og, off_oh;  // FP32 dense families: per-patch offsets (0: none)
  long long list_off;        // byte offset of the list in the arena
  long long M;               // capacity in items (memory test of Alg. 1 line 4)
  long long slot_off;        // offset of this problem in the per-slot scratch arrays
  long long tile_off;        // offset in the per-tile scratch array
  long long mono_off;        // offset (doubles) of the monomial input
  long long trace_off;       // offset (rows) in the trace buffer
  int trace_rows;
  int units_k1;              // 1 + alpha + beta patches to convert
  // linear families (pcba_create_linear): alpha = K shared patches, nlin
  // constraints g_i = c_i + sum_m w_im s_m with rows at lin_off of the tables
  int lin, nlin;
  int mwords;                // activity words per item (32 constraints each)
  int lin_chunks;            // subdivision units per item (PCBA_LIN_WORDS words each)
  long long off_mask;        // activity bits of the item
  long long off_sum;         // two u64: bit t set iff chunk t has an active constraint
  long long copy_g, copy_e;  // byte distance between the two copies of the shared
                             // patches / of their error bounds (0: one copy)
  long long lin_off;         // first row of this problem in the constraint tables
};

// Per-child bound record, each field an order-preserving 64-bit key of a
// double so that it can be reduced with integer atomics.  A zero field is the
// identity of a max-reduction ("minus infinity").
struct ChildRec {
  unsigned long long pmin, pmax;      // min / max B_p
  unsigned long long gminmax;         // max_i min B_gi   (infeasible iff > 0)
  unsigned long long gmaxmax;         // max_i max B_gi   (feasible iff <= 0)
  unsigned long long hminmax;         // max_j min B_hj
  unsigned long long hnegmaxmin;      // max_j (-max B_hj) = -(min_j max B_hj)
  unsigned long long habsmax;         // max_j max(max B_hj, -min B_hj)
  unsigned long long perr;            // FP32: bits of the cost patch's error bound e_p
  // vertex incumbents (batch flag 8): per corner, the max over the child's
  // active constraints of (corner value + bound), as okey32 (0: none), and
  // an upper bound of the cost at the corner
  unsigned vtxg[4];
  float vtxc[4];
};

struct ProbState {
  int status;
  int K;            // list length before the next step's subdivision
  int twoK;         // children of the current step
  int K_save;
  int F;            // hole-filling moves of the current step (Alg. 5)
  int r;            // next bisection direction (0-based)
  int n;            // iteration counter n of Alg. 1 (sweeps)
  int steps;
  int level[PCBA_MAXD];
  unsigned long long best_key;  // (slot << 32) | e_p bits of the least slot attaining p_up
  unsigned k3_arrive;
  int have_box;
  int from_warm;
  unsigned best_index[PCBA_MAXD];
  int best_level[PCBA_MAXD];
  unsigned long long pup_key;   // atomicMin over feasible children (this step)
  unsigned long long plo_key;   // atomicMin over kept children (this step)
  double p_up, p_lo;            // reported bounds
  double p_up_carry;            // incumbent carried across steps (or warm start)
  double warm_x[PCBA_MAXD];
  long long peak_items;
  unsigned long long t_end;
  int done_flag;
  int ftop;                     // free-slot stack height before the coming step's pops
  int hw;                       // physical slots >= hw have never been used
  int ftop_push;                // stack height after this step's pops (base of its pushes)
  // levels and count of the children of a step, by the parity of the step:
  // the loop control sets the coming step's while the refresh of the step
  // just done still reads its own
  int child_level[2][PCBA_MAXD];
  int child_twoK[2];
  int seeded;                   // a warm-start candidate was certified feasible
  double seed_cost;             // its certified cost bound (the initial p_up)
  double seed_x[PCBA_MAXD];     // the candidate
  float box_err;                // FP32: e_p of the returned box's cost patch (in p_up)
  double warm_err;              // FP64 rounding bound of the warm point's cost (in p_up)
  unsigned long long vtx_key;   // this step: okey32(corner cost bound) << 32 | child << 2 | corner
};

struct SolveParams {
  double opt_tol, eq_tol;
  int max_iters;
  int max_steps;      // 0: no step limit
  int step_guard;     // hard bound on device loop iterations
  int np;
  unsigned long long time_limit_ns;  // 0: none; else stop running problems (TIMEOUT)
  int vertex;         // vertex incumbents (linear families)
};

struct Plan {
  unsigned k2_units;
  unsigned k3_tiles;
  unsigned k3_tiles_next;
  unsigned k4_units;
  unsigned kr_units;
  unsigned mark_count[2];  // marked patches appended by the subdivision of even / odd steps
  unsigned long long marks_total, refreshed_total;
  unsigned kr_par;               // parity of the step whose marks the refresh takes (set by the subdivision)
  unsigned long long lin_pairs;  // linear families: (child, active constraint) bounds of the solve
  unsigned long long lin_full;   // of which bounded from the coefficient range (not the interval)
  unsigned lin_next;             // next unit of the linear bound kernel to hand out
  unsigned lin_next2;            // next item of the linear split kernel to hand out
  unsigned lin_qcount;           // (item, window) units queued for the linear bound kernel
  unsigned k3_done;
  unsigned k4_done;             // blocks of k_move_control finished (the last one runs the control)
  int any_running;
  int steps_global;
  int guard_hit;
  unsigned long long t0;
};

// Everything a kernel needs, passed by value.
struct Engine {
  int np;
  int precision;           // 32 or 64
  const ProbDesc* desc;
  ProbState* state;
  Plan* plan;
  const SolveParams* params;
  unsigned* k2_pre;        // [np + 1]
  unsigned* k3_pre;        // [np + 1]
  unsigned* k3_pre_next;   // [np + 1]
  unsigned* k4_pre;        // [np + 1]
  unsigned* kr_pre;        // [np + 1] parent items per problem (linear split kernel)
  uint4* marks;            // [2][mark_cap] (problem, child slot, family, patch) of marked patches
  unsigned mark_cap;
  char* arena;
  ChildRec* rec;           // per slot
  unsigned* map;           // per slot: logical list position -> physical item slot
  unsigned* fstack;        // per slot: stack of free physical item slots
  unsigned* flagrank;      // per slot: keep << 31 | rank within its tile
  unsigned* hole;          // per slot
  unsigned* filler;        // per slot
  unsigned* tilecnt;       // per tile: kept count, then exclusive offset
  const double* mono;      // monomial inputs of every problem
  const float* mono32;     // the same rounded to FP32 (filled when candidates are evaluated)
  double* trace;           // rows of (K, K_save, p_up, p_lo)
  const double* warm;      // [np][n_warm][PCBA_MAXD] candidate points, or null
  int n_warm;              // candidates per problem (a row starting with NaN is empty)
  double* root_raw;        // optional FP64 root patch dump
  const unsigned* k1_pre;  // [np + 1] patches per problem prefix
  const void* tmaps;       // [np][2] tensor maps (CUtensorMap) of the g / h blocks, or null
  uint4* lin_queue;        // linear families: (item, window, problem, k) units of heavy items
  unsigned lin_qcap;       // its capacity (a full queue leaves the units to the split kernel)
  const float* lin32;      // linear families: constraint rows in FP32, [rows][16]: the
                           // FP64 row rounded to nearest (8), then the remainders
                           // fl(x - hi) (8), so that hi + lo carries x to 2^-48
  const double* lin64;     // the same in FP64
};

// ---------------------------------------------------------------------------
// order-preserving keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long okey(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
// okey((double)x) of an FP32 x by integer operations alone (the conversion
// is exact; an FP64 conversion would occupy the SM partition's FP64 unit).
__device__ __forceinline__ unsigned long long okey_f32(float x) {
  const unsigned b = __float_as_uint(x), e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  unsigned long long d;
  if (e == 0xffu) {
    d = (0x7ffull << 52) | ((unsigned long long)m << 29);  // infinities, NaN
  } else if (e != 0u) {
    d = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0u) {
    d = 0ull;  // zeros
  } else {
    // subnormal: m 2^-149 with its leading bit at p, a normal FP64 value
    const int p = 31 - __clz(m);
    d = ((unsigned long long)(p + 874) << 52) |
        (((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
  }
  d |= (unsigned long long)(b >> 31) << 63;
  return (d & 0x8000000000000000ull) ? ~d : (d | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_dec(unsigned long long k) {
  unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}
// decode a max-reduced field: 0 means nothing was reduced
__device__ __forceinline__ double okey_dec_max(unsigned long long k) {
  return k == 0ull ? -INFINITY : okey_dec(k);
}
// decode a min-reduced field: all ones means nothing was reduced
__device__ __forceinline__ double okey_dec_min(unsigned long long k) {
  return k == ~0ull ? INFINITY : okey_dec(k);
}

__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
  return __ldcg(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// problem owning work unit u: largest p with pre[p] <= u (pre[0] = 0)
__device__ __forceinline__ int find_problem(const unsigned* pre, int np, unsigned u) {
  int lo = 0, hi = np;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= u) lo = mid; else hi = mid;
  }
  return lo;
}

// Programmatic dependent launch of the per-step kernels: a kernel launched
// with the attribute is scheduled as soon as its predecessor's blocks have
// all left (no explicit trigger: a trigger at the start, which lets the
// blocks of the next kernel wait on the SMs, measured slower), and before
// touching any state it waits for that predecessor's completion and memory.
// A kernel launched without the attribute passes the wait at once.
__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The same search by a whole warp (all 32 lanes, warp-uniform u): each round
// splits [lo, hi) into 32 parts and reads one boundary per lane, so 1024
// problems take two dependent loads instead of ten.
__device__ __forceinline__ int find_problem_warp(const unsigned* pre, int np, unsigned u,
                                                 int lane) {
  int lo = 0, hi = np;  // pre[lo] <= u; the answer lies in [lo, hi)
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const int idx = lo + lane * step;
    const unsigned b = __ballot_sync(0xffffffffu, idx < hi && __ldg(pre + idx) <= u);
    lo += (31 - __clz(b)) * step;  // lane 0 reads pre[lo] <= u: b != 0
    hi = min(hi, lo + step);
  }
  return lo;
}

// ---------------------------------------------------------------------------
// block-wide reductions and scans (PCBA_TPB threads)
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_max(double (&v)[NV], double* smem /* 8*NV */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) smem[wid * NV + q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double m = smem[q];
    for (int w = 1; w < PCBA_TPB / 32; ++w) m = fmax(m, smem[w * NV + q]);
    v[q] = m;
  }
  __syncthreads();
}

// exclusive scan of one unsigned per thread; returns the exclusive prefix and
// writes the block total to *total
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned x, unsigned* smem /* 8 */,
                                                        unsigned* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) smem[wid] = inc;
  __syncthreads();
  unsigned woff = 0, tot = 0;
  for (int w = 0; w < PCBA_TPB / 32; ++w) {
    if (w < wid) woff += smem[w];
    tot += smem[w];
  }
  __syncthreads();
  *total = tot;
  return woff + inc - x;
}

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

// order-preserving 32-bit key of a float (0 = below everything)
__device__ __forceinline__ unsigned okey32(float x) {
  const unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float okey32_dec(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Flat index of corner q of a patch of multi-degree deg (row-major, last
// axis fastest): bit a of q (a < 2) selects the upper end of axis a, later
// axes stay at their lower end.  The coefficient there is the polynomial's
// value at that corner of the box (Sec. II-D).
__device__ __forceinline__ int corner_index(const int* deg, int l, int q) {
  int idx = 0;
  for (int a = 0; a < l; ++a) idx = idx * (deg[a] + 1) + ((a < 2 && ((q >> a) & 1)) ? deg[a] : 0);
  return idx;
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
  c.perr = __ldcg(s + 7);
  return c;
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
