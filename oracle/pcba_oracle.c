/*
 * PCBA oracle: a plain, slow, single-threaded FP64 implementation of the
 * Parallel Constrained Bernstein Algorithm (arXiv 2003.01758).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker for the CUDA library in
 * paper_2003_01758_b300/.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no source,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Every routine follows a passage of the paper, cited by section, equation,
 * definition or algorithm:
 *   - polynomial notation, multi-degree                 Sec. II-A, Def. 1
 *   - POP (P)                                           Sec. II-B, Eq. (P)
 *   - Bernstein form and patch                          Sec. II-D, Eq. (BF)
 *   - range enclosure                                   Sec. II-D, Thm. 1
 *   - subdivision into x_L, x_R                         Sec. II-E
 *   - PCBA main loop                                    Sec. III, Algorithm 1
 *   - items and the list                                Sec. III-B
 *   - tolerances and stopping                           Sec. III-C, Def. 2
 *   - Subdivision                                       Sec. III-D, Alg. 2
 *   - feasible / infeasible / undecided                 Sec. III-E, Def. 3
 *   - solution estimate p_up, suboptimal                Def. 4, Def. 5
 *   - FindBounds, CutOffTest, Eliminate                 Alg. 3, 4, 5
 *   - memory per item                                   Sec. IV-C, Eq. (memory_per_item)
 *
 * Readings taken where the paper is garbled or silent (each is listed with its
 * reason in the design notes of the repository):
 *   R1  the direction cycles r = 1, 2, ..., l, 1, ...; n grows by one each
 *       time r returns to 1 (Sec. III-D; Alg. 1 line 11 as printed would keep
 *       r at 1 when l = 2).
 *   R2  max_iters counts sweeps n; Alg. 1 returns when n reaches N after the
 *       update of line 11, i.e. after (N-1)*l steps at most.
 *   R3  an item is kept iff it is not infeasible (Def. 3 (c)-(e)) and it is not
 *       suboptimal (Def. 5).  Alg. 4 as printed also demands the equality
 *       window of Def. 3 (b) to keep an item, which would eliminate every
 *       undecided item once beta > 0.
 *   R4  the conditions over i and j in Alg. 4 hold "for all i" / "for all j"
 *       as in Def. 3.
 *   R5  p_lo = min over kept items of min B_p (a sound lower bound: every
 *       feasible point lies in a kept item by Cor. 2).
 *   R6  stop when p_up - p_lo <= eps (Alg. 1 line 9; Def. 2 (d)); the step
 *       tolerance delta is used only when it is positive.
 *   R8  the memory test of Alg. 1 line 4 compares 2*K with M = max_items.
 *   R9  the returned box is the feasible item with max B_p = p_up that sits at
 *       the lowest list position (the list order is the paper's, Alg. 2 and
 *       Alg. 5, so it is deterministic).
 *   R10 the returned point is the centre of that box.
 *   R11 Alg. 5: holes are the eliminated slots below K_save; the k-th hole
 *       (ascending) receives the item at save-list position K_save-1-k.
 *   R14 boxes are stored as dyadic integers: one level per axis (shared by
 *       every item, since all items are bisected alike) and one index per axis.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXDIM 8

enum {
  OR_OPTIMAL = 0,
  OR_INFEASIBLE = 1,
  OR_MEMCAP = 2,
  OR_MAXITER = 3,
  OR_RUNNING = 10,
  OR_ERR_INVALID = -1,
  OR_ERR_OOM = -3
};

/* ------------------------------------------------------------------------- */
/* Small exact helpers                                                        */
/* ------------------------------------------------------------------------- */

/* Binomial coefficient C(n, k) in double; exact for the degrees used here
 * (n <= 60 keeps every partial product an integer below 2^53). */
static double or_binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  if (k > n - k) k = n - k;
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
  return c;
}

static double or_ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

/* Number of coefficients of a dense tensor of multi-degree N: Pi(N+1)
 * (Sec. IV-C, notation of Eq. (memory_per_item)). */
static long or_count(int l, const int* N) {
  long c = 1;
  for (int r = 0; r < l; ++r) c *= (long)(N[r] + 1);
  return c;
}

/* Row-major strides, axis 0 slowest. */
static void or_strides(int l, const int* N, long* stride) {
  long s = 1;
  for (int r = l - 1; r >= 0; --r) {
    stride[r] = s;
    s *= (long)(N[r] + 1);
  }
}

/* ------------------------------------------------------------------------- */
/* Monomial to Bernstein form over a box (Sec. II-D, Eq. (BF);                */
/* Assumption 1 maps the box affinely onto the unit box).                     */
/* ------------------------------------------------------------------------- */

/* One axis of the conversion, applied to every fibre along axis r.
 * Step (i): substitute x_r = lo + w t (w = hi - lo) and collect powers of t:
 *     c_k = sum_{j >= k} a_j C(j,k) lo^(j-k) w^k.
 * Step (ii): power basis of degree n on [0,1] to Bernstein basis:
 *     b_i = sum_{k <= i} [C(i,k) / C(n,k)] c_k.
 * Both are the textbook definitions, summed directly. */
static void or_convert_axis(int l, const int* N, double* t, int r, double lo,
                            double hi) {
  long stride[OR_MAXDIM] = {0};
  or_strides(l, N, stride);
  const int n = N[r];
  const long total = or_count(l, N);
  const long block = (long)(n + 1) * stride[r];
  const double w = hi - lo;
  double a[64], c[64];
  for (long base = 0; base < total; base += block) {
    for (long in = 0; in < stride[r]; ++in) {
      for (int j = 0; j <= n; ++j) a[j] = t[base + in + (long)j * stride[r]];
      for (int k = 0; k <= n; ++k) {
        double s = 0.0;
        for (int j = k; j <= n; ++j)
          s += a[j] * or_binom(j, k) * or_ipow(lo, j - k) * or_ipow(w, k);
        c[k] = s;
      }
      for (int i = 0; i <= n; ++i) {
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s += or_binom(i, k) / or_binom(n, k) * c[k];
        t[base + in + (long)i * stride[r]] = s;
      }
    }
  }
}

/* Bernstein patch B(x) of the polynomial with monomial coefficients a over
 * the box [lo, hi] (Sec. II-D).  a and b are dense row-major tensors of
 * multi-degree N.  Returns 0, or OR_ERR_INVALID for a bad shape. */
int or_bernstein_from_monomial(int l, const int* N, const double* a,
                               const double* lo, const double* hi, double* b) {
  if (l < 1 || l > OR_MAXDIM) return OR_ERR_INVALID;
  for (int r = 0; r < l; ++r)
    if (N[r] < 0 || N[r] > 60 || !(lo[r] < hi[r])) return OR_ERR_INVALID;
  const long total = or_count(l, N);
  memcpy(b, a, sizeof(double) * (size_t)total);
  for (int r = 0; r < l; ++r) or_convert_axis(l, N, b, r, lo[r], hi[r]);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Evaluation (used by the tests and by the check of the returned point).    */
/* ------------------------------------------------------------------------- */

/* p(x) = sum_{J <= N} a_J x^J (Sec. II-A, Eq. (poly_monomial_basis)). */
double or_eval_monomial(int l, const int* N, const double* a, const double* x) {
  const long total = or_count(l, N);
  long stride[OR_MAXDIM] = {0};
  or_strides(l, N, stride);
  double s = 0.0;
  for (long idx = 0; idx < total; ++idx) {
    double term = a[idx];
    for (int r = 0; r < l; ++r) {
      int j = (int)((idx / stride[r]) % (N[r] + 1));
      term *= or_ipow(x[r], j);
    }
    s += term;
  }
  return s;
}

/* p(x) = sum_J B_J b_J(x, x) with the Bernstein basis of multi-degree N over
 * the box [lo, hi]: b_J = prod_r C(n_r, j_r) t_r^j_r (1 - t_r)^(n_r - j_r),
 * t_r = (x_r - lo_r) / (hi_r - lo_r) (Sec. II-D, Eq. (BF)). */
double or_eval_bernstein(int l, const int* N, const double* b, const double* lo,
                         const double* hi, const double* x) {
  const long total = or_count(l, N);
  long stride[OR_MAXDIM] = {0};
  or_strides(l, N, stride);
  double s = 0.0;
  for (long idx = 0; idx < total; ++idx) {
    double term = b[idx];
    for (int r = 0; r < l; ++r) {
      int j = (int)((idx / stride[r]) % (N[r] + 1));
      double t = (x[r] - lo[r]) / (hi[r] - lo[r]);
      term *= or_binom(N[r], j) * or_ipow(t, j) * or_ipow(1.0 - t, N[r] - j);
    }
    s += term;
  }
  return s;
}

/* ------------------------------------------------------------------------- */
/* Subdivision (Sec. II-E): bisect the box in direction r and compute the     */
/* patches over x_L and x_R.  Each fibre along axis r is split by the de      */
/* Casteljau triangle at 1/2:                                                 */
/*     q_j^(0) = f_j,   q_j^(k) = (q_j^(k-1) + q_{j+1}^(k-1)) / 2,            */
/*     left_i = q_0^(i),   right_i = q_i^(n-i).                               */
/* ------------------------------------------------------------------------- */

int or_subdivide_patch(int l, const int* N, const double* b, int r, double* left,
                       double* right) {
  if (l < 1 || l > OR_MAXDIM || r < 0 || r >= l || N[r] > 60) return OR_ERR_INVALID;
  long stride[OR_MAXDIM] = {0};
  or_strides(l, N, stride);
  const int n = N[r];
  const long total = or_count(l, N);
  const long block = (long)(n + 1) * stride[r];
  double q[64];
  for (long base = 0; base < total; base += block) {
    for (long in = 0; in < stride[r]; ++in) {
      const long off = base + in;
      for (int j = 0; j <= n; ++j) q[j] = b[off + (long)j * stride[r]];
      left[off] = q[0];
      right[off + (long)n * stride[r]] = q[n];
      for (int k = 1; k <= n; ++k) {
        for (int j = 0; j <= n - k; ++j) q[j] = (q[j] + q[j + 1]) / 2.0;
        left[off + (long)k * stride[r]] = q[0];
        right[off + (long)(n - k) * stride[r]] = q[n - k];
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* The list of items (Sec. III-B).  An item holds its box and the patches of  */
/* p, every g_i and every h_j; here one item is one contiguous run of         */
/* doubles: [B_p | B_g1 ... B_galpha | B_h1 ... B_hbeta].                     */
/* ------------------------------------------------------------------------- */

typedef struct {
  double pmin, pmax;   /* min B_p, max B_p                     */
  double* gmin;        /* per inequality: min B_gi             */
  double* gmax;        /* per inequality: max B_gi             */
  double* hmin;        /* per equality:   min B_hj             */
  double* hmax;        /* per equality:   max B_hj             */
} or_bounds;

typedef struct {
  int K;               /* list length before the step's subdivision */
  int K_save;          /* kept items after CutOffTest              */
  double p_up, p_lo;   /* solution estimate and lower bound        */
} or_trace_rec;

typedef struct or_state {
  int l;
  double lo[OR_MAXDIM], hi[OR_MAXDIM];
  int P[OR_MAXDIM], G[OR_MAXDIM], H[OR_MAXDIM];
  int n_ineq, n_eq;
  long cp, cg, ch;     /* coefficients per patch of each family   */
  long item_len;       /* doubles per item                        */
  long long max_items; /* M of Alg. 1                             */

  /* the list */
  long cap;            /* allocated items                         */
  long K;              /* current length                          */
  double* patches;     /* cap * item_len                          */
  uint32_t* index;     /* cap * l dyadic box indices              */
  int level[OR_MAXDIM];/* shared dyadic level per axis            */
  or_bounds* bounds;   /* cap records                             */
  double* bnd_store;   /* backing store of per-patch bounds       */
  unsigned char* keep; /* cap flags                               */

  /* iteration state (Alg. 1 line 3) */
  int n, r, steps, status;
  double p_up, p_lo;
  int have_best;
  uint32_t best_index[OR_MAXDIM];
  int best_level[OR_MAXDIM];
  long long peak_items;

  or_trace_rec* trace;
  long trace_len, trace_cap;
} or_state;

static void or_free_state(or_state* s) {
  if (!s) return;
  free(s->patches);
  free(s->index);
  free(s->bounds);
  free(s->bnd_store);
  free(s->keep);
  free(s->trace);
  free(s);
}

void or_destroy(or_state* s) { or_free_state(s); }

/* Grow the list storage to hold at least want items. */
static int or_reserve(or_state* s, long want) {
  if (want <= s->cap) return 0;
  long nc = s->cap ? s->cap : 16;
  while (nc < want) nc *= 2;
  double* p = (double*)realloc(s->patches, sizeof(double) * (size_t)(nc * s->item_len));
  if (!p) return OR_ERR_OOM;
  s->patches = p;
  uint32_t* ix = (uint32_t*)realloc(s->index, sizeof(uint32_t) * (size_t)(nc * s->l));
  if (!ix) return OR_ERR_OOM;
  s->index = ix;
  unsigned char* kp = (unsigned char*)realloc(s->keep, (size_t)nc);
  if (!kp) return OR_ERR_OOM;
  s->keep = kp;
  const long per = 2 * (long)s->n_ineq + 2 * (long)s->n_eq;
  free(s->bounds);
  free(s->bnd_store);
  s->bounds = (or_bounds*)calloc((size_t)nc, sizeof(or_bounds));
  s->bnd_store = (double*)calloc((size_t)(nc * (per > 0 ? per : 1)), sizeof(double));
  if (!s->bounds || !s->bnd_store) return OR_ERR_OOM;
  for (long k = 0; k < nc; ++k) {
    double* base = s->bnd_store + k * per;
    s->bounds[k].gmin = base;
    s->bounds[k].gmax = base + s->n_ineq;
    s->bounds[k].hmin = base + 2 * s->n_ineq;
    s->bounds[k].hmax = base + 2 * s->n_ineq + s->n_eq;
  }
  s->cap = nc;
  return 0;
}

/* Alg. 1 lines 1-3: InitPatches over the domain and the one-item list.
 * form = 0: cost/ineq/eq hold monomial coefficients over the box [lo, hi]
 *           and are converted here (Sec. II-D);
 * form = 1: they already hold the Bernstein patches over [lo, hi].
 * Each family is given at one common multi-degree (P, G, H; Sec. IV-C):
 * ineq is n_ineq consecutive tensors of multi-degree G, eq n_eq tensors of H. */
or_state* or_create(int l, const double* lo, const double* hi, const int* P,
                    const double* cost, int n_ineq, const int* G, const double* ineq,
                    int n_eq, const int* H, const double* eq, int form,
                    long long max_items) {
  if (l < 1 || l > OR_MAXDIM || n_ineq < 0 || n_eq < 0 || max_items < 1) return NULL;
  or_state* s = (or_state*)calloc(1, sizeof(or_state));
  if (!s) return NULL;
  s->l = l;
  for (int r = 0; r < l; ++r) {
    if (!(lo[r] < hi[r])) { or_free_state(s); return NULL; }
    s->lo[r] = lo[r];
    s->hi[r] = hi[r];
    s->P[r] = P[r];
    s->G[r] = n_ineq ? G[r] : 0;
    s->H[r] = n_eq ? H[r] : 0;
  }
  s->n_ineq = n_ineq;
  s->n_eq = n_eq;
  s->cp = or_count(l, s->P);
  s->cg = n_ineq ? or_count(l, s->G) : 0;
  s->ch = n_eq ? or_count(l, s->H) : 0;
  s->item_len = s->cp + (long)n_ineq * s->cg + (long)n_eq * s->ch;
  s->max_items = max_items;
  if (or_reserve(s, 2)) { or_free_state(s); return NULL; }

  double* it = s->patches;
  if (form == 0) {
    if (or_bernstein_from_monomial(l, s->P, cost, lo, hi, it)) { or_free_state(s); return NULL; }
    for (int i = 0; i < n_ineq; ++i)
      if (or_bernstein_from_monomial(l, s->G, ineq + (long)i * s->cg, lo, hi,
                                     it + s->cp + (long)i * s->cg)) { or_free_state(s); return NULL; }
    for (int j = 0; j < n_eq; ++j)
      if (or_bernstein_from_monomial(l, s->H, eq + (long)j * s->ch, lo, hi,
                                     it + s->cp + (long)n_ineq * s->cg + (long)j * s->ch)) {
        or_free_state(s);
        return NULL;
      }
  } else {
    memcpy(it, cost, sizeof(double) * (size_t)s->cp);
    if (n_ineq) memcpy(it + s->cp, ineq, sizeof(double) * (size_t)(n_ineq * s->cg));
    if (n_eq)
      memcpy(it + s->cp + (long)n_ineq * s->cg, eq, sizeof(double) * (size_t)(n_eq * s->ch));
  }
  for (int r = 0; r < l; ++r) {
    s->index[r] = 0;
    s->level[r] = 0;
  }
  s->K = 1;
  s->n = 1;       /* Alg. 1 line 3 */
  s->r = 0;       /* direction 1, zero-based */
  s->steps = 0;
  s->status = OR_RUNNING;
  s->p_up = INFINITY;
  s->p_lo = -INFINITY;
  s->peak_items = 1;
  return s;
}

/* Alg. 2 (Subdivision) for one item: item k becomes x_L in place and its right
 * half goes to slot k + K. */
static void or_subdivide_item(or_state* s, long k, long K) {
  const int l = s->l, r = s->r;
  double* src = s->patches + k * s->item_len;
  double* dst = s->patches + (k + K) * s->item_len;
  double* tmpL = (double*)malloc(sizeof(double) * (size_t)s->item_len);
  /* cost */
  or_subdivide_patch(l, s->P, src, r, tmpL, dst);
  /* inequalities */
  for (int i = 0; i < s->n_ineq; ++i) {
    long off = s->cp + (long)i * s->cg;
    or_subdivide_patch(l, s->G, src + off, r, tmpL + off, dst + off);
  }
  /* equalities */
  for (int j = 0; j < s->n_eq; ++j) {
    long off = s->cp + (long)s->n_ineq * s->cg + (long)j * s->ch;
    or_subdivide_patch(l, s->H, src + off, r, tmpL + off, dst + off);
  }
  memcpy(src, tmpL, sizeof(double) * (size_t)s->item_len);
  free(tmpL);
  /* boxes: x_L keeps the lower half, x_R the upper half of axis r */
  for (int q = 0; q < l; ++q) s->index[(k + K) * l + q] = s->index[k * l + q];
  s->index[k * l + r] = 2u * s->index[k * l + r];
  s->index[(k + K) * l + r] = 2u * s->index[(k + K) * l + r] + 1u;
}

static void or_patch_minmax(const double* b, long c, double* mn, double* mx) {
  double a = b[0], z = b[0];
  for (long i = 1; i < c; ++i) {
    if (b[i] < a) a = b[i];
    if (b[i] > z) z = b[i];
  }
  *mn = a;
  *mx = z;
}

/* Alg. 3 (FindBounds) for one item. */
static void or_find_bounds(or_state* s, long k) {
  const double* it = s->patches + k * s->item_len;
  or_bounds* bd = &s->bounds[k];
  or_patch_minmax(it, s->cp, &bd->pmin, &bd->pmax);
  for (int i = 0; i < s->n_ineq; ++i)
    or_patch_minmax(it + s->cp + (long)i * s->cg, s->cg, &bd->gmin[i], &bd->gmax[i]);
  for (int j = 0; j < s->n_eq; ++j)
    or_patch_minmax(it + s->cp + (long)s->n_ineq * s->cg + (long)j * s->ch, s->ch,
                    &bd->hmin[j], &bd->hmax[j]);
}

/* Def. 3 (a)-(b): feasible. */
static int or_is_feasible(const or_state* s, const or_bounds* bd, double eq_tol) {
  for (int i = 0; i < s->n_ineq; ++i)
    if (!(bd->gmax[i] <= 0.0)) return 0;
  for (int j = 0; j < s->n_eq; ++j)
    if (!(-eq_tol <= bd->hmin[j] && bd->hmin[j] <= 0.0 && 0.0 <= bd->hmax[j] &&
          bd->hmax[j] <= eq_tol))
      return 0;
  return 1;
}

/* Def. 3 (c)-(e): infeasible. */
static int or_is_infeasible(const or_state* s, const or_bounds* bd) {
  for (int i = 0; i < s->n_ineq; ++i)
    if (bd->gmin[i] > 0.0) return 1;
  for (int j = 0; j < s->n_eq; ++j)
    if (bd->hmin[j] > 0.0 || bd->hmax[j] < 0.0) return 1;
  return 0;
}

static void or_push_trace(or_state* s, int K, int K_save) {
  if (s->trace_len == s->trace_cap) {
    long nc = s->trace_cap ? 2 * s->trace_cap : 64;
    or_trace_rec* t = (or_trace_rec*)realloc(s->trace, sizeof(or_trace_rec) * (size_t)nc);
    if (!t) return;
    s->trace = t;
    s->trace_cap = nc;
  }
  or_trace_rec* t = &s->trace[s->trace_len++];
  t->K = K;
  t->K_save = K_save;
  t->p_up = s->p_up;
  t->p_lo = s->p_lo;
}

/* One pass of Alg. 1 lines 4-11 in direction r.  Returns the status:
 * OR_RUNNING to continue, or the final outcome. */
int or_step(or_state* s, double opt_tol, double eq_tol, int max_iters, double step_tol) {
  if (s->status != OR_RUNNING) return s->status;
  const int l = s->l;
  const long K = s->K;

  /* dyadic indices are 32-bit: a 32nd bisection of one axis ends the run */
  if (s->level[s->r] >= 31) {
    s->status = OR_MAXITER;
    return s->status;
  }
  /* line 4: memory test (R8) */
  if (2 * (long long)K > s->max_items) {
    s->status = OR_MEMCAP;
    return s->status;
  }
  if (or_reserve(s, 2 * K)) return OR_ERR_OOM;

  /* line 5: Alg. 2, every item k -> slots k and k + K */
  for (long k = 0; k < K; ++k) or_subdivide_item(s, k, K);
  s->level[s->r] += 1;
  const long K2 = 2 * K;
  if (K2 > s->peak_items) s->peak_items = K2;

  /* line 6: Alg. 3 */
  for (long k = 0; k < K2; ++k) or_find_bounds(s, k);

  /* line 7: Alg. 4 with readings R3-R5.  Solution estimate (Def. 4). */
  double p_up = INFINITY;
  long best = -1;
  for (long k = 0; k < K2; ++k) {
    if (or_is_feasible(s, &s->bounds[k], eq_tol)) {
      if (s->bounds[k].pmax < p_up) {  /* strict: the lowest position wins (R9) */
        p_up = s->bounds[k].pmax;
        best = k;
      }
    }
  }
  /* keep = not infeasible and not suboptimal (Def. 5) */
  double p_lo = INFINITY;
  long K_save = 0;
  for (long k = 0; k < K2; ++k) {
    const or_bounds* bd = &s->bounds[k];
    int keep = !or_is_infeasible(s, bd) && bd->pmin <= p_up;
    s->keep[k] = (unsigned char)keep;
    if (keep) {
      K_save++;
      if (bd->pmin < p_lo) p_lo = bd->pmin;
    }
  }
  s->p_up = p_up;
  s->p_lo = p_lo;
  if (best >= 0) {
    s->have_best = 1;
    for (int q = 0; q < l; ++q) {
      s->best_index[q] = s->index[best * l + q];
      s->best_level[q] = s->level[q];
    }
  }
  s->steps += 1;
  or_push_trace(s, (int)K, (int)K_save);

  /* line 8: every item infeasible */
  if (K_save == 0) {
    s->K = K2;
    s->status = OR_INFEASIBLE;
    return s->status;
  }

  /* line 9: stopping criteria (Def. 2, R6) */
  int width_ok = 1;
  if (step_tol > 0.0) {
    for (int q = 0; q < l; ++q)
      if (ldexp(s->hi[q] - s->lo[q], -s->level[q]) > step_tol) width_ok = 0;
  }
  if (p_up - p_lo <= opt_tol && width_ok) {
    s->K = K2;
    s->status = OR_OPTIMAL;
    return s->status;
  }

  /* line 10: Alg. 5 (Eliminate), reading R11.  Build L_save and L_elim in
   * ascending order, then fill each hole below K_save with the item at
   * save-list position K_save - 1 - k. */
  long* save = (long*)malloc(sizeof(long) * (size_t)K_save);
  long* elim = (long*)malloc(sizeof(long) * (size_t)(K2 - K_save + 1));
  long ns = 0, ne = 0;
  for (long k = 0; k < K2; ++k) {
    if (s->keep[k]) save[ns++] = k;
    else elim[ne++] = k;
  }
  long K_replace = 0;
  while (K_replace < ne && elim[K_replace] < K_save) K_replace++;
  for (long k = 0; k < K_replace; ++k) {
    long dst = elim[k], src = save[K_save - 1 - k];
    memcpy(s->patches + dst * s->item_len, s->patches + src * s->item_len,
           sizeof(double) * (size_t)s->item_len);
    for (int q = 0; q < l; ++q) s->index[dst * l + q] = s->index[src * l + q];
  }
  free(save);
  free(elim);
  s->K = K_save;

  /* line 11: next direction (R1) and the iteration cap (R2) */
  s->r = (s->r + 1) % l;
  if (s->r == 0) s->n += 1;
  if (s->n >= max_iters) {
    s->status = OR_MAXITER;
    return s->status;
  }
  return OR_RUNNING;
}

/* Runs Alg. 1 to completion.  out receives, in order:
 *   [0] status, [1] p_lo, [2] p_up, [3] steps, [4] n (sweeps), [5] peak items,
 *   [6 .. 6+l) returned point x*, [6+l .. 6+2l) box lower corner,
 *   [6+2l .. 6+3l) box upper corner.
 * p_up = +inf and a NaN point when no feasible item was ever found. */
int or_solve(or_state* s, double opt_tol, double eq_tol, int max_iters, double step_tol,
             double* out) {
  int st = s->status;
  while (st == OR_RUNNING) st = or_step(s, opt_tol, eq_tol, max_iters, step_tol);
  const int l = s->l;
  out[0] = (double)st;
  out[1] = s->p_lo;
  out[2] = s->p_up;
  out[3] = (double)s->steps;
  out[4] = (double)s->n;
  out[5] = (double)s->peak_items;
  for (int q = 0; q < l; ++q) {
    if (s->have_best && st != OR_INFEASIBLE) {
      double w = ldexp(s->hi[q] - s->lo[q], -s->best_level[q]);
      double blo = s->lo[q] + w * (double)s->best_index[q];
      double bhi = s->lo[q] + w * (double)(s->best_index[q] + 1u);
      out[6 + l + q] = blo;
      out[6 + 2 * l + q] = bhi;
      out[6 + q] = 0.5 * (blo + bhi);
    } else {
      out[6 + q] = NAN;
      out[6 + l + q] = NAN;
      out[6 + 2 * l + q] = NAN;
    }
  }
  return st;
}

/* ---- accessors for the tests ------------------------------------------- */

long or_list_length(const or_state* s) { return s->K; }
long or_item_len(const or_state* s) { return s->item_len; }
long or_trace_length(const or_state* s) { return s->trace_len; }
int or_status(const or_state* s) { return s->status; }

/* Copies the first K items: patches (K * item_len doubles, layout
 * [B_p | B_g1..B_galpha | B_h1..B_hbeta]), box indices (K * l) and the
 * shared levels (l). */
void or_get_list(const or_state* s, double* patches, uint32_t* index, int* level) {
  memcpy(patches, s->patches, sizeof(double) * (size_t)(s->K * s->item_len));
  memcpy(index, s->index, sizeof(uint32_t) * (size_t)(s->K * s->l));
  for (int q = 0; q < s->l; ++q) level[q] = s->level[q];
}

/* Copies the keep flags of the last CutOffTest (length 2K of that step). */
void or_get_keep(const or_state* s, unsigned char* keep, long count) {
  memcpy(keep, s->keep, (size_t)count);
}

/* Trace rows: [K, K_save, p_up, p_lo] per step. */
void or_get_trace(const or_state* s, double* rows) {
  for (long t = 0; t < s->trace_len; ++t) {
    rows[4 * t + 0] = (double)s->trace[t].K;
    rows[4 * t + 1] = (double)s->trace[t].K_save;
    rows[4 * t + 2] = s->trace[t].p_up;
    rows[4 * t + 3] = s->trace[t].p_lo;
  }
}

/* Number of list entries of one item per Eq. (memory_per_item):
 * 2l + Pi(P+1) + alpha Pi(G+1) + beta Pi(H+1). */
long long or_memory_per_item(int l, const int* P, int n_ineq, const int* G, int n_eq,
                             const int* H) {
  long long e = 2LL * l + or_count(l, P);
  if (n_ineq) e += (long long)n_ineq * or_count(l, G);
  if (n_eq) e += (long long)n_eq * or_count(l, H);
  return e;
}
