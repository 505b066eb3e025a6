/*
 * pcba.h - C ABI of libpcba.so, a B300 (sm_103a) implementation of the
 * Parallel Constrained Bernstein Algorithm (PCBA) of
 * "Safe, Optimal, Real-time Trajectory Planning with a Parallel Constrained
 * Bernstein Algorithm" (arXiv 2003.01758).
 *
 * The library solves polynomial optimisation problems (POPs, Eq. (P)):
 *
 *     min p(x)   s.t.  g_i(x) <= 0 (i = 1..alpha),  h_j(x) = 0 (j = 1..beta),
 *     x in the box D = [lo_1, hi_1] x ... x [lo_l, hi_l],
 *
 * by the branch and bound of Algorithm 1: every surviving box of the list is
 * bisected (Alg. 2), every Bernstein patch is bounded by the min and max of its
 * coefficients (Thm. 1, Alg. 3), the solution estimate p_up is the least upper
 * bound over feasible items (Def. 4), infeasible and suboptimal items are cut
 * off (Def. 3, Def. 5, Thm. 3, Alg. 4) and the list is compacted in place
 * (Alg. 5).  The result is a certified interval [lower, upper] on the optimum
 * and a point whose box achieved the upper bound.
 *
 * Conventions
 *   - Every function returns 0 on success or a negative PCBA_ERR_* code;
 *     pcba_last_error() then gives a static, thread-local message.
 *   - Host arrays passed in are copied; the caller keeps ownership.  A handle
 *     owns its device memory until pcba_destroy.
 *   - A non-negative result.status is a solver outcome, not an error.
 *   - Polynomials are dense monomial tensors in row-major order, axis 0
 *     slowest: coeff[j_1 (N_2+1)...(N_l+1) + ... + j_l] multiplies
 *     x_1^j_1 ... x_l^j_l (Sec. II-A, Eq. (poly_monomial_basis)).
 *   - One handle is used by one host thread at a time.
 *   - l <= PCBA_MAX_DIM, every multi-degree entry <= PCBA_MAX_DEGREE, and a
 *     patch has at most PCBA_MAX_PATCH coefficients; larger inputs are
 *     rejected with PCBA_ERR_INVALID.
 */
#ifndef PCBA_H_
#define PCBA_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PCBA_MAX_DIM 8
#define PCBA_MAX_DEGREE 16
#define PCBA_MAX_PATCH 8192
#define PCBA_MAX_SHARED 4

/* Solver outcomes (result.status) and error codes (return values). */
enum {
  PCBA_OPTIMAL = 0,      /* p_up - p_lo <= opt_tol (Alg. 1 line 9, Def. 2)      */
  PCBA_INFEASIBLE = 1,   /* every item infeasible: certified (Alg. 1 line 8)    */
  PCBA_MEMCAP = 2,       /* 2 * length(L) > M (Alg. 1 line 4); best so far      */
  PCBA_MAXITER = 3,      /* the sweep counter reached max_iters (Alg. 1 line 11) */
  PCBA_TIMEOUT = 4,      /* the time limit ran out (pcba_set_time_limit); best so far */
  PCBA_STEPLIMIT = 5,    /* stopped after max_steps steps (pcba_solve_steps)     */
  PCBA_ERR_INVALID = -1, /* bad argument                                         */
  PCBA_ERR_CUDA = -2,    /* a CUDA runtime call failed                           */
  PCBA_ERR_OOM = -3,     /* device allocation failed                             */
  PCBA_ERR_DEVICE_TIMEOUT = -4 /* the device loop hit its step guard             */
};

/* Arithmetic of the list (pcba_create 'precision'). */
enum {
  PCBA_FP64 = 64, /* plain IEEE double patches, no rounding control, as the
                     paper's method; bit-for-bit reproducible                   */
  PCBA_FP32 = 32  /* float patches with a per-patch error bound kept with
                     directed rounding, so every bound encloses the exact range
                     (Thm. 1 holds for the stored patches); the root patches are
                     converted in FP64 and the returned point is checked in FP64 */
};

typedef struct pcba_handle pcba_handle;
typedef struct pcba_batch pcba_batch;

/* A polynomial in nvars variables of multi-degree degree[0..nvars) (Def. 1),
 * coefficient tensor of prod(degree[r]+1) doubles. */
typedef struct {
  int nvars;
  const int* degree;
  const double* coeff;
} pcba_poly;

/* The box domain D (Sec. II-A); lo[r] < hi[r]. */
typedef struct {
  int nvars;
  const double* lo;
  const double* hi;
} pcba_box;

/* One solve's outcome. */
typedef struct {
  int status;               /* PCBA_OPTIMAL .. PCBA_STEPLIMIT                      */
  int steps;                /* bisection steps done (one direction each)           */
  int sweeps;               /* iteration counter n of Alg. 1 at return             */
  int from_warm_start;      /* 1 if 'upper' and 'x' come from a certified warm point */
  double lower;             /* certified lower bound p_lo (Alg. 4; +inf if none)   */
  double upper;             /* solution estimate p_up (Def. 4; +inf if no feasible item) */
  double x[PCBA_MAX_DIM];   /* returned point: centre of the box achieving 'upper' */
  double box_lo[PCBA_MAX_DIM], box_hi[PCBA_MAX_DIM]; /* that box (Alg. 1 line 12)  */
  long long peak_items;     /* largest list length 2K reached                      */
  long long peak_bytes;     /* peak_items * stored bytes per item                  */
  double verify_cost;       /* p(x) evaluated in FP64                              */
  double verify_max_g;      /* max_i g_i(x) + its FP64 rounding bound              */
  double verify_max_abs_h;  /* max_j |h_j(x)| + its FP64 rounding bound            */
  double time_ms;           /* device time from the batch start to this problem's end */
  double upper_err;         /* the rounding-error bound included in 'upper': FP32, the
                               bound e_p of the returned box's cost patch (upper = its
                               largest stored coefficient + e_p); a warm point, the FP64
                               bound of its cost evaluation; a vertex incumbent (batch
                               flag 8), the e_p of the cost patch whose corner it is;
                               FP64 boxes and corners: 0                               */
} pcba_result;

/* Builds a problem: cost p (Eq. (P)), n_ineq inequality constraints g_i <= 0,
 * n_eq equality constraints h_j = 0 and the box.  All polynomials must have
 * box->nvars variables.  Each constraint family is zero-padded to one common
 * multi-degree G (resp. H), which leaves the polynomials unchanged (Sec. IV-C,
 * Eq. (memory_per_item)).  precision is PCBA_FP64 or PCBA_FP32.  The monomial
 * coefficients are copied to the device; the monomial-to-Bernstein conversion
 * (Sec. II-D, Alg. 1 line 1) runs on the device at the start of every solve. */
int pcba_create(pcba_handle** out, const pcba_poly* cost, const pcba_poly* ineq,
                int n_ineq, const pcba_poly* eq, int n_eq, const pcba_box* box,
                int precision);

/* As pcba_create, but the coefficient tensors already hold Bernstein patches
 * over 'box' (Eq. (BF)); the conversion step is skipped.  Used to start the
 * branch and bound from given patches. */
int pcba_create_bernstein(pcba_handle** out, const pcba_poly* cost, const pcba_poly* ineq,
                          int n_ineq, const pcba_poly* eq, int n_eq, const pcba_box* box,
                          int precision);

/* A family of inequality constraints that are affine in a few shared
 * polynomials:
 *
 *     g_i(x) = offset[i] + sum_{m < n_shared} weight[i * n_shared + m] s_m(x) <= 0,
 *     i = 0 .. n_constraints - 1.
 *
 * The Bernstein transform is linear (Sec. II-D, Eq. (BF): the coefficients of a
 * constant are that constant, Thm. 1's partition of unity), so on every box
 * B(g_i) = offset[i] + sum_m weight[i][m] B(s_m), coefficient by coefficient.
 * A list item then stores the n_shared patches B(s_m) instead of one patch
 * per constraint, and every constraint's bounds are computed from them when
 * its box is bounded; in exact arithmetic the coefficients, and therefore the
 * whole branch and bound, are those of the expanded constraints.  Obstacle
 * constraints of the trajectory-planning POPs (Sec. II-C, Sec. VI) have this
 * form: r^2 - ||F(q) - o_i||^2 = (r^2 - ||o_i||^2) - ||F||^2 + 2 o_i . F.
 *   n_shared       1 .. PCBA_MAX_SHARED
 *   shared         n_shared polynomials (zero-padded to one common degree)
 *   n_constraints  alpha >= 0
 *   weight         [alpha][n_shared] doubles, row-major
 *   offset         [alpha] doubles */
typedef struct {
  int n_shared;
  const pcba_poly* shared;
  int n_constraints;
  const double* weight;
  const double* offset;
} pcba_linear_family;

/* Builds a problem whose inequalities are a linear family (no equality
 * constraints): cost p, the family and the box, as pcba_create.  Each item
 * also keeps one bit per constraint: a constraint whose bound proves
 * g_i <= 0 on a box is dropped from that box and all its descendants (the
 * Bernstein range of a sub-box lies in that of the box, Thm. 1 and Sec. II-E),
 * so later bisections bound only the constraints still undecided there.
 * Batches must not mix linear and dense problems. */
int pcba_create_linear(pcba_handle** out, const pcba_poly* cost,
                       const pcba_linear_family* ineq, const pcba_box* box, int precision);

/* Per-item activity bits of the list of the last pcba_solve_steps on a
 * linear-family problem: bits[k * words + w] holds constraints 32 w .. 32 w + 31
 * of list item k (bit set: still undecided or violated on that box; clear:
 * proven g_i <= 0 there), words = ceil(n_constraints / 32).  Returns the
 * number of words per item (0 for a dense problem). */
int pcba_get_active(pcba_handle* h, unsigned* bits, long long max_words);

/* Runs Algorithm 1 to completion on one problem.
 *   opt_tol   optimality tolerance epsilon > 0 (Def. 2): stop when p_up - p_lo <= opt_tol
 *   eq_tol    equality tolerance epsilon_eq > 0 (Def. 2, Def. 3 (b))
 *   max_iters N of Alg. 1: the solve ends with PCBA_MAXITER when the sweep
 *             counter n reaches N, i.e. after (N-1) l steps at most
 *   mem_cap   bytes of list storage; M = floor(mem_cap / bytes per item)
 *             (Eq. (memory_per_item) as stored here, see pcba_item_bytes)
 * Blocks until the result is on the host.  Returns 0 or a PCBA_ERR_* code. */
int pcba_solve(pcba_handle* h, double opt_tol, double eq_tol, int max_iters,
               size_t mem_cap, pcba_result* out);

/* As pcba_solve, but stops after at most max_steps steps (status
 * PCBA_STEPLIMIT if the solve was not over); the list stays on the device and
 * can be read with pcba_get_list.  The cut-off bookkeeping of the last step
 * (Alg. 5) is complete when it returns. */
int pcba_solve_steps(pcba_handle* h, double opt_tol, double eq_tol, int max_iters,
                     size_t mem_cap, int max_steps, pcba_result* out);

/* Solves n independent problems together on the device: each keeps its own
 * list, incumbent and status, and all advance one bisection step per
 * iteration of one device loop.  All handles must share the precision.
 * mem_cap_total bytes are shared so that every problem gets the same item
 * capacity M = floor(mem_cap_total / sum of bytes per item).
 * warm_start is NULL or n * PCBA_MAX_DIM doubles (row k = point of problem k,
 * first nvars used; a NaN first entry means none); each point is rounded to
 * FP32 coordinates, its constraints are evaluated in FP32 with a rigorous
 * rounding-error bound and its cost in FP64 with one, and only if it is
 * certified feasible does it lower that problem's p_up to its certified cost
 * bound (this never removes a feasible minimiser, Thm. 3).
 * out receives n results. */
int pcba_solve_batch(pcba_handle** hs, int n, double opt_tol, double eq_tol, int max_iters,
                     size_t mem_cap_total, const double* warm_start, pcba_result* out);

/* A reusable batch: device buffers are allocated once and the device loop is
 * built once, so repeated solves do no allocation.  flags (bits):
 *   0 = device loop in a CUDA graph with a conditional WHILE node (default);
 *   1 = host loop that reads one status word per step;
 *   3 = host loop with CUDA events around every subdivision launch;
 *   4 = do not use the TMA-staged subdivision kernel (the direct-load one runs;
 *       it is also used when a constraint patch exceeds 256 coefficients);
 *   8 = vertex incumbents (linear-family batches only, else PCBA_ERR_INVALID):
 *       the corner coefficients of a patch are the polynomial's values at the
 *       box's corners (Sec. II-D), so a child box's corner at which every
 *       active constraint's corner value plus its bound E is <= 0 is a
 *       feasible point, and its corner cost coefficient plus e_p bounds p
 *       there.  The least such bound lowers p_up in the same step (before the
 *       cut-off test) and the corner becomes the returned point (FP32 and
 *       FP64; up to 4 corners per box: those of the first two axes, the
 *       other axes at their lower end).  Sound (Thm. 3 holds for any p_up
 *       attained at a feasible point); without it the lists follow Alg. 1-5
 *       exactly. */
int pcba_batch_create(pcba_batch** out, pcba_handle** hs, int n, size_t mem_cap_total,
                      int flags);
int pcba_batch_solve(pcba_batch* b, double opt_tol, double eq_tol, int max_iters,
                     const double* warm_start, pcba_result* out);
/* As pcba_batch_solve, but the monomial coefficients of every problem are
 * first copied from the given pinned or pageable host buffer (the layout of
 * pcba_batch_input_layout) inside the same stream: the end-to-end call. */
int pcba_batch_solve_from_host(pcba_batch* b, const double* host_coeffs, double opt_tol,
                               double eq_tol, int max_iters, const double* warm_start,
                               pcba_result* out);
/* Number of doubles pcba_batch_solve_from_host reads. */
long long pcba_batch_input_doubles(const pcba_batch* b);
/* Per-step records (K before the step, K_save, p_up, p_lo) of problem k of the
 * last solve; returns the number of rows written (at most max_rows). */
int pcba_batch_trace(const pcba_batch* b, int k, double* rows, int max_rows);
/* Device time in ms of the last solve (CUDA events around the whole device
 * work on the batch stream), and the kernel-level split used for the roofline:
 * ms spent in the subdivide/bound kernel and its algorithmic bytes. */
int pcba_batch_timing(const pcba_batch* b, double* total_ms, double* subdiv_ms,
                      double* subdiv_bytes, long long* subdiv_launches);
/* Autotuner (not in the paper): times one solve of this batch under every
 * feasible configuration of the subdivision kernel - direct loads, or TMA
 * staging with 8/4/2 warps per block and 2/3 pipeline stages per warp - keeps
 * the fastest and rebuilds the device loop for it.  ms_per_config[i] (if not
 * NULL, up to max_configs entries) receives each configuration's solve time,
 * *chosen the index kept.  Returns the number of configurations. */
int pcba_batch_autotune(pcba_batch* b, double opt_tol, double eq_tol, int max_iters,
                        double* ms_per_config, int max_configs, int* chosen);
/* The subdivision configuration in use: returns its index and, if not NULL,
 * whether it uses TMA staging, warps per block, stages and grid size. */
int pcba_batch_config(const pcba_batch* b, int* tma, int* warps_per_block, int* stages,
                      int* grid);
/* Algorithmic bytes (3 x K x stored bytes of the patches of every running
 * problem: one parent read, two children written) of each subdivision launch
 * of the last instrumented solve (flags 3); returns the number written. */
int pcba_batch_launch_bytes(const pcba_batch* b, double* bytes, int max_launches);
/* Counters of the last solve: iterations of the device loop (one bisection
 * step of every running problem each), kernels this library launched, and the
 * bytes the call copied host->device and device->host. */
int pcba_batch_stats(const pcba_batch* b, long long* loop_iters, long long* kernel_launches,
                     long long* h2d_bytes, long long* d2h_bytes);
/* FP32 mode: marks for a refresh from the FP64 monomials during the last
 * solve (a patch, or all shared patches of a linear-family child, whose error
 * bound changed a classification) and patches recomputed (K per linear-family
 * mark; marks of patches larger than the refresh buffers are skipped). */
int pcba_batch_refresh_stats(const pcba_batch* b, long long* marked, long long* refreshed);
/* Linear families: constraint bounds computed by the last solve - pairs of
 * (child box, active constraint), and how many of them needed the range of
 * the constraint's coefficients rather than the interval bound from the
 * shared patches' ranges - and the coefficients per shared patch (of the
 * first problem).  All 0 for dense batches. */
int pcba_batch_linear_stats(const pcba_batch* b, long long* pairs, long long* full,
                            long long* coeffs);
/* Local polish of the point each problem's last solve returned (not in the
 * paper).  From the centre of the last solve's best box (or its certified
 * warm point): a log-barrier Newton method in FP64 on
 *   min p(x) - mu sum_i log(-g_i(x))  subject to  h_j(x) = 0, x in the box,
 * starting at mu = mu0 max(1, |p(x0)|) and lowered tenfold per level down to
 * gap / max(1, alpha) (for a convex program the barrier point is within
 * alpha mu of the optimum), at most iters Newton steps per level.  After each
 * level the iterate rounded to FP32 coordinates is kept if every g_i < 0 and
 * sum_j |h_j| <= eq_tol / 2 there.  x receives np rows of PCBA_MAX_DIM
 * doubles (host memory): the last kept point (entries past l are 0), or NaN
 * where there is none (infeasible, no point, more than PCBA_MAX_DIM
 * equalities, or no level kept).  The result is only a candidate: it lowers
 * p_up only if a later solve's warm-start certification accepts it.  Runs on
 * the batch's stream and blocks until x is written.  PCBA_ERR_INVALID unless
 * mu0, gap, eq_tol > 0 and 1 <= iters <= 200. */
int pcba_batch_polish(pcba_batch* b, double mu0, double gap, double eq_tol, int iters,
                      double* x);
/* Two solves for tight equality tolerances (not in the paper): a solve with
 * (relax_opt_tol, relax_eq_tol), then pcba_batch_polish of its points
 * (mu0 = 1e-2, gap = opt_tol / 10, 30 steps per level; the points stay on
 * the device), then a solve with (opt_tol, eq_tol) whose warm starts are the
 * polished points.  Every reported bound and point comes from the second
 * solve, so the certificate is that of pcba_batch_solve with (opt_tol,
 * eq_tol): the first solve and the polish only decide how early p_up becomes
 * finite.  time_ms and pcba_batch_timing's total count from the start of the
 * first solve, and pcba_batch_stats counts the kernel launches and copies of
 * all three phases.  PCBA_ERR_INVALID unless 0 < eq_tol <= relax_eq_tol and
 * both optimality tolerances are > 0. */
int pcba_batch_solve_polished(pcba_batch* b, double opt_tol, double eq_tol, double relax_opt_tol,
                              double relax_eq_tol, int max_iters, pcba_result* out);
int pcba_batch_set_stream(pcba_batch* b, void* cuda_stream);
/* The time limit of pcba_set_time_limit for the solves of a batch: every
 * problem still running when it runs out stops with PCBA_TIMEOUT.  In
 * pcba_batch_solve_polished it applies to each of the two solves. */
int pcba_batch_set_time_limit(pcba_batch* b, double seconds);
void pcba_batch_destroy(pcba_batch* b);

/* Copies the list of the last pcba_solve / pcba_solve_steps to the host in the
 * layout of the oracle: cost[K][cp], ineq[K][alpha][cg], eq[K][beta][ch] as
 * doubles (FP32 patches are widened, and their stored per-patch error bounds
 * go to err[K][1 + alpha + beta] if err is not NULL), index[K][nvars] dyadic
 * box indices and level[nvars].  *K_out = list length.  Any output pointer may
 * be NULL to skip it; call once with all NULL to learn K. */
int pcba_get_list(pcba_handle* h, long long* K_out, double* cost, double* ineq, double* eq,
                  float* err, unsigned* index, int* level);

/* Root Bernstein patches (Alg. 1 line 1) of the problem as computed on the
 * device in FP64: cost[cp], ineq[alpha][cg], eq[beta][ch]. */
int pcba_root_patches(pcba_handle* h, double* cost, double* ineq, double* eq);

/* Stored bytes of one list item of this problem (the per-item storage behind
 * M = floor(mem_cap / bytes)). */
long long pcba_item_bytes(const pcba_handle* h);

int pcba_set_stream(pcba_handle* h, void* cuda_stream);
int pcba_set_warm_start(pcba_handle* h, const double* x);  /* NULL clears */

/* Time limit of the solves of this handle (pcba_solve, pcba_solve_steps), in
 * seconds of device time from the start of the solve's device work; 0 (the
 * default) means none.  The robot of Sec. VI gives PCBA 0.4 s per problem.
 * The limit is checked on the device between two bisection steps: a problem
 * still running then stops with status PCBA_TIMEOUT and returns the interval
 * [lower, upper] certified by the last finished step (and its point, if a
 * feasible item was found), like PCBA_MAXITER.  A solve can therefore run one
 * step past the limit.  PCBA_ERR_INVALID if seconds is negative or not finite. */
int pcba_set_time_limit(pcba_handle* h, double seconds);
void pcba_destroy(pcba_handle* h);

/* Monomial-to-Bernstein conversion (the step pcba_root_patches runs) that
 * allocates nothing.  There is no counterpart in the paper: it exists for
 * callers that cannot call cudaMalloc - code running inside another
 * framework's memory pool or a real-time loop where allocation is forbidden
 * after start-up, or a caller that hands every buffer in from its own arena.
 *   d_mono     device pointer: n_patches dense monomial tensors of multi-degree
 *              degree[0..nvars), each prod(degree[r]+1) doubles, row-major
 *   degree, lo, hi   host arrays of nvars entries: the multi-degree and the box
 *   d_out      device pointer, same layout: the Bernstein patches over the box
 *   stream     cudaStream_t to launch on (NULL: the default stream)
 * Returns once the work is queued on the stream; the caller synchronises.
 * Limits: nvars <= 8, every degree <= 16 and at most 8192 coefficients per
 * patch (the fixed scratch holds one 17x17 matrix per axis); anything larger
 * returns PCBA_ERR_INVALID.
 * The per-axis matrices live in one fixed 18.5 KB device array in the library,
 * kept by every GPU that loads the library until the process exits.  The first
 * call in each CUDA context of a device (the first call on the device, and the
 * first after cudaDeviceReset or in another context of it) looks up that
 * array's device address, so make that call before capturing a stream into a
 * CUDA graph.  All calls share the array: two calls that overlap on the GPU
 * (for instance on two streams) race on it. */
int pcba_bernstein_convert_noalloc(const double* d_mono, int n_patches, int nvars,
                                   const int* degree, const double* lo, const double* hi,
                                   double* d_out, void* stream);

const char* pcba_status_string(int status);
const char* pcba_last_error(void);
int pcba_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PCBA_H_ */
