/* Learned warm start for PCBA (not part of the paper).
 *
 * The paper's Alg. 1 starts every solve with no incumbent: the upper bound p_up
 * of Def. 4 is +inf until a box is certified feasible.  Any point that is
 * certified feasible in FP64 gives a valid p_up before the first step, so the
 * cut-off test (Alg. 4) can discard suboptimal boxes (Def. 5) earlier without
 * ever discarding a minimiser (Thm. 3).  This header adds
 *
 *   1. a set-encoder network (pcba_mlp_*) that maps a problem - a set of points
 *      (obstacles) and a global feature vector - to a guess of the minimiser in
 *      the box's normalised coordinates [-1, 1]^2, trained on the device with
 *      hand-written kernels (BF16 tensor-core GEMMs, FP32 accumulation and FP32
 *      master weights, Adam); and
 *   2. pcba_batch_solve_guided: a batch solve whose incumbent is seeded by the
 *      best certified-feasible point among a stencil of candidates around each
 *      problem's guess.  The guess never changes the solver's result other than
 *      through this incumbent: the certified bounds hold whatever it is.
 *
 * Network (weights row-major [in][out], parameter vector W1 b1 ... W6 b6):
 *   h1_p = relu(x_p W1 + b1)    point_dim -> H
 *   h2_p = relu(h1_p W2 + b2)   H -> H
 *   h3_p = relu(h2_p W3 + b3)   H -> H
 *   z    = max over the set of h3_p (elementwise)
 *   h4   = relu([z, u] W4 + b4) H + global_dim -> H
 *   h5   = relu(h4 W5 + b5)     H -> H
 *   y    = tanh(h5 W6 + b6)     H -> 2
 *   loss = (1/B) sum_b ||y_b - t_b||^2
 * Precision 16: dense-layer operands rounded to BF16, FP32 accumulation.
 * Precision 32: every product in FP32 (a debugging reference).
 *
 * Errors: functions return 0 or a negative PCBA_ERR_* code (pcba.h) with the
 * message in pcba_last_error().  Device pointers must be valid for the given
 * sizes on the given stream (NULL: the default stream).
 */
#ifndef PCBA_WARMSTART_H_
#define PCBA_WARMSTART_H_

#include "pcba.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcba_mlp pcba_mlp;

/* Allocates the network on the current device with seeded He-normal weights
 * (std sqrt(2 / fan_in)) and zero biases.  precision is 16 or 32; hidden in
 * [1, 4096]; point_dim >= 1; global_dim >= 0.  The caller owns *out and frees
 * it with pcba_mlp_destroy. */
int pcba_mlp_create(pcba_mlp** out, int point_dim, int global_dim, int hidden, int precision,
                    unsigned long long seed);
void pcba_mlp_destroy(pcba_mlp* m);
long long pcba_mlp_num_params(const pcba_mlp* m);
/* Kernels this network has launched since it was created. */
long long pcba_mlp_kernel_launches(const pcba_mlp* m);
/* Host copies of the FP32 parameter vector (n must equal pcba_mlp_num_params).
 * set_params also resets the Adam moments and step count. */
int pcba_mlp_set_params(pcba_mlp* m, const float* host_params, long long n);
int pcba_mlp_get_params(const pcba_mlp* m, float* host_params, long long n);

/* Inputs of a batch of n_sets problems (all device pointers):
 *   d_points   [n_points][point_dim] float, the sets one after another
 *   d_offsets  [n_sets + 1] int, set b = points d_offsets[b] .. d_offsets[b+1]-1;
 *              d_offsets[0] = 0, d_offsets[n_sets] = n_points, every set
 *              non-empty (the library does not read them on the host)
 *   d_global   [n_sets][global_dim] float
 *   d_target   [n_sets][2] float
 * Forward: d_out [n_sets][2] receives y.  Queued on the stream. */
int pcba_mlp_forward(pcba_mlp* m, const float* d_points, const int* d_offsets, int n_sets,
                     int n_points, const float* d_global, float* d_out, void* stream);
/* Loss and gradient at the current parameters; host_grad (may be NULL)
 * receives pcba_mlp_num_params floats.  Synchronises the stream. */
int pcba_mlp_gradient(pcba_mlp* m, const float* d_points, const int* d_offsets, int n_sets,
                      int n_points, const float* d_global, const float* d_target,
                      float* host_grad, float* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * batch.  If loss is not NULL the stream is synchronised and *loss receives
 * the batch loss before the step. */
int pcba_mlp_train_step(pcba_mlp* m, const float* d_points, const int* d_offsets, int n_sets,
                        int n_points, const float* d_global, const float* d_target, float lr,
                        float* loss, void* stream);

/* Batch solve (as pcba_batch_solve) with the incumbent seeded from guesses.
 *   d_guess     device [np][guess_dim] float: problem k's guess in normalised
 *               coordinates u in [-1, 1] (x_r = lo_r + (u_r + 1)(hi_r - lo_r)/2)
 *               of its first guess_dim axes; other axes use the box centre
 *   stencil     host [n_stencil][guess_dim] doubles: candidate c of problem k is
 *               the guess plus stencil row c, clamped to [-1, 1]
 *   n_stencil   1 .. 1024 (a row of zeros makes the guess itself a candidate)
 * Every candidate is rounded to FP32 coordinates and certified as for
 * pcba_solve_batch's warm start (constraints in FP32, cost in FP64, both with
 * rigorous rounding-error bounds); the lowest certified cost bound among the
 * feasible ones (ties: the lower stencil row) becomes the problem's initial
 * p_up.  The
 * costs of all candidates are computed and sorted first and the constraints
 * evaluated in that order, so the work stops at the cheapest feasible one.
 * out receives np results; from_warm_start is set where the returned point is
 * a candidate (no box of the solve beat it). */
int pcba_batch_solve_guided(pcba_batch* b, double opt_tol, double eq_tol, int max_iters,
                            const float* d_guess, int guess_dim, const double* stencil,
                            int n_stencil, pcba_result* out);

/* Refinement of guided solves: after the first round of candidates, up to
 * four more rounds, each around each problem's current seed (its normalised
 * coordinates; the guess where no candidate was certified yet): candidate
 * c = centre + stencil row c, clamped, certified and picked the same way.
 * Include a row of zeros so that the seed stays a candidate (it then never
 * gets worse).  round: 0..3, at most one past the last round set; n_stencil =
 * 0 removes this round and the later ones; otherwise 1..1024 rows of
 * guess_dim values (the guess_dim of the guided solves, the same for every
 * round).  The library keeps a copy. */
int pcba_batch_set_refine_stencil(pcba_batch* b, int round, const double* stencil,
                                  int n_stencil, int guess_dim);

/* Queues the copy of every problem's monomial coefficients (the layout of
 * pcba_batch_solve_from_host, pcba_batch_input_doubles of them) from host
 * memory to the batch's device copy on the batch's stream, so that feature
 * kernels (pcba_batch_cost_grid) and a following pcba_batch_solve_guided see
 * new inputs; the bytes are counted in the next solve's host-to-device total.
 * Pageable host memory makes the copy synchronous. */
int pcba_batch_upload(pcba_batch* b, const double* host_coeffs);

/* The same for the constraint rows of a batch of linear-family problems
 * (pcba_create_linear): pcba_batch_rows_doubles(b) doubles, per problem in
 * batch order and per constraint the row (offset, weight_0 .. weight_K-1)
 * padded with zeros to PCBA_LIN_STRIDE (8) doubles.  The library keeps the
 * FP64 rows and their FP32 roundings (made on the device); queued on the
 * batch's stream, counted in the next solve's host-to-device bytes.
 * PCBA_ERR_INVALID for a dense batch. */
int pcba_batch_upload_rows(pcba_batch* b, const double* host_rows);
long long pcba_batch_rows_doubles(const pcba_batch* b);

/* The same rows without the padding: per constraint (offset, weight_0 ..
 * weight_K-1), 1 + K doubles, for a batch whose problems all have K shared
 * polynomials (PCBA_ERR_INVALID otherwise, and for a dense batch);
 * pcba_batch_rows_packed_doubles(b) doubles (0 when the K differ).  The
 * library pads them on the device. */
int pcba_batch_upload_rows_packed(pcba_batch* b, const double* host_rows);
long long pcba_batch_rows_packed_doubles(const pcba_batch* b);

/* Page-locked host memory for the inputs of pcba_batch_upload and the row
 * uploads (cudaHostAlloc: copied by DMA at the link's rate,
 * and the uploads stay asynchronous).  bytes > 0; returns NULL on failure
 * (the reason in pcba_last_error).  The caller owns the memory and releases
 * it with pcba_host_free (NULL is accepted) after the last queued copy from
 * it has completed. */
void* pcba_host_alloc(size_t bytes);
int pcba_host_free(void* p);

/* The incumbent seed of problem k in the last solve of the batch: returns 1
 * if a candidate (or the warm start point) was certified feasible, writing it
 * (nvars coordinates) to x and its certified cost bound - the initial p_up -
 * to *cost (either may be NULL); returns 0 if none was. */
int pcba_batch_warm_point(const pcba_batch* b, int k, double* x, double* cost);

/* Features for the network (queued on the batch's stream): the cost p of
 * every problem k on a G x G grid of its box over the first two axes (G nodes
 * when nvars = 1; other axes at the box centre), node (i, j) at
 * x_0 = lo_0 + i (hi_0 - lo_0) / (G - 1) and x_1 = lo_1 + j (hi_1 - lo_1) / (G - 1),
 * evaluated in FP64 from the monomial coefficients and written as
 * log(p - min over the grid + 1e-3) to d_out[k * ld + col0 + i * G + j]
 * (device floats).  2 <= G <= 32, ld >= col0 + G * G. */
int pcba_batch_cost_grid(pcba_batch* b, int G, float* d_out, int ld, int col0);

/* The FP32 point check of the certification above, on its own: the value of
 * one polynomial at n_points points with a rigorous rounding-error bound,
 * |d_val[i] - p(x_i)| <= d_err[i], where p has the FP64 coefficients whose
 * round-to-nearest FP32 copies are d_coeff (device, dense monomial tensor of
 * multi-degree degree[0..nvars), row-major) and x_i is row i of d_points
 * (device, [n_points][nvars] floats).  The bound is the nested-Horner bound of
 * Higham (Accuracy and Stability of Numerical Algorithms, Sec. 5.1) with a
 * factor-2 margin plus the subnormal range.  unrolled = 0: the generic nested
 * Horner; 1: the fully unrolled form the certification uses for two variables
 * of equal degree 2, 3, 4, 6 or 8 (the same operations in the same order, so
 * the same bits), the generic one for other shapes.  Queued on the stream;
 * PCBA_ERR_INVALID for shapes beyond the limits of pcba.h. */
int pcba_eval_points_f32(const float* d_coeff, int nvars, const int* degree,
                         const float* d_points, int n_points, int unrolled, float* d_val,
                         float* d_err, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCBA_WARMSTART_H_ */
