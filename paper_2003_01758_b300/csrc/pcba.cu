// libpcba: host engine and C ABI (see include/pcba.h).
//
// A solve of n problems runs as:
//   prologue  k1_matrices, k1_convert (Alg. 1 line 1), the warm start
//             (k_mono32, k_candidates, k_cand_* or k_eval), k_init (Alg. 1
//             lines 2-3, first memory test)
//   loop      the subdivision kernel, then k_refresh (FP32, forked stream)
//             beside k_pup, k3_classify and k4_index, then k_move_control:
//             one bisection step of every running problem per iteration
//             (Alg. 1 lines 4-11); by default the loop is a CUDA graph with a
//             conditional WHILE node whose condition the loop control sets on
//             the device, so the host never waits inside the loop
//   epilogue  k_eval (FP64 check of the returned point), copies to the host.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pcba.h"
#include "pcba_host.h"

// Blocks per SM of the per-step kernels over child tiles (0: as many as fit)
// and of the compaction.
#ifndef PCBA_K3_BLOCKS_PER_SM
#define PCBA_K3_BLOCKS_PER_SM 0
#endif
#ifndef PCBA_KR_BLOCKS_PER_SM
#define PCBA_KR_BLOCKS_PER_SM 8
#endif
#ifndef PCBA_K4_BLOCKS_PER_SM
#define PCBA_K4_BLOCKS_PER_SM 1
#endif
// 1: the kernels after the subdivision are launched as dependent steps
#ifndef PCBA_PDL_STEPS
#define PCBA_PDL_STEPS 1
#endif
#include "pcba_kernels.cuh"
#include "pcba_warmstart.h"

static_assert(PCBA_MAX_DIM == PCBA_MAXD, "dimension limits differ");

namespace {

// largest shared-memory copy of a problem's constraint coefficients made by
// the candidate certification (k_cand_first); larger problems read them from
// global memory
constexpr size_t kCandStageMax = 200 * 1024;

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define PCBA_CK(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(PCBA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Test hook: PCBA_TEST_FAIL_ALLOC=1 makes every device allocation fail, so the
// out-of-memory path can be exercised without exhausting a GPU.
cudaError_t dev_alloc(void** p, size_t bytes) {
  const char* f = std::getenv("PCBA_TEST_FAIL_ALLOC");
  if (f && f[0] == '1') {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (bytes == 0) bytes = 256;
  return cudaMalloc(p, bytes);
}

long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

// Row length of a constraint family in the coefficient-major layout: a
// multiple of 32 patches (128-byte rows in FP32) for large families, of 4
// (16-byte rows) for small ones so that a single constraint is not padded 32x.
long long family_pad(long long n) { return n >= 32 ? round_up(n, 32) : round_up(n, 4); }

struct HostProblem {
  int l = 0, precision = 64, form = 0;
  int P[PCBA_MAXD] = {0}, G[PCBA_MAXD] = {0}, H[PCBA_MAXD] = {0};
  int alpha = 0, beta = 0;   // stored inequality / equality patches
  long long cp = 1, cg = 0, ch = 0;
  double lo[PCBA_MAXD] = {0}, hi[PCBA_MAXD] = {0};
  std::vector<double> mono;  // cost | ineq (alpha * cg) | eq (beta * ch)
  // linear family (pcba_create_linear): the stored inequality patches are the
  // alpha = n_shared shared polynomials; nlin constraints g_i = c_i + w_i . s
  int lin = 0, nlin = 0;
  std::vector<double> lin_c, lin_w;  // [nlin], [nlin][alpha]
};

// Item layout of one problem (see pcba_device.cuh): offsets, stride and the
// algorithmic bytes of one item.  Linear-family items hold two copies of the
// shared patches and their error bounds (read from one, written to the other,
// alternating by step) and one activity bit per constraint.
void layout_item(const HostProblem& P, int prec, ProbDesc& d) {
  const int w = prec == PCBA_FP32 ? 4 : 8;
  d.apad = (int)family_pad(P.alpha);
  d.bpad = (int)family_pad(P.beta);
  d.lin = P.lin;
  d.nlin = P.nlin;
  d.mwords = P.lin ? (P.nlin + 31) / 32 : 0;
  d.lin_chunks = P.lin ? std::max(1, (d.mwords + PCBA_LIN_WORDS - 1) / PCBA_LIN_WORDS) : 0;
  const int copies = P.lin ? 2 : 1;
  long long off = 64;
  d.off_cost = off;
  off = round_up(off + P.cp * w, 128);
  d.off_eg = off;
  // linear families: per copy the metadata of the shared patches (FP32: error
  // bounds, the FP64 offsets the patches are stored relative to, extremes of
  // the stored values; FP64: the extremes)
  d.copy_e = P.lin ? (prec == PCBA_FP32 ? 20LL : 16LL) * d.apad : 0;
  d.off_og = d.off_oh = 0;
  if (P.lin) off = round_up(off + copies * d.copy_e, 128);
  else if (prec == PCBA_FP32) {
    // dense FP32 families: error bounds, then the per-patch offsets, each
    // array at least 32 floats (the TMA kernel loads 32 of each per group)
    const long long ea = 4LL * std::max(d.apad, 32);
    d.off_og = off + ea;
    off = round_up(off + 2 * ea, 128);
  }
  d.off_eh = off;
  if (prec == PCBA_FP32) {
    const long long eb = 4LL * std::max(d.bpad, 32);
    d.off_oh = off + eb;
    off = round_up(off + 2 * eb, 128);
  }
  d.off_g = off;
  d.copy_g = P.lin ? round_up(P.cg * d.apad * w, 128) : 0;
  off = P.lin ? off + 2 * d.copy_g : round_up(off + P.cg * d.apad * w, 128);
  d.off_h = off;
  off = off + P.ch * d.bpad * w;
  // linear families: two 64-bit summaries of the non-empty activity chunks
  // (read from one, written to the other, alternating by step), then the bits
  d.off_sum = off;
  if (P.lin) off += 16;
  d.off_mask = off;
  off += 4LL * d.mwords;
  d.item_bytes = round_up(off, 256);
  d.payload_bytes = 4LL * P.l + (P.cp + P.alpha * P.cg + P.beta * P.ch) * w +
                    (prec == PCBA_FP32 ? 12LL + 4LL * (P.alpha + P.beta) : 0) +
                    (prec == PCBA_FP32 && !P.lin ? 4LL * (P.alpha + P.beta) : 0) +
                    4LL * d.mwords;
}

struct Grids {
  K2Plan k2;          // subdivision kernels (pcba_k2.cu): variant and configurations
  int cfg = 0;        // configuration in use (index into k2.cfgs)
  bool tma = false;   // it stages parents with TMA (tensor maps needed)
  int sms = 148;
  int k1_grid = 1, k1_wpb = 1, k1_cmax = 1;
  size_t k1_smem = 0;
  int k3_grid = 1, k4_grid = 1;
  // FP32 refresh kernel
  int kr_grid = 1, kr_cmax = 1, kr_lmax = 1;
  size_t kr_smem = 0;
};

}  // namespace

struct pcba_batch {
  int np = 0;
  int lin = 0;                 // linear-family problems (pcba_create_linear)
  long long nslots_total = 0;  // entries of each per-slot scratch array
  long long lin_rows = 0;      // constraints of all linear-family problems
  bool want_tma = true;
  double time_limit_s = 0.0;   // pcba_batch_set_time_limit (0: none)
  int precision = 64;
  int flags = 0;
  std::vector<ProbDesc> desc;
  std::vector<const HostProblem*> probs;
  long long mono_doubles = 0;
  long long M = 0;
  long long sum_item_bytes = 0;
  int max_l = 1;
  // device
  ProbDesc* d_desc = nullptr;
  ProbState* d_state = nullptr;
  Plan* d_plan = nullptr;
  SolveParams* d_params = nullptr;
  unsigned* d_pre = nullptr;  // 5 arrays of np+1
  char* d_arena = nullptr;
  ChildRec* d_rec = nullptr;
  unsigned* d_slots = nullptr;  // flagrank | hole | filler | map | fstack
  unsigned* d_tilecnt = nullptr;
  double* d_mono = nullptr;
  float* d_mono32 = nullptr;
  double* d_trace = nullptr;
  double* d_warm = nullptr;
  double* d_mat = nullptr;
  void* d_tmaps = nullptr;
  uint4* d_marks = nullptr;
  double* d_raw = nullptr;
  EvalOut* d_eval = nullptr;
  double* d_cand = nullptr;     // guided solves: [np][cand_cap][PCBA_MAXD]
  float* d_ckey = nullptr;      // warm starts: [np][ckey_cap] FP32 cost bounds of candidates
  int* d_corder = nullptr;      // warm starts: [np][ckey_cap] candidates in rank order
  int* d_cres = nullptr;        // warm starts: [np] lowest certified-feasible rank
  long long ckey_cap = 0;
  long long cand_floats = 0;    // largest constraint coefficient count (alpha cg + beta ch)
  double* d_stencil = nullptr;  // guided solves: [stencil_cap] doubles
  double* d_polish = nullptr;   // pcba_batch_polish output: [np][PCBA_MAXD]
  float* d_lin32 = nullptr;     // linear families: [lin_rows][PCBA_LIN32_STRIDE] FP32 pairs of the rows
  uint4* d_lin_queue = nullptr; // linear families: heavy (item, window, problem, k) units
  double* d_lin64 = nullptr;    // the same in FP64
  // pcba_batch_solve_polished: the warm points are already in d_warm (written
  // by the polish kernel), and the counts of the phases before the last solve
  bool warm_on_device = false;
  long long prior_launches = 0, prior_h2d = 0, prior_d2h = 0;
  cudaEvent_t ev_pipe = nullptr;
  long long cand_cap = 0, stencil_cap = 0;
  // refinement rounds of guided solves (host copies of their stencils)
  std::vector<std::vector<double>> refine;
  std::vector<int> refine_rows;
  int refine_dim = 0;
  long long refine_total() const {
    long long t = 0;
    for (int r : refine_rows) t += r;
    return t;
  }
  int refine_max() const {
    int m = 0;
    for (int r : refine_rows) m = std::max(m, r);
    return m;
  }
  long long trace_rows_total = 0;
  // host mirrors (pinned)
  ProbState* h_state = nullptr;
  EvalOut* h_eval = nullptr;
  Plan* h_plan = nullptr;
  SolveParams* h_params = nullptr;
  int* h_running = nullptr;
  // streams and graph
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStream_t side = nullptr;                        // k_refresh beside k_pup..k4_index
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool refresh_pending = false;  // a refresh on the side stream not yet joined
  cudaEvent_t ev_k1f = nullptr, ev_k1j = nullptr;  // K1 on the side stream beside the warm start
  std::vector<cudaEvent_t> kev;
  Engine E{};
  Grids g;
  // timing of the last solve
  double total_ms = 0, subdiv_ms = 0, subdiv_bytes = 0;
  long long subdiv_launches = 0;
  long long h2d_bytes = 0, d2h_bytes = 0;
  long long pending_h2d = 0;      // bytes queued by pcba_batch_upload since the last solve
  long long extra_launches = 0;   // prologue kernels of warm starts in the last solve
  long long extra_launches_pending = 0;  // kernels queued by uploads since the last solve
  std::vector<double> launch_bytes;
};

struct pcba_handle {
  HostProblem prob;
  cudaStream_t stream = nullptr;
  bool has_warm = false;
  double warm[PCBA_MAXD];
  pcba_batch* own = nullptr;
  size_t own_cap = 0;
  double time_limit_s = 0.0;   // pcba_set_time_limit (0: none)
};

namespace {

int check_poly(const pcba_poly* q, int l, const char* what) {
  if (!q || !q->degree || !q->coeff) return fail(PCBA_ERR_INVALID, std::string(what) + ": null");
  if (q->nvars != l) return fail(PCBA_ERR_INVALID, std::string(what) + ": nvars differs from box");
  long long c = 1;
  for (int r = 0; r < l; ++r) {
    if (q->degree[r] < 0 || q->degree[r] > PCBA_MAX_DEGREE)
      return fail(PCBA_ERR_INVALID, std::string(what) + ": degree out of range");
    c *= q->degree[r] + 1;
  }
  if (c > PCBA_MAX_PATCH) return fail(PCBA_ERR_INVALID, std::string(what) + ": patch too large");
  return 0;
}

// Copies a polynomial of multi-degree deg into a tensor of multi-degree big
// (zero padding = degree elevation of the tensor, the polynomial is unchanged).
void embed(const pcba_poly* q, int l, const int* big, double* out) {
  long long total = 1;
  for (int r = 0; r < l; ++r) total *= big[r] + 1;
  std::fill(out, out + total, 0.0);
  long long src_total = 1;
  for (int r = 0; r < l; ++r) src_total *= q->degree[r] + 1;
  for (long long s = 0; s < src_total; ++s) {
    long long rem = s, dst = 0, mul = 1;
    int digit[PCBA_MAXD];
    for (int r = l - 1; r >= 0; --r) {
      digit[r] = (int)(rem % (q->degree[r] + 1));
      rem /= q->degree[r] + 1;
    }
    for (int r = l - 1; r >= 0; --r) {
      dst += digit[r] * mul;
      mul *= big[r] + 1;
    }
    out[dst] = q->coeff[s];
  }
}

int create_impl(pcba_handle** out, const pcba_poly* cost, const pcba_poly* ineq, int n_ineq,
                const pcba_poly* eq, int n_eq, const pcba_box* box, int precision, int form) {
  if (!out) return fail(PCBA_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!box || !box->lo || !box->hi) return fail(PCBA_ERR_INVALID, "box is null");
  const int l = box->nvars;
  if (l < 1 || l > PCBA_MAX_DIM) return fail(PCBA_ERR_INVALID, "nvars out of range");
  if (precision != PCBA_FP64 && precision != PCBA_FP32)
    return fail(PCBA_ERR_INVALID, "precision must be PCBA_FP64 or PCBA_FP32");
  if (n_ineq < 0 || n_eq < 0 || (n_ineq > 0 && !ineq) || (n_eq > 0 && !eq))
    return fail(PCBA_ERR_INVALID, "constraint arrays");
  for (int r = 0; r < l; ++r)
    if (!(box->lo[r] < box->hi[r]) || !std::isfinite(box->lo[r]) || !std::isfinite(box->hi[r]))
      return fail(PCBA_ERR_INVALID, "box needs finite lo < hi");
  int rc = check_poly(cost, l, "cost");
  if (rc) return rc;
  for (int i = 0; i < n_ineq; ++i)
    if ((rc = check_poly(ineq + i, l, "ineq"))) return rc;
  for (int j = 0; j < n_eq; ++j)
    if ((rc = check_poly(eq + j, l, "eq"))) return rc;
  pcba_handle* h = new pcba_handle();
  HostProblem& P = h->prob;
  P.l = l;
  P.precision = precision;
  P.form = form;
  P.alpha = n_ineq;
  P.beta = n_eq;
  for (int r = 0; r < l; ++r) {
    P.lo[r] = box->lo[r];
    P.hi[r] = box->hi[r];
    P.P[r] = cost->degree[r];
    for (int i = 0; i < n_ineq; ++i) P.G[r] = std::max(P.G[r], ineq[i].degree[r]);
    for (int j = 0; j < n_eq; ++j) P.H[r] = std::max(P.H[r], eq[j].degree[r]);
  }
  P.cp = 1;
  P.cg = n_ineq ? 1 : 0;
  P.ch = n_eq ? 1 : 0;
  for (int r = 0; r < l; ++r) {
    P.cp *= P.P[r] + 1;
    if (n_ineq) P.cg *= P.G[r] + 1;
    if (n_eq) P.ch *= P.H[r] + 1;
  }
  if (P.cg > PCBA_MAX_PATCH || P.ch > PCBA_MAX_PATCH) {
    delete h;
    return fail(PCBA_ERR_INVALID, "padded patch too large");
  }
  if (form == 1) {
    // Bernstein patches cannot be zero-padded: every family must share its degree
    for (int i = 0; i < n_ineq; ++i)
      for (int r = 0; r < l; ++r)
        if (ineq[i].degree[r] != P.G[r]) { delete h; return fail(PCBA_ERR_INVALID, "Bernstein ineq degrees differ"); }
    for (int j = 0; j < n_eq; ++j)
      for (int r = 0; r < l; ++r)
        if (eq[j].degree[r] != P.H[r]) { delete h; return fail(PCBA_ERR_INVALID, "Bernstein eq degrees differ"); }
  }
  P.mono.assign((size_t)(P.cp + n_ineq * P.cg + n_eq * P.ch), 0.0);
  embed(cost, l, P.P, P.mono.data());
  for (int i = 0; i < n_ineq; ++i) embed(ineq + i, l, P.G, P.mono.data() + P.cp + i * P.cg);
  for (int j = 0; j < n_eq; ++j)
    embed(eq + j, l, P.H, P.mono.data() + P.cp + n_ineq * P.cg + j * P.ch);
  for (double v : P.mono)
    if (!std::isfinite(v)) { delete h; return fail(PCBA_ERR_INVALID, "non-finite coefficient"); }
  *out = h;
  return 0;
}

void free_batch(pcba_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  for (cudaEvent_t e : b->kev) cudaEventDestroy(e);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->ev_k1f) cudaEventDestroy(b->ev_k1f);
  if (b->ev_k1j) cudaEventDestroy(b->ev_k1j);
  if (b->ev_pipe) cudaEventDestroy(b->ev_pipe);
  if (b->side) cudaStreamDestroy(b->side);
  void* dev[] = {b->d_desc, b->d_state, b->d_plan, b->d_params, b->d_pre, b->d_arena, b->d_rec,
                 b->d_slots, b->d_tilecnt, b->d_mono, b->d_trace, b->d_warm, b->d_mat,
                 b->d_raw, b->d_eval, b->d_tmaps, b->d_marks, b->d_cand, b->d_stencil,
                 b->d_mono32, b->d_ckey, b->d_corder, b->d_cres, b->d_polish, b->d_lin32,
                 b->d_lin64, b->d_lin_queue};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {b->h_state, b->h_eval, b->h_plan, b->h_params, b->h_running};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  delete b;
}

template <typename T>
void launch_k2(const pcba_batch* b, cudaStream_t s) {
  if (sizeof(T) == 4) pcba_k2_launch_f32(b->g.k2, b->g.cfg, b->E, s);
  else pcba_k2_launch_f64(b->g.k2, b->g.cfg, b->E, s);
}

// The main stream waits for the last refresh launched on the side stream:
// before the next subdivision (which reads the refreshed patches), and
// before anything reads results.
int join_refresh(pcba_batch* b, cudaStream_t s) {
  if (!b->refresh_pending) return 0;
  b->refresh_pending = false;
  PCBA_CK(cudaStreamWaitEvent(s, b->ev_join, 0));
  return 0;
}

// The kernels of one device-loop iteration after the subdivision: the FP32
// refresh of the patches it marked runs on a side stream beside k_pup,
// k3_classify, k4_index and k_move_control (which read only the child
// records and the slot map; the refresh finds its items through the map
// before the compaction, whose moves change no item) and joins before the
// next subdivision.
template <typename T>
int launch_after_k2(pcba_batch* b, cudaStream_t s, int use_graph) {
  const Grids& g = b->g;
  const bool fp32 = sizeof(T) == 4;
  if (fp32) {
    PCBA_CK(cudaEventRecord(b->ev_fork, s));
    PCBA_CK(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    k_refresh<<<g.kr_grid, PCBA_KRB, g.kr_smem, b->side>>>(b->E, g.kr_cmax, g.kr_lmax);
    PCBA_CK(cudaEventRecord(b->ev_join, b->side));
    b->refresh_pending = true;
  }
  PCBA_CK(pcba_launch_step(PCBA_PDL_STEPS, k_pup, g.k3_grid, PCBA_TPB, 0, s, b->E));
  PCBA_CK(pcba_launch_step(PCBA_PDL_STEPS, k3_classify, g.k3_grid, PCBA_TPB, 0, s, b->E));
  PCBA_CK(pcba_launch_step(PCBA_PDL_STEPS, k4_index, g.k3_grid, PCBA_TPB, 0, s, b->E));
  PCBA_CK(pcba_launch_step(PCBA_PDL_STEPS, k_move_control, g.k4_grid, PCBA_TPB, 0, s, b->E, b->cond, use_graph));
  PCBA_CK(cudaGetLastError());
  return 0;
}

template <typename T>
int launch_loop_body(pcba_batch* b, cudaStream_t s, int use_graph) {
  if (int rc = join_refresh(b, s)) return rc;
  launch_k2<T>(b, s);
  return launch_after_k2<T>(b, s, use_graph);
}

template <typename T>
int setup_kernels(pcba_batch* b) {
  Grids& g = b->g;
  int dev = 0;
  PCBA_CK(cudaGetDevice(&dev));
  PCBA_CK(cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, dev));
  int smem_optin = 0;
  PCBA_CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  long long cmax = 1, cpmax = 1;
  for (const ProbDesc& d : b->desc) {
    cmax = std::max<long long>(cmax, std::max<long long>(d.cp, std::max<long long>(d.cg, d.ch)));
    cpmax = std::max<long long>(cpmax, d.cp);
  }
  g.k1_cmax = (int)cmax;
  // K1: warps per block limited by shared memory
  const size_t per_warp = (size_t)(4 * cmax + 578) * sizeof(double);
  g.k1_wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(smem_optin - 1024) / per_warp));
  g.k1_smem = per_warp * g.k1_wpb;
  if (g.k1_smem > (size_t)smem_optin) return fail(PCBA_ERR_INVALID, "patch too large for shared memory");
  PCBA_CK(cudaFuncSetAttribute(k1_convert<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)g.k1_smem));
  int occ = 0;
  PCBA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k1_convert<T>, 32 * g.k1_wpb,
                                                        g.k1_smem));
  g.k1_grid = std::max(1, occ) * g.sms;
  // K2: the subdivision kernel variant and its configurations
  {
    const int rc = sizeof(T) == 4 ? pcba_k2_prepare_f32(g.k2, b->desc, b->lin != 0, g.sms, smem_optin)
                                  : pcba_k2_prepare_f64(g.k2, b->desc, b->lin != 0, g.sms, smem_optin);
    if (rc) return rc;
  }
  // FP32 refresh: a block per marked item, 4 patch buffers of the largest
  // patch (all shared patches of a linear-family item) and the per-axis
  // matrices in its shared memory
  if (sizeof(T) == 4) {
    g.kr_lmax = b->max_l;
    long long krc = cmax;
    for (const ProbDesc& d : b->desc)
      if (d.lin) krc = std::max<long long>(krc, (long long)d.alpha * d.cg);
    g.kr_cmax = (int)krc;
    auto need = [&](long long c) {
      return refresh_smem_doubles((int)c, g.kr_lmax) * sizeof(double);
    };
    while (g.kr_cmax > 1 && need(g.kr_cmax) > (size_t)smem_optin - 4096) g.kr_cmax /= 2;
    g.kr_smem = need(g.kr_cmax);
    PCBA_CK(cudaFuncSetAttribute(k_refresh, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)g.kr_smem));
    PCBA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_refresh, PCBA_KRB, g.kr_smem));
    // marks are tens to thousands per step: up to PCBA_KR_BLOCKS_PER_SM
    // resident blocks per SM
    g.kr_grid = std::max(1, std::min(occ, PCBA_KR_BLOCKS_PER_SM)) * g.sms;
    double binom[17 * 17], binom_inv[17 * 17];
    for (int n = 0; n < 17; ++n)
      for (int k = 0; k < 17; ++k) {
        double c = 0.0;
        if (k <= n) {
          c = 1.0;
          for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
        }
        binom[n * 17 + k] = c;
        binom_inv[n * 17 + k] = c > 0.0 ? 1.0 / c : 0.0;
      }
    PCBA_CK(cudaMemcpyToSymbol(c_binom, binom, sizeof(binom)));
    PCBA_CK(cudaMemcpyToSymbol(c_binom_inv, binom_inv, sizeof(binom_inv)));
  }
  PCBA_CK(cudaFuncSetAttribute(k_cand_first<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kCandStageMax));
  PCBA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k3_classify, PCBA_TPB, 0));
  g.k3_grid = std::max(1, PCBA_K3_BLOCKS_PER_SM > 0 ? std::min(occ, PCBA_K3_BLOCKS_PER_SM) : occ) * g.sms;
  // the compaction: every block of k_move_control takes a ticket for the
  // last-block test, so few blocks (the holes of a step fit one pass)
  PCBA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_move_control, PCBA_TPB, 0));
  g.k4_grid = std::max(1, std::min(occ, PCBA_K4_BLOCKS_PER_SM)) * g.sms;
  return 0;
}

#ifndef PCBA_BODY_STEPS
#define PCBA_BODY_STEPS 4
#endif

template <typename T>
int build_graph(pcba_batch* b) {
  PCBA_CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  PCBA_CK(cudaGraphCreate(&b->graph, 0));
  PCBA_CK(cudaGraphConditionalHandleCreate(&b->cond, b->graph, 1, cudaGraphCondAssignDefault));
  // the parameter union has no default constructor: build it in zeroed storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp->type = cudaGraphNodeTypeConditional;
  cp->conditional.handle = b->cond;
  cp->conditional.type = cudaGraphCondTypeWhile;
  cp->conditional.size = 1;
  cudaGraphNode_t node;
  PCBA_CK(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, cp));
  cudaGraph_t body = cp->conditional.phGraph_out[0];
  PCBA_CK(cudaStreamBeginCaptureToGraph(b->cap_stream, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  // PCBA_BODY_STEPS iterations per body: the conditional node's relaunch
  // between bodies costs a few microseconds; an iteration after the loop's
  // end finds no work in any kernel (and is not counted as a step)
  int rc = 0;
  b->refresh_pending = false;
  for (int it = 0; it < PCBA_BODY_STEPS && !rc; ++it) rc = launch_loop_body<T>(b, b->cap_stream, 1);
  if (!rc) rc = join_refresh(b, b->cap_stream);  // the body ends with every stream joined
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &captured);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(PCBA_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  PCBA_CK(cudaGraphInstantiate(&b->gexec, b->graph, 0));
  return 0;
}

// One 3-D tensor map per problem and constraint family over the list:
// dims (patch column, coefficient row, item), strides (row bytes, item bytes),
// box (32, C, 1): one copy brings the [C][32] column block of one parent.
int build_tensor_maps(pcba_batch* b) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  PCBA_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess)
    return fail(PCBA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  auto encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  const int n = b->np;
  std::vector<CUtensorMap> maps((size_t)2 * n);
  std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
  const bool f32 = b->precision == PCBA_FP32;
  const size_t w = f32 ? 4 : 8;
  for (int k = 0; k < n; ++k) {
    const ProbDesc& d = b->desc[k];
    for (int fam = 0; fam < 2; ++fam) {
      const int cnt = fam ? d.beta : d.alpha;
      if (cnt == 0) continue;
      const cuuint64_t pad = (cuuint64_t)(fam ? d.bpad : d.apad);
      const cuuint64_t C = (cuuint64_t)(fam ? d.ch : d.cg);
      char* base = b->d_arena + d.list_off + (fam ? d.off_h : d.off_g);
      const cuuint64_t dims[3] = {pad, C, (cuuint64_t)std::max<long long>(d.M, 1)};
      const cuuint64_t strides[2] = {pad * w, (cuuint64_t)d.item_bytes};
      const cuuint32_t box[3] = {32, (cuuint32_t)C, 1};
      const cuuint32_t estr[3] = {1, 1, 1};
      CUresult r = encode(&maps[(size_t)2 * k + fam],
                          f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                          base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(PCBA_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    }
  }
  cudaError_t e = dev_alloc(&b->d_tmaps, sizeof(CUtensorMap) * maps.size());
  if (e != cudaSuccess) return fail(PCBA_ERR_OOM, "tensor map allocation failed");
  PCBA_CK(cudaMemcpy(b->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                     cudaMemcpyHostToDevice));
  b->E.tmaps = b->d_tmaps;
  return 0;
}

// Selects subdivision configuration 'idx' (0 = direct loads, >= 1 TMA):
// the work units per item follow the kernel (256-patch tiles or 32-patch
// groups), so the descriptors are re-uploaded.
int apply_k2_config(pcba_batch* b, int idx) {
  Grids& g = b->g;
  if (idx < 0 || idx >= (int)g.k2.cfgs.size()) return fail(PCBA_ERR_INVALID, "no such configuration");
  const K2Cfg& c = g.k2.cfgs[idx];
  g.cfg = idx;
  g.tma = c.tma;
  if (c.tma) {
    if (!b->d_tmaps) {
      const int rc = build_tensor_maps(b);
      if (rc) return rc;
    }
  }
  for (ProbDesc& d : b->desc)
    d.tiles = d.lin ? d.lin_chunks
                    : (c.tma ? std::max(1, d.groups_g + d.groups_h) : std::max(1, d.tiles_g + d.tiles_h));
  PCBA_CK(cudaMemcpy(b->d_desc, b->desc.data(), sizeof(ProbDesc) * b->np, cudaMemcpyHostToDevice));
  return 0;
}

int rebuild_graph(pcba_batch* b) {
  if ((b->flags & 3) != 0) return 0;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->cap_stream = nullptr;
  return b->precision == PCBA_FP32 ? build_graph<float>(b) : build_graph<double>(b);
}

int batch_create_impl(pcba_batch** out, pcba_handle** hs, int n, size_t mem_cap_total, int flags) {
  if (!out) return fail(PCBA_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!hs || n < 1) return fail(PCBA_ERR_INVALID, "need at least one problem");
  const int prec = hs[0] ? hs[0]->prob.precision : 0;
  for (int k = 0; k < n; ++k)
    if (!hs[k] || hs[k]->prob.precision != prec)
      return fail(PCBA_ERR_INVALID, "every handle must exist and share one precision");
  pcba_batch* b = new pcba_batch();
  b->np = n;
  b->precision = prec;
  b->flags = flags;
  {
    const char* nt = std::getenv("PCBA_NO_TMA");
    b->want_tma = !(flags & 4) && !(nt && nt[0] == '1');
  }
  b->stream = hs[0]->stream;
  b->lin = hs[0]->prob.lin;
  for (int k = 0; k < n; ++k)
    if (hs[k]->prob.lin != b->lin || (b->lin && hs[k]->prob.alpha != hs[0]->prob.alpha)) {
      delete b;
      return fail(PCBA_ERR_INVALID, "a batch must not mix linear-family and dense problems, "
                                    "and its linear families must share n_shared");
    }
  if ((flags & 8) && !b->lin) {
    delete b;
    return fail(PCBA_ERR_INVALID, "vertex incumbents (flag 8) need linear-family problems");
  }
  b->desc.resize(n);
  long long mono = 0, sum_item = 0, trace_rows = 0, lin_rows = 0;
  for (int k = 0; k < n; ++k) {
    const HostProblem& P = hs[k]->prob;
    b->probs.push_back(&P);
    ProbDesc& d = b->desc[k];
    std::memset(&d, 0, sizeof(d));
    d.l = P.l;
    b->max_l = std::max(b->max_l, P.l);
    d.cp = (int)P.cp;
    d.cg = (int)P.cg;
    d.ch = (int)P.ch;
    d.alpha = P.alpha;
    d.beta = P.beta;
    d.tiles_g = (P.alpha + PCBA_TPB - 1) / PCBA_TPB;
    d.tiles_h = (P.beta + PCBA_TPB - 1) / PCBA_TPB;
    d.tiles = std::max(1, d.tiles_g + d.tiles_h);
    d.groups_g = (P.alpha + 31) / 32;
    d.groups_h = (P.beta + 31) / 32;
    d.form_bernstein = P.form;
    for (int r = 0; r < PCBA_MAXD; ++r) {
      d.P[r] = P.P[r];
      d.G[r] = P.G[r];
      d.H[r] = P.H[r];
      d.lo[r] = P.lo[r];
      d.hi[r] = P.hi[r];
    }
    layout_item(P, prec, d);
    d.lin_off = lin_rows;
    lin_rows += P.nlin;
    d.move_chunks = 1;  // Eliminate moves one map entry per hole
    d.mono_off = mono;
    mono += (long long)P.mono.size();
    d.trace_rows = PCBA_TRACE_PER_DIM * P.l;
    d.trace_off = trace_rows;
    trace_rows += d.trace_rows;
    d.units_k1 = 1 + P.alpha + P.beta;
    sum_item += d.item_bytes;
  }
  long long M = (long long)(mem_cap_total / (size_t)sum_item);
  M = std::min<long long>(M, 1LL << 30);
  b->M = M;
  b->sum_item_bytes = sum_item;
  b->mono_doubles = mono;
  b->lin_rows = lin_rows;
  b->trace_rows_total = trace_rows;
  const long long Mslots = std::max<long long>(M, 2);
  const long long tiles_per = (Mslots + PCBA_TPB - 1) / PCBA_TPB + 1;
  long long list_off = 0;
  for (int k = 0; k < n; ++k) {
    ProbDesc& d = b->desc[k];
    d.M = M;
    d.list_off = list_off;
    list_off += std::max<long long>(M, 1) * d.item_bytes;
    d.slot_off = (long long)k * Mslots;
    d.tile_off = (long long)k * tiles_per;
  }
  const long long arena_bytes = list_off;
  const long long nslots = (long long)n * Mslots;
  b->nslots_total = nslots;
  int rc = 0;
#define PCBA_ALLOC(ptr, bytes)                                                        \
  do {                                                                                \
    cudaError_t e_ = dev_alloc((void**)&(ptr), (size_t)(bytes));                     \
    if (e_ != cudaSuccess) {                                                          \
      free_batch(b);                                                                  \
      return fail(PCBA_ERR_OOM, std::string("device allocation of ") +                \
                                    std::to_string((long long)(bytes)) + " bytes failed"); \
    }                                                                                 \
  } while (0)
  PCBA_ALLOC(b->d_desc, sizeof(ProbDesc) * n);
  PCBA_ALLOC(b->d_state, sizeof(ProbState) * n);
  PCBA_ALLOC(b->d_plan, sizeof(Plan));
  PCBA_ALLOC(b->d_params, sizeof(SolveParams));
  PCBA_ALLOC(b->d_pre, sizeof(unsigned) * 6 * (n + 1));
  PCBA_ALLOC(b->d_arena, arena_bytes);
  PCBA_ALLOC(b->d_rec, sizeof(ChildRec) * nslots);
  PCBA_ALLOC(b->d_slots, sizeof(unsigned) * 5 * nslots);
  PCBA_ALLOC(b->d_tilecnt, sizeof(unsigned) * tiles_per * n);
  PCBA_ALLOC(b->d_mono, sizeof(double) * mono);
  PCBA_ALLOC(b->d_mono32, sizeof(float) * mono);
  PCBA_ALLOC(b->d_ckey, sizeof(float) * n);
  PCBA_ALLOC(b->d_corder, sizeof(int) * n);
  PCBA_ALLOC(b->d_cres, sizeof(int) * n);
  b->ckey_cap = 1;
  for (const ProbDesc& d : b->desc)
    b->cand_floats = std::max(b->cand_floats, (long long)d.alpha * d.cg + (long long)d.beta * d.ch);
  PCBA_ALLOC(b->d_trace, sizeof(double) * 4 * trace_rows);
  PCBA_ALLOC(b->d_warm, sizeof(double) * PCBA_MAXD * n);
  PCBA_ALLOC(b->d_mat, sizeof(double) * 3 * PCBA_MAXD * 578 * n);
  PCBA_ALLOC(b->d_raw, sizeof(double) * mono);
  PCBA_ALLOC(b->d_eval, sizeof(EvalOut) * n);
  PCBA_ALLOC(b->d_lin32, sizeof(float) * PCBA_LIN32_STRIDE * std::max<long long>(lin_rows, 1));
  PCBA_ALLOC(b->d_lin64, sizeof(double) * PCBA_LIN_STRIDE * std::max<long long>(lin_rows, 1));
  // queue of heavy (item, window) units: every item of every problem with all
  // its chunks, at most 4 Mi entries (a full queue leaves units to the split)
  long long qcap = 0;
  if (b->lin)
    for (int k = 0; k < n; ++k)
      qcap = std::min<long long>(qcap + (long long)std::max<long long>(M, 2) *
                                            b->desc[k].lin_chunks, 1LL << 22);
  PCBA_ALLOC(b->d_lin_queue, sizeof(uint4) * std::max<long long>(qcap, 1));
  const unsigned mark_cap = 1u << 20;  // marked patches per step (extra marks are dropped)
  PCBA_ALLOC(b->d_marks, sizeof(uint4) * 2 * (prec == PCBA_FP32 ? mark_cap : 1));
#undef PCBA_ALLOC
  auto host_alloc = [&](void** p, size_t bytes) { return cudaMallocHost(p, bytes); };
  if (host_alloc((void**)&b->h_state, sizeof(ProbState) * n) != cudaSuccess ||
      host_alloc((void**)&b->h_eval, sizeof(EvalOut) * n) != cudaSuccess ||
      host_alloc((void**)&b->h_plan, sizeof(Plan)) != cudaSuccess ||
      host_alloc((void**)&b->h_params, sizeof(SolveParams)) != cudaSuccess ||
      host_alloc((void**)&b->h_running, sizeof(int)) != cudaSuccess) {
    free_batch(b);
    return fail(PCBA_ERR_OOM, "pinned host allocation failed");
  }
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      free_batch(b);
      return fail(PCBA_ERR_CUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  auto cleanup_ck = [&](cudaError_t e, const char* what) -> int {
    if (e == cudaSuccess) return 0;
    free_batch(b);
    return fail(PCBA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  if ((rc = cleanup_ck(cudaMemcpy(b->d_desc, b->desc.data(), sizeof(ProbDesc) * n,
                                  cudaMemcpyHostToDevice), "desc upload")))
    return rc;
  {
    std::vector<double> all((size_t)mono);
    for (int k = 0; k < n; ++k)
      std::copy(b->probs[k]->mono.begin(), b->probs[k]->mono.end(),
                all.begin() + b->desc[k].mono_off);
    if ((rc = cleanup_ck(cudaMemcpy(b->d_mono, all.data(), sizeof(double) * mono,
                                    cudaMemcpyHostToDevice), "mono upload")))
      return rc;
  }
  if (lin_rows > 0) {
    // constraint rows (c_i, w_i0 .. w_i,K-1), in FP64 and as FP32 pairs
    std::vector<double> t64((size_t)(PCBA_LIN_STRIDE * lin_rows), 0.0);
    std::vector<float> t32((size_t)(PCBA_LIN32_STRIDE * lin_rows), 0.0f);
    for (int k = 0; k < n; ++k) {
      const HostProblem& P = *b->probs[k];
      for (int i = 0; i < P.nlin; ++i) {
        double* row = t64.data() + (size_t)(b->desc[k].lin_off + i) * PCBA_LIN_STRIDE;
        row[0] = P.lin_c[i];
        for (int m = 0; m < P.alpha; ++m) row[1 + m] = P.lin_w[(size_t)i * P.alpha + m];
      }
    }
    for (long long q = 0; q < lin_rows; ++q)
      for (int j = 0; j < PCBA_LIN_STRIDE; ++j) {
        const double x = t64[(size_t)q * PCBA_LIN_STRIDE + j];
        const float hi = (float)x;
        t32[(size_t)q * PCBA_LIN32_STRIDE + j] = hi;
        t32[(size_t)q * PCBA_LIN32_STRIDE + PCBA_LIN_STRIDE + j] = (float)(x - (double)hi);
      }
    if ((rc = cleanup_ck(cudaMemcpy(b->d_lin64, t64.data(), sizeof(double) * t64.size(),
                                    cudaMemcpyHostToDevice), "linear rows upload")))
      return rc;
    if ((rc = cleanup_ck(cudaMemcpy(b->d_lin32, t32.data(), sizeof(float) * t32.size(),
                                    cudaMemcpyHostToDevice), "linear rows upload")))
      return rc;
  }
  std::vector<unsigned> k1pre(n + 1, 0);
  for (int k = 0; k < n; ++k) k1pre[k + 1] = k1pre[k] + (unsigned)b->desc[k].units_k1;
  unsigned* pre = b->d_pre;
  if ((rc = cleanup_ck(cudaMemcpy(pre + 4 * (n + 1), k1pre.data(), sizeof(unsigned) * (n + 1),
                                  cudaMemcpyHostToDevice), "k1 prefix")))
    return rc;
  if ((rc = cleanup_ck(cudaMemset(b->d_rec, 0, sizeof(ChildRec) * nslots), "rec clear"))) return rc;
  if ((rc = cleanup_ck(cudaMemset(b->d_slots, 0, sizeof(unsigned) * 5 * nslots), "slot clear")))
    return rc;
  if ((rc = cleanup_ck(cudaMemset(b->d_state, 0, sizeof(ProbState) * n), "state clear"))) return rc;
  if ((rc = cleanup_ck(cudaEventCreate(&b->ev0), "event"))) return rc;
  if ((rc = cleanup_ck(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming), "event")))
    return rc;
  if ((rc = cleanup_ck(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming), "event")))
    return rc;
  if ((rc = cleanup_ck(cudaEventCreateWithFlags(&b->ev_k1f, cudaEventDisableTiming), "event")))
    return rc;
  if ((rc = cleanup_ck(cudaEventCreateWithFlags(&b->ev_k1j, cudaEventDisableTiming), "event")))
    return rc;
  if ((rc = cleanup_ck(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking), "stream")))
    return rc;
  if ((rc = cleanup_ck(cudaEventCreate(&b->ev1), "event"))) return rc;
  Engine& E = b->E;
  E.np = n;
  E.precision = prec;
  E.desc = b->d_desc;
  E.state = b->d_state;
  E.plan = b->d_plan;
  E.params = b->d_params;
  E.k2_pre = pre;
  E.k3_pre = pre + (n + 1);
  E.k3_pre_next = pre + 2 * (n + 1);
  E.k4_pre = pre + 3 * (n + 1);
  E.k1_pre = pre + 4 * (n + 1);
  E.kr_pre = pre + 5 * (n + 1);
  E.marks = b->d_marks;
  E.mark_cap = prec == PCBA_FP32 ? mark_cap : 0;
  E.arena = b->d_arena;
  E.rec = b->d_rec;
  E.flagrank = b->d_slots;
  E.hole = b->d_slots + nslots;
  E.filler = b->d_slots + 2 * nslots;
  E.map = b->d_slots + 3 * nslots;
  E.fstack = b->d_slots + 4 * nslots;
  E.tilecnt = b->d_tilecnt;
  E.mono = b->d_mono;
  E.mono32 = b->d_mono32;
  E.trace = b->d_trace;
  E.warm = b->d_warm;
  E.n_warm = 1;
  E.root_raw = nullptr;
  E.lin32 = b->d_lin32;
  E.lin64 = b->d_lin64;
  E.lin_queue = b->d_lin_queue;
  E.lin_qcap = (unsigned)qcap;
  rc = prec == PCBA_FP32 ? setup_kernels<float>(b) : setup_kernels<double>(b);
  if (!rc) rc = apply_k2_config(b, (b->want_tma && b->g.k2.cfgs.size() > 1) ? 1 : 0);
  if (!rc && (flags & 3) == 0) rc = prec == PCBA_FP32 ? build_graph<float>(b) : build_graph<double>(b);
  if (rc) {
    std::string msg = g_err;
    free_batch(b);
    return fail(rc, msg);
  }
  *out = b;
  return 0;
}

// Guesses of a guided solve (pcba_batch_solve_guided).
struct Guide {
  const float* guess;
  int dim;
  const double* stencil;  // host
  int n;
};

template <typename T>
int run_solve(pcba_batch* b, const double* host_coeffs, double opt_tol, double eq_tol,
              int max_iters, int max_steps, const double* warm, bool want_raw,
              const Guide* guide) {
  cudaStream_t s = b->stream;
  const int n = b->np;
  SolveParams& P = *b->h_params;
  P.opt_tol = opt_tol;
  P.eq_tol = eq_tol;
  P.max_iters = max_iters;
  P.max_steps = max_steps;
  P.step_guard = b->max_l * max_iters + 4;
  {
    // test hook: a smaller guard makes the device loop stop before max_iters
    // does, so that PCBA_ERR_DEVICE_TIMEOUT can be exercised without a fault
    const char* g = std::getenv("PCBA_TEST_STEP_GUARD");
    if (g && std::atoi(g) > 0) P.step_guard = std::min(P.step_guard, std::atoi(g));
  }
  P.np = n;
  P.time_limit_ns = b->time_limit_s > 0.0 ? (unsigned long long)(b->time_limit_s * 1e9) : 0ull;
  P.vertex = (b->flags & 8) ? 1 : 0;

  PCBA_CK(cudaEventRecord(b->ev0, s));
  b->h2d_bytes = (long long)sizeof(SolveParams) + (host_coeffs ? 8LL * b->mono_doubles : 0) +
                 (warm ? 8LL * PCBA_MAXD * n : 0) +
                 (guide ? 8LL * guide->n * guide->dim : 0) +
                 (guide ? 8LL * b->refine_total() * b->refine_dim : 0) + b->pending_h2d;
  b->pending_h2d = 0;
  const bool have_warm = warm || b->warm_on_device;
  b->extra_launches = (guide || have_warm ? 1 : 0) + (guide ? 1 : 0) + b->extra_launches_pending;
  b->extra_launches_pending = 0;
  b->d2h_bytes = (long long)(sizeof(ProbState) + sizeof(EvalOut)) * n + (long long)sizeof(Plan);
  if (host_coeffs)
    PCBA_CK(cudaMemcpyAsync(b->d_mono, host_coeffs, sizeof(double) * b->mono_doubles,
                            cudaMemcpyHostToDevice, s));
  PCBA_CK(cudaMemcpyAsync(b->d_params, b->h_params, sizeof(SolveParams), cudaMemcpyHostToDevice, s));
  if (warm)
    PCBA_CK(cudaMemcpyAsync(b->d_warm, warm, sizeof(double) * PCBA_MAXD * n,
                            cudaMemcpyHostToDevice, s));
  else if (!b->warm_on_device)
    PCBA_CK(cudaMemsetAsync(b->d_warm, 0xFF, sizeof(double) * PCBA_MAXD * n, s));  // NaN
  Engine E1 = b->E;
  E1.root_raw = want_raw ? b->d_raw : nullptr;
  // InitPatches (Alg. 1 line 1) writes only the root items; the warm-start
  // kernels read the monomials and write candidate buffers and the seed
  // fields of the state, so K1 runs on the side stream beside them and
  // joins before k_init
  PCBA_CK(cudaEventRecord(b->ev_k1f, s));
  PCBA_CK(cudaStreamWaitEvent(b->side, b->ev_k1f, 0));
  const int nmat = n * 3 * PCBA_MAXD * 17;
  k1_matrices<<<(nmat + 255) / 256, 256, 0, b->side>>>(E1, b->d_mat);
  k1_convert<T><<<b->g.k1_grid, 32 * b->g.k1_wpb, b->g.k1_smem, b->side>>>(E1, b->d_mat, b->g.k1_cmax,
                                                                   b->g.k1_wpb);
  if (guide || have_warm) {
    const unsigned cg = (unsigned)std::min<long long>((b->mono_doubles + 255) / 256, 4LL * b->g.sms);
    k_mono32<<<cg, 256, 0, s>>>(b->d_mono, b->d_mono32, b->mono_doubles);
  }
  if (guide) {
    PCBA_CK(cudaMemcpyAsync(b->d_stencil, guide->stencil, sizeof(double) * guide->n * guide->dim,
                            cudaMemcpyHostToDevice, s));
    const long long nc = (long long)n * guide->n;
    k_candidates<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(E1, guide->guess, guide->dim,
                                                             b->d_stencil, guide->n, b->d_cand, 0);
    E1.warm = b->d_cand;
    E1.n_warm = guide->n;
  }
  // candidates ranked by their FP32 cost bound; the lowest certified-feasible
  // rank seeds p_up (the constraint coefficients staged in shared memory when
  // they fit)
  auto certify = [&](const Engine& Ec) -> int {
    if (b->ckey_cap < Ec.n_warm || Ec.n_warm > PCBA_MAX_CAND) {
      k_eval<<<n, PCBA_TPB, 0, s>>>(Ec, 0, nullptr);
      return 0;
    }
    const long long nc = (long long)n * Ec.n_warm;
    k_cand_cost<<<(unsigned)std::min<long long>((nc + 255) / 256, 8LL * b->g.sms), 256, 0, s>>>(
        Ec, b->d_ckey);
    k_cand_rank<<<n, PCBA_TPB, 0, s>>>(Ec, b->d_ckey, b->d_corder, b->d_cres);
    const size_t stage = sizeof(float) * (size_t)b->cand_floats;
    // blocks per problem: enough to cover about twice the SMs, at most 4
    const dim3 fgrid((unsigned)n, (unsigned)std::max(1, std::min(4, 2 * b->g.sms / std::max(1, n))));
    if (stage <= kCandStageMax)
      k_cand_first<true><<<fgrid, PCBA_CAND_TPB, stage, s>>>(Ec, b->d_ckey, b->d_corder, b->d_cres);
    else
      k_cand_first<false><<<fgrid, PCBA_CAND_TPB, 0, s>>>(Ec, b->d_ckey, b->d_corder, b->d_cres);
    k_cand_pick<<<n, 32, 0, s>>>(Ec, b->d_corder, b->d_cres);
    b->extra_launches += 3;
    return 0;
  };
  if (guide || have_warm) {
    int rc = certify(E1);
    if (rc) return rc;
    for (size_t rd = 0; guide && rd < b->refine.size(); ++rd) {
      // a finer stencil around each problem's seed (the centre row of zeros
      // keeps the previous seed among the candidates)
      const int rn = b->refine_rows[rd];
      PCBA_CK(cudaMemcpyAsync(b->d_stencil, b->refine[rd].data(),
                              sizeof(double) * rn * b->refine_dim, cudaMemcpyHostToDevice, s));
      const long long nc = (long long)n * rn;
      k_candidates<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(
          E1, guide->guess, b->refine_dim, b->d_stencil, rn, b->d_cand, 1);
      Engine E2 = E1;
      E2.n_warm = rn;
      b->extra_launches += 1;
      rc = certify(E2);
      if (rc) return rc;
    }
  } else {
    k_eval<<<n, PCBA_TPB, 0, s>>>(E1, 0, nullptr);
  }
  PCBA_CK(cudaEventRecord(b->ev_k1j, b->side));
  PCBA_CK(cudaStreamWaitEvent(s, b->ev_k1j, 0));
  k_init<<<1, PCBA_TPB, 0, s>>>(E1);
  PCBA_CK(cudaGetLastError());
  b->subdiv_ms = 0;
  b->subdiv_bytes = 0;
  b->subdiv_launches = 0;
  const bool instrument = (b->flags & 2) != 0;
  if ((b->flags & 3) == 0) {
    PCBA_CK(cudaGraphLaunch(b->gexec, s));
  } else {
    const int guard = b->max_l * max_iters + 8;
    std::vector<double> launch_bytes;
    if (instrument) {
      PCBA_CK(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(ProbState) * n,
                              cudaMemcpyDeviceToHost, s));
      PCBA_CK(cudaStreamSynchronize(s));
      while ((int)b->kev.size() < 2 * guard) {
        cudaEvent_t e;
        PCBA_CK(cudaEventCreate(&e));
        b->kev.push_back(e);
      }
    }
    int it = 0;
    for (;; ++it) {
      if (it >= guard) return fail(PCBA_ERR_DEVICE_TIMEOUT, "host loop guard reached");
      if (int rc2 = join_refresh(b, s)) return rc2;
      if (instrument) {
        double bytes = 0;
        for (int k = 0; k < n; ++k)
          if (b->h_state[k].status == PCBA_RUNNING)
            bytes += 3.0 * (double)b->h_state[k].K * (double)b->desc[k].payload_bytes;
        launch_bytes.push_back(bytes);
        PCBA_CK(cudaEventRecord(b->kev[2 * it], s));
      }
      launch_k2<T>(b, s);
      if (instrument) PCBA_CK(cudaEventRecord(b->kev[2 * it + 1], s));
      const int rc = launch_after_k2<T>(b, s, 0);
      if (rc) return rc;
      PCBA_CK(cudaMemcpyAsync(b->h_running, &b->d_plan->any_running, sizeof(int),
                              cudaMemcpyDeviceToHost, s));
      if (instrument)
        PCBA_CK(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(ProbState) * n,
                                cudaMemcpyDeviceToHost, s));
      PCBA_CK(cudaStreamSynchronize(s));
      if (!*b->h_running) break;
    }
    if (instrument) {
      b->launch_bytes = launch_bytes;
      for (int q = 0; q <= it; ++q) {
        if (launch_bytes[q] <= 0) continue;
        float ms = 0;
        PCBA_CK(cudaEventElapsedTime(&ms, b->kev[2 * q], b->kev[2 * q + 1]));
        b->subdiv_ms += ms;
        b->subdiv_bytes += launch_bytes[q];
        b->subdiv_launches += 1;
      }
    }
  }
  if (int rc2 = join_refresh(b, s)) return rc2;
  k_eval<<<n, PCBA_TPB, 0, s>>>(b->E, 1, b->d_eval);
  PCBA_CK(cudaGetLastError());
  PCBA_CK(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(ProbState) * n, cudaMemcpyDeviceToHost, s));
  PCBA_CK(cudaMemcpyAsync(b->h_eval, b->d_eval, sizeof(EvalOut) * n, cudaMemcpyDeviceToHost, s));
  PCBA_CK(cudaMemcpyAsync(b->h_plan, b->d_plan, sizeof(Plan), cudaMemcpyDeviceToHost, s));
  PCBA_CK(cudaEventRecord(b->ev1, s));
  PCBA_CK(cudaStreamSynchronize(s));
  float ms = 0;
  PCBA_CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  b->total_ms = ms;
  if (b->h_plan->guard_hit == 2)
    return fail(PCBA_ERR_DEVICE_TIMEOUT, "a bulk copy of the subdivision kernel did not complete");

  if (b->h_plan->guard_hit) return fail(PCBA_ERR_DEVICE_TIMEOUT, "device loop guard reached");
  return 0;
}

void fill_results(const pcba_batch* b, pcba_result* out) {
  for (int k = 0; k < b->np; ++k) {
    const ProbState& S = b->h_state[k];
    const ProbDesc& d = b->desc[k];
    const EvalOut& ev = b->h_eval[k];
    pcba_result& R = out[k];
    std::memset(&R, 0, sizeof(R));
    R.status = S.status;
    R.steps = S.steps;
    R.sweeps = S.n;
    R.lower = S.p_lo;
    R.upper = S.p_up;
    R.peak_items = S.peak_items;
    R.peak_bytes = S.peak_items * d.item_bytes;
    const bool point = S.status != PCBA_INFEASIBLE && (S.have_box || S.from_warm);
    R.from_warm_start = point && !S.have_box && S.from_warm ? 1 : 0;
    for (int q = 0; q < PCBA_MAX_DIM; ++q) {
      R.x[q] = R.box_lo[q] = R.box_hi[q] = NAN;
    }
    if (point) {
      for (int q = 0; q < d.l; ++q) {
        if (S.have_box) {
          const double w = std::ldexp(d.hi[q] - d.lo[q], -S.best_level[q]);
          R.box_lo[q] = d.lo[q] + w * (double)S.best_index[q];
          R.box_hi[q] = d.lo[q] + w * (double)(S.best_index[q] + 1u);
          R.x[q] = 0.5 * (R.box_lo[q] + R.box_hi[q]);
        } else {
          R.x[q] = S.warm_x[q];
        }
      }
    }
    if (S.status == PCBA_INFEASIBLE) {
      R.verify_cost = R.verify_max_g = R.verify_max_abs_h = NAN;
    } else {
      R.verify_cost = ev.ok ? ev.cost : NAN;
      R.verify_max_g = ev.ok ? ev.max_g : NAN;
      R.verify_max_abs_h = ev.ok ? ev.max_abs_h : NAN;
    }
    const unsigned long long t0 = b->h_plan->t0;
    R.time_ms = S.t_end >= t0 ? (double)(S.t_end - t0) * 1e-6 : 0.0;
    R.upper_err = !point ? 0.0 : (S.have_box ? (double)S.box_err : S.warm_err);
  }
}

// barrier weight of the first polish level relative to max(1, |p(x0)|), and
// the Newton steps per level
constexpr double kPolishMu0 = 1e-2;
constexpr int kPolishIters = 30;

// k_polish for every dimension present in the batch, on the batch's stream
int launch_polish(pcba_batch* b, double* d_out, double mu0, double gap, double eq_tol, int iters,
                  int* launches) {
  if (b->lin) return fail(PCBA_ERR_INVALID, "the polish needs dense constraints (no linear family)");
  if (!(mu0 > 0.0) || !(gap > 0.0) || !(eq_tol > 0.0) || iters < 1 || iters > 200)
    return fail(PCBA_ERR_INVALID, "need mu0, gap, eq_tol > 0 and 1 <= iters <= 200");
  bool seen[PCBA_MAXD + 1] = {};
  for (int k = 0; k < b->np; ++k) seen[b->desc[k].l] = true;
  for (int L = 1; L <= PCBA_MAXD; ++L) {
    if (!seen[L]) continue;
    const int rc = pcba_polish_launch(b->E, L, (unsigned)b->np, b->stream, d_out, mu0, gap,
                                      eq_tol, iters);
    if (rc) return rc;
    ++*launches;
  }
  return 0;
}

int batch_solve_impl(pcba_batch* b, const double* host_coeffs, double opt_tol, double eq_tol,
                     int max_iters, int max_steps, const double* warm, pcba_result* out,
                     bool want_raw = false, const Guide* guide = nullptr) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (!(opt_tol > 0) || !(eq_tol > 0)) return fail(PCBA_ERR_INVALID, "tolerances must be > 0");
  if (max_iters < 1 || max_iters > 64) return fail(PCBA_ERR_INVALID, "max_iters must be in [1, 64]");
  if (max_steps < 0) return fail(PCBA_ERR_INVALID, "max_steps must be >= 0");
  b->prior_launches = b->prior_h2d = b->prior_d2h = 0;
  const int rc = b->precision == PCBA_FP32
                     ? run_solve<float>(b, host_coeffs, opt_tol, eq_tol, max_iters, max_steps, warm,
                                        want_raw, guide)
                     : run_solve<double>(b, host_coeffs, opt_tol, eq_tol, max_iters, max_steps, warm,
                                         want_raw, guide);
  if (rc) return rc;
  if (out) fill_results(b, out);
  return 0;
}

int own_batch(pcba_handle* h, size_t mem_cap, pcba_batch** out) {
  if (h->own && h->own_cap == mem_cap) {
    *out = h->own;
    return 0;
  }
  if (h->own) {
    free_batch(h->own);
    h->own = nullptr;
  }
  pcba_handle* hs[1] = {h};
  const int rc = batch_create_impl(&h->own, hs, 1, mem_cap, 0);
  if (rc) return rc;
  h->own_cap = mem_cap;
  *out = h->own;
  return 0;
}

}  // namespace

// error reporting shared with the other source files of the library
int pcba_internal_fail(int code, const std::string& msg) { return fail(code, msg); }

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int pcba_version(void) { return 1; }

const char* pcba_last_error(void) { return g_err.c_str(); }

const char* pcba_status_string(int s) {
  switch (s) {
    case PCBA_OPTIMAL: return "OPTIMAL";
    case PCBA_INFEASIBLE: return "INFEASIBLE";
    case PCBA_MEMCAP: return "MEMCAP";
    case PCBA_MAXITER: return "MAXITER";
    case PCBA_TIMEOUT: return "TIMEOUT";
    case PCBA_STEPLIMIT: return "STEPLIMIT";
    case PCBA_ERR_INVALID: return "ERR_INVALID";
    case PCBA_ERR_CUDA: return "ERR_CUDA";
    case PCBA_ERR_OOM: return "ERR_OOM";
    case PCBA_ERR_DEVICE_TIMEOUT: return "ERR_DEVICE_TIMEOUT";
    default: return "UNKNOWN";
  }
}

int pcba_create(pcba_handle** out, const pcba_poly* cost, const pcba_poly* ineq, int n_ineq,
                const pcba_poly* eq, int n_eq, const pcba_box* box, int precision) {
  return create_impl(out, cost, ineq, n_ineq, eq, n_eq, box, precision, 0);
}

int pcba_create_bernstein(pcba_handle** out, const pcba_poly* cost, const pcba_poly* ineq,
                          int n_ineq, const pcba_poly* eq, int n_eq, const pcba_box* box,
                          int precision) {
  return create_impl(out, cost, ineq, n_ineq, eq, n_eq, box, precision, 1);
}

int pcba_create_linear(pcba_handle** out, const pcba_poly* cost,
                       const pcba_linear_family* fam, const pcba_box* box, int precision) {
  if (out) *out = nullptr;
  if (!fam) return fail(PCBA_ERR_INVALID, "linear family is null");
  if (fam->n_shared < 1 || fam->n_shared > PCBA_MAX_SHARED || !fam->shared)
    return fail(PCBA_ERR_INVALID, "linear family: n_shared must be 1..4");
  if (fam->n_constraints < 0 || fam->n_constraints > (1 << 20))
    return fail(PCBA_ERR_INVALID, "linear family: n_constraints must be 0..2^20");
  if (fam->n_constraints > 0 && (!fam->weight || !fam->offset))
    return fail(PCBA_ERR_INVALID, "linear family: weight or offset is null");
  const long long nw = (long long)fam->n_constraints * fam->n_shared;
  for (long long q = 0; q < nw; ++q)
    if (!std::isfinite(fam->weight[q])) return fail(PCBA_ERR_INVALID, "non-finite weight");
  for (int i = 0; i < fam->n_constraints; ++i)
    if (!std::isfinite(fam->offset[i])) return fail(PCBA_ERR_INVALID, "non-finite offset");
  // the shared polynomials are stored as the inequality family of the handle
  int rc = create_impl(out, cost, fam->shared, fam->n_shared, nullptr, 0, box, precision, 0);
  if (rc) return rc;
  HostProblem& P = (*out)->prob;
  P.lin = 1;
  P.nlin = fam->n_constraints;
  P.lin_c.assign(fam->offset, fam->offset + fam->n_constraints);
  P.lin_w.assign(fam->weight, fam->weight + nw);
  return 0;
}

int pcba_get_active(pcba_handle* h, unsigned* bits, long long max_words) {
  if (!h) return fail(PCBA_ERR_INVALID, "handle is null");
  if (!h->prob.lin) return 0;
  if (!h->own) return fail(PCBA_ERR_INVALID, "no solve has run on this handle");
  pcba_batch* b = h->own;
  const ProbDesc& d = b->desc[0];
  const long long K = b->h_state[0].K;
  if (bits) {
    if (max_words < K * d.mwords) return fail(PCBA_ERR_INVALID, "activity buffer too small");
    const long long nslots_total = b->nslots_total;
    std::vector<unsigned> slot((size_t)std::max<long long>(K, 1));
    PCBA_CK(cudaMemcpy(slot.data(), b->d_slots + 3 * nslots_total + d.slot_off,
                       sizeof(unsigned) * (size_t)K, cudaMemcpyDeviceToHost));
    for (long long k = 0; k < K; ++k)
      PCBA_CK(cudaMemcpy(bits + k * d.mwords,
                         b->d_arena + d.list_off + (size_t)slot[(size_t)k] * d.item_bytes +
                             d.off_mask,
                         sizeof(unsigned) * (size_t)d.mwords, cudaMemcpyDeviceToHost));
  }
  return d.mwords;
}

void pcba_destroy(pcba_handle* h) {
  if (!h) return;
  free_batch(h->own);
  delete h;
}

int pcba_set_stream(pcba_handle* h, void* stream) {
  if (!h) return fail(PCBA_ERR_INVALID, "handle is null");
  h->stream = (cudaStream_t)stream;
  if (h->own) {
    free_batch(h->own);
    h->own = nullptr;
  }
  return 0;
}

int pcba_set_warm_start(pcba_handle* h, const double* x) {
  if (!h) return fail(PCBA_ERR_INVALID, "handle is null");
  if (!x) {
    h->has_warm = false;
    return 0;
  }
  for (int q = 0; q < h->prob.l; ++q)
    if (!std::isfinite(x[q])) return fail(PCBA_ERR_INVALID, "warm start must be finite");
  h->has_warm = true;
  for (int q = 0; q < PCBA_MAXD; ++q) h->warm[q] = q < h->prob.l ? x[q] : 0.0;
  return 0;
}

int pcba_set_time_limit(pcba_handle* h, double seconds) {
  if (!h) return fail(PCBA_ERR_INVALID, "handle is null");
  if (!(seconds >= 0.0) || !std::isfinite(seconds))
    return fail(PCBA_ERR_INVALID, "time limit must be finite and >= 0");
  h->time_limit_s = seconds;
  return 0;
}

int pcba_batch_set_time_limit(pcba_batch* b, double seconds) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (!(seconds >= 0.0) || !std::isfinite(seconds))
    return fail(PCBA_ERR_INVALID, "time limit must be finite and >= 0");
  b->time_limit_s = seconds;
  return 0;
}

long long pcba_item_bytes(const pcba_handle* h) {
  if (!h) return fail(PCBA_ERR_INVALID, "handle is null");
  ProbDesc d;
  std::memset(&d, 0, sizeof(d));
  layout_item(h->prob, h->prob.precision, d);
  return d.item_bytes;
}

int pcba_solve_steps(pcba_handle* h, double opt_tol, double eq_tol, int max_iters, size_t mem_cap,
                     int max_steps, pcba_result* out) {
  if (!h) return fail(PCBA_ERR_INVALID, "handle is null");
  pcba_batch* b = nullptr;
  int rc = own_batch(h, mem_cap, &b);
  if (rc) return rc;
  b->time_limit_s = h->time_limit_s;
  return batch_solve_impl(b, nullptr, opt_tol, eq_tol, max_iters, max_steps,
                          h->has_warm ? h->warm : nullptr, out);
}

int pcba_solve(pcba_handle* h, double opt_tol, double eq_tol, int max_iters, size_t mem_cap,
               pcba_result* out) {
  return pcba_solve_steps(h, opt_tol, eq_tol, max_iters, mem_cap, 0, out);
}

int pcba_batch_create(pcba_batch** out, pcba_handle** hs, int n, size_t mem_cap_total, int flags) {
  if (flags < 0 || flags > 15) return fail(PCBA_ERR_INVALID, "flags must be 0..15");
  return batch_create_impl(out, hs, n, mem_cap_total, flags);
}

int pcba_batch_solve(pcba_batch* b, double opt_tol, double eq_tol, int max_iters,
                     const double* warm_start, pcba_result* out) {
  return batch_solve_impl(b, nullptr, opt_tol, eq_tol, max_iters, 0, warm_start, out);
}

int pcba_batch_solve_from_host(pcba_batch* b, const double* host_coeffs, double opt_tol,
                               double eq_tol, int max_iters, const double* warm_start,
                               pcba_result* out) {
  if (!host_coeffs) return fail(PCBA_ERR_INVALID, "host_coeffs is null");
  return batch_solve_impl(b, host_coeffs, opt_tol, eq_tol, max_iters, 0, warm_start, out);
}

int pcba_batch_solve_guided(pcba_batch* b, double opt_tol, double eq_tol, int max_iters,
                            const float* d_guess, int guess_dim, const double* stencil,
                            int n_stencil, pcba_result* out) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (!d_guess || !stencil) return fail(PCBA_ERR_INVALID, "guess or stencil is null");
  if (guess_dim < 1 || guess_dim > PCBA_MAX_DIM)
    return fail(PCBA_ERR_INVALID, "guess_dim must be in [1, 8]");
  if (n_stencil < 1 || n_stencil > 1024)
    return fail(PCBA_ERR_INVALID, "n_stencil must be in [1, 1024]");
  for (long long i = 0; i < (long long)n_stencil * guess_dim; ++i)
    if (!std::isfinite(stencil[i])) return fail(PCBA_ERR_INVALID, "stencil must be finite");
  const int n_cap = std::max(n_stencil, b->refine_max());
  if (!b->refine.empty() && b->refine_dim != guess_dim)
    return fail(PCBA_ERR_INVALID, "refinement stencil and guess dimensions differ");
  if (b->cand_cap < n_cap) {
    if (b->d_cand) cudaFree(b->d_cand);
    b->d_cand = nullptr;
    b->cand_cap = 0;
    if (cudaMalloc((void**)&b->d_cand, sizeof(double) * PCBA_MAXD * (size_t)b->np * n_cap) !=
        cudaSuccess)
      return fail(PCBA_ERR_OOM, "candidate buffer allocation failed");
    b->cand_cap = n_cap;
  }
  if (b->stencil_cap < (long long)n_cap * guess_dim) {
    if (b->d_stencil) cudaFree(b->d_stencil);
    b->d_stencil = nullptr;
    b->stencil_cap = 0;
    if (cudaMalloc((void**)&b->d_stencil, sizeof(double) * (size_t)n_cap * guess_dim) !=
        cudaSuccess)
      return fail(PCBA_ERR_OOM, "stencil buffer allocation failed");
    b->stencil_cap = (long long)n_cap * guess_dim;
  }
  if (b->ckey_cap < n_cap) {
    if (b->d_ckey) cudaFree(b->d_ckey);
    if (b->d_corder) cudaFree(b->d_corder);
    b->d_ckey = nullptr;
    b->d_corder = nullptr;
    b->ckey_cap = 0;
    if (cudaMalloc((void**)&b->d_ckey, sizeof(float) * (size_t)b->np * n_cap) != cudaSuccess ||
        cudaMalloc((void**)&b->d_corder, sizeof(int) * (size_t)b->np * n_cap) != cudaSuccess)
      return fail(PCBA_ERR_OOM, "candidate key allocation failed");
    b->ckey_cap = n_cap;
  }
  const Guide g{d_guess, guess_dim, stencil, n_stencil};
  return batch_solve_impl(b, nullptr, opt_tol, eq_tol, max_iters, 0, nullptr, out, false, &g);
}

int pcba_batch_set_refine_stencil(pcba_batch* b, int round, const double* stencil,
                                  int n_stencil, int guess_dim) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (round < 0 || round >= 4 || round > (int)b->refine.size())
    return fail(PCBA_ERR_INVALID, "refinement round must be in [0, 4) and follow the set ones");
  if (n_stencil == 0) {
    b->refine.resize((size_t)round);
    b->refine_rows.resize((size_t)round);
    return 0;
  }
  if (!stencil || n_stencil < 0 || n_stencil > 1024 || guess_dim < 1 || guess_dim > PCBA_MAX_DIM)
    return fail(PCBA_ERR_INVALID, "refinement stencil: 1..1024 rows of 1..8 values");
  if (round > 0 && guess_dim != b->refine_dim)
    return fail(PCBA_ERR_INVALID, "refinement rounds must share the guess dimension");
  for (long long i = 0; i < (long long)n_stencil * guess_dim; ++i)
    if (!std::isfinite(stencil[i])) return fail(PCBA_ERR_INVALID, "stencil must be finite");
  b->refine.resize((size_t)round + 1);
  b->refine_rows.resize((size_t)round + 1);
  b->refine[(size_t)round].assign(stencil, stencil + (size_t)n_stencil * guess_dim);
  b->refine_rows[(size_t)round] = n_stencil;
  b->refine_dim = guess_dim;
  return 0;
}

int pcba_batch_upload(pcba_batch* b, const double* host_coeffs) {
  if (!b || !host_coeffs) return fail(PCBA_ERR_INVALID, "batch or host_coeffs is null");
  PCBA_CK(cudaMemcpyAsync(b->d_mono, host_coeffs, sizeof(double) * b->mono_doubles,
                          cudaMemcpyHostToDevice, b->stream));
  b->pending_h2d += 8LL * b->mono_doubles;
  return 0;
}

int pcba_batch_upload_rows(pcba_batch* b, const double* host_rows) {
  if (!b || !host_rows) return fail(PCBA_ERR_INVALID, "batch or host_rows is null");
  if (!b->lin) return fail(PCBA_ERR_INVALID, "the batch has no linear-family constraints");
  const long long n = (long long)PCBA_LIN_STRIDE * b->lin_rows;
  if (n == 0) return 0;
  PCBA_CK(cudaMemcpyAsync(b->d_lin64, host_rows, sizeof(double) * n, cudaMemcpyHostToDevice,
                          b->stream));
  const unsigned g = (unsigned)std::min<long long>((n + 255) / 256, 4LL * b->g.sms);
  k_rows32<<<g, 256, 0, b->stream>>>(b->d_lin64, b->d_lin32, b->lin_rows);
  PCBA_CK(cudaGetLastError());
  b->pending_h2d += 8LL * n;
  b->extra_launches_pending += 1;
  return 0;
}

long long pcba_batch_rows_doubles(const pcba_batch* b) {
  return b ? (long long)PCBA_LIN_STRIDE * b->lin_rows : 0;
}

// The packed row width 1 + K when every problem of the batch has K shared
// polynomials, else 0.
static int packed_row_width(const pcba_batch* b) {
  if (!b || !b->lin || b->desc.empty()) return 0;
  const int K = b->desc[0].alpha;
  for (const ProbDesc& d : b->desc)
    if (d.alpha != K) return 0;
  return 1 + K;
}

long long pcba_batch_rows_packed_doubles(const pcba_batch* b) {
  return (long long)packed_row_width(b) * (b ? b->lin_rows : 0);
}

int pcba_batch_upload_rows_packed(pcba_batch* b, const double* host_rows) {
  if (!b || !host_rows) return fail(PCBA_ERR_INVALID, "batch or host_rows is null");
  if (!b->lin) return fail(PCBA_ERR_INVALID, "the batch has no linear-family constraints");
  const int w = packed_row_width(b);
  if (w == 0) return fail(PCBA_ERR_INVALID, "packed rows need the same K in every problem");
  const long long n = (long long)w * b->lin_rows;
  if (n == 0) return 0;
  // staged in the FP32 row table (64 bytes per row, w <= 5 doubles), which
  // the conversion below then rewrites
  double* stage = reinterpret_cast<double*>(b->d_lin32);
  PCBA_CK(cudaMemcpyAsync(stage, host_rows, sizeof(double) * n, cudaMemcpyHostToDevice,
                          b->stream));
  const long long m = (long long)PCBA_LIN_STRIDE * b->lin_rows;
  const unsigned g = (unsigned)std::min<long long>((m + 255) / 256, 4LL * b->g.sms);
  k_rows_unpack<<<g, 256, 0, b->stream>>>(stage, b->d_lin64, b->lin_rows, w);
  k_rows32<<<g, 256, 0, b->stream>>>(b->d_lin64, b->d_lin32, b->lin_rows);
  PCBA_CK(cudaGetLastError());
  b->pending_h2d += 8LL * n;
  b->extra_launches_pending += 2;
  return 0;
}

void* pcba_host_alloc(size_t bytes) {
  if (bytes == 0) {
    fail(PCBA_ERR_INVALID, "bytes must be > 0");
    return nullptr;
  }
  void* p = nullptr;
  const cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    fail(PCBA_ERR_CUDA, std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
    return nullptr;
  }
  return p;
}

int pcba_host_free(void* p) {
  if (!p) return 0;
  PCBA_CK(cudaFreeHost(p));
  return 0;
}

int pcba_batch_warm_point(const pcba_batch* b, int k, double* x, double* cost) {
  if (!b || k < 0 || k >= b->np) return fail(PCBA_ERR_INVALID, "bad batch or index");
  const ProbState& S = b->h_state[k];
  if (!S.seeded) return 0;
  if (x)
    for (int q = 0; q < b->desc[k].l; ++q) x[q] = S.seed_x[q];
  if (cost) *cost = S.seed_cost;
  return 1;
}

int pcba_batch_cost_grid(pcba_batch* b, int G, float* d_out, int ld, int col0) {
  if (!b || !d_out) return fail(PCBA_ERR_INVALID, "batch or output is null");
  if (G < 2 || G > 32) return fail(PCBA_ERR_INVALID, "G must be in [2, 32]");
  if (col0 < 0 || ld < col0 + G * G) return fail(PCBA_ERR_INVALID, "need ld >= col0 + G * G");
  k_cost_grid<<<b->np, PCBA_TPB, 0, b->stream>>>(b->E, G, d_out, ld, col0);
  PCBA_CK(cudaGetLastError());
  return 0;
}

int pcba_eval_points_f32(const float* d_coeff, int nvars, const int* degree,
                         const float* d_points, int n_points, int unrolled, float* d_val,
                         float* d_err, void* stream) {
  if (!d_coeff || !degree || !d_val || !d_err || (n_points > 0 && !d_points))
    return fail(PCBA_ERR_INVALID, "point evaluation: null argument");
  if (nvars < 1 || nvars > PCBA_MAX_DIM || n_points < 0)
    return fail(PCBA_ERR_INVALID, "point evaluation: nvars must be 1..8 and n_points >= 0");
  PointPoly q;
  std::memset(&q, 0, sizeof(q));
  q.l = nvars;
  long long C = 1;
  for (int r = 0; r < nvars; ++r) {
    if (degree[r] < 0 || degree[r] > PCBA_MAX_DEGREE)
      return fail(PCBA_ERR_INVALID, "point evaluation: degree out of range");
    q.deg[r] = degree[r];
    C *= degree[r] + 1;
  }
  if (C > PCBA_MAX_PATCH) return fail(PCBA_ERR_INVALID, "point evaluation: patch too large");
  if (n_points == 0) return 0;
  k_eval_points_f32<<<(n_points + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      d_coeff, q, d_points, n_points, unrolled ? 1 : 0, d_val, d_err);
  PCBA_CK(cudaGetLastError());
  return 0;
}

int pcba_batch_polish(pcba_batch* b, double mu0, double gap, double eq_tol, int iters,
                      double* x) {
  if (!b || !x) return fail(PCBA_ERR_INVALID, "batch or output is null");
  if (!b->d_polish && cudaMalloc((void**)&b->d_polish, sizeof(double) * PCBA_MAXD * b->np) !=
                          cudaSuccess) {
    b->d_polish = nullptr;
    return fail(PCBA_ERR_OOM, "cannot allocate the polish output");
  }
  int launches = 0;
  const int rc = launch_polish(b, b->d_polish, mu0, gap, eq_tol, iters, &launches);
  if (rc) return rc;
  PCBA_CK(cudaMemcpyAsync(x, b->d_polish, sizeof(double) * PCBA_MAXD * b->np,
                          cudaMemcpyDeviceToHost, b->stream));
  PCBA_CK(cudaStreamSynchronize(b->stream));
  return 0;
}

int pcba_batch_solve_polished(pcba_batch* b, double opt_tol, double eq_tol, double relax_opt_tol,
                              double relax_eq_tol, int max_iters, pcba_result* out) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (!(eq_tol > 0) || !(relax_eq_tol >= eq_tol))
    return fail(PCBA_ERR_INVALID, "need 0 < eq_tol <= relax_eq_tol");
  if (!(opt_tol > 0) || !(relax_opt_tol > 0))
    return fail(PCBA_ERR_INVALID, "tolerances must be > 0");
  if (!b->ev_pipe && cudaEventCreate(&b->ev_pipe) != cudaSuccess) {
    b->ev_pipe = nullptr;
    return fail(PCBA_ERR_CUDA, "event creation failed");
  }
  PCBA_CK(cudaEventRecord(b->ev_pipe, b->stream));
  int rc = batch_solve_impl(b, nullptr, relax_opt_tol, relax_eq_tol, max_iters, 0, nullptr,
                            nullptr);
  if (rc) return rc;
  long long l1 = 0, h1 = 0, d1 = 0;
  pcba_batch_stats(b, nullptr, &l1, &h1, &d1);
  const unsigned long long t0 = b->h_plan->t0;
  int lp = 0;
  rc = launch_polish(b, b->d_warm, kPolishMu0, 0.1 * opt_tol, eq_tol, kPolishIters, &lp);
  if (rc) return rc;
  b->warm_on_device = true;
  rc = batch_solve_impl(b, nullptr, opt_tol, eq_tol, max_iters, 0, nullptr, nullptr);
  b->warm_on_device = false;
  if (rc) return rc;
  b->prior_launches = l1 + lp;
  b->prior_h2d = h1;
  b->prior_d2h = d1;
  float ms = 0;
  PCBA_CK(cudaEventElapsedTime(&ms, b->ev_pipe, b->ev1));
  b->total_ms = ms;
  b->h_plan->t0 = t0;  // per-problem times count from the start of the first solve
  if (out) fill_results(b, out);
  return 0;
}

long long pcba_batch_input_doubles(const pcba_batch* b) { return b ? b->mono_doubles : 0; }

int pcba_batch_trace(const pcba_batch* b, int k, double* rows, int max_rows) {
  if (!b || k < 0 || k >= b->np || !rows) return fail(PCBA_ERR_INVALID, "bad trace request");
  const int steps = std::min(b->h_state[k].steps, b->desc[k].trace_rows);
  const int nrow = std::min(steps, max_rows);
  if (nrow <= 0) return 0;
  PCBA_CK(cudaMemcpy(rows, b->d_trace + b->desc[k].trace_off * 4, sizeof(double) * 4 * nrow,
                     cudaMemcpyDeviceToHost));
  return nrow;
}

int pcba_batch_timing(const pcba_batch* b, double* total_ms, double* subdiv_ms,
                      double* subdiv_bytes, long long* subdiv_launches) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (total_ms) *total_ms = b->total_ms;
  if (subdiv_ms) *subdiv_ms = b->subdiv_ms;
  if (subdiv_bytes) *subdiv_bytes = b->subdiv_bytes;
  if (subdiv_launches) *subdiv_launches = b->subdiv_launches;
  return 0;
}

int pcba_batch_autotune(pcba_batch* b, double opt_tol, double eq_tol, int max_iters,
                        double* ms_per_config, int max_configs, int* chosen) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  const int ncfg = (int)b->g.k2.cfgs.size();
  double best = 1e300;
  int best_i = b->g.cfg;
  for (int i = 0; i < ncfg; ++i) {
    if (b->g.k2.cfgs[i].tma && !b->want_tma) continue;
    int rc = apply_k2_config(b, i);
    if (!rc) rc = rebuild_graph(b);
    if (!rc) rc = batch_solve_impl(b, nullptr, opt_tol, eq_tol, max_iters, 0, nullptr, nullptr);
    if (!rc) rc = batch_solve_impl(b, nullptr, opt_tol, eq_tol, max_iters, 0, nullptr, nullptr);
    if (rc) return rc;
    if (ms_per_config && i < max_configs) ms_per_config[i] = b->total_ms;
    if (b->total_ms < best) {
      best = b->total_ms;
      best_i = i;
    }
  }
  int rc = apply_k2_config(b, best_i);
  if (!rc) rc = rebuild_graph(b);
  if (rc) return rc;
  if (chosen) *chosen = best_i;
  return ncfg;
}

int pcba_batch_config(const pcba_batch* b, int* tma, int* warps_per_block, int* stages,
                      int* grid) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  const K2Cfg& c = b->g.k2.cfgs[b->g.cfg];
  if (tma) *tma = c.tma ? 1 : 0;
  if (warps_per_block) *warps_per_block = c.wpb;
  if (stages) *stages = c.stages;
  if (grid) *grid = c.grid;
  return b->g.cfg;
}

int pcba_batch_launch_bytes(const pcba_batch* b, double* bytes, int max_launches) {
  if (!b || !bytes || max_launches < 0) return fail(PCBA_ERR_INVALID, "bad launch-bytes request");
  const int n = std::min<int>(max_launches, (int)b->launch_bytes.size());
  for (int q = 0; q < n; ++q) bytes[q] = b->launch_bytes[q];
  return n;
}

int pcba_batch_stats(const pcba_batch* b, long long* loop_iters, long long* kernel_launches,
                     long long* h2d_bytes, long long* d2h_bytes) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  const long long it = b->h_plan ? b->h_plan->steps_global : 0;
  if (loop_iters) *loop_iters = it;
  // prologue: k1_matrices, k1_convert, k_eval, k_init (plus the warm-start
  // kernels); epilogue: k_eval
  // per iteration: subdivision, k_pup, k3_classify, k4_index, k_move_control,
  // and k_refresh in FP32
  const long long per_it = 5 + (b->precision == PCBA_FP32 ? 1 : 0) + (b->lin ? 1 : 0);
  // the graph runs iterations in pairs: an odd count adds one empty iteration
  const long long it_run = (b->flags & 3) == 0 ? it + (it & 1) : it;
  if (kernel_launches) *kernel_launches = 5 + per_it * it_run + b->extra_launches + b->prior_launches;
  if (h2d_bytes) *h2d_bytes = b->h2d_bytes + b->prior_h2d;
  if (d2h_bytes) *d2h_bytes = b->d2h_bytes + b->prior_d2h;
  return 0;
}

int pcba_batch_refresh_stats(const pcba_batch* b, long long* marked, long long* refreshed) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (marked) *marked = (long long)b->h_plan->marks_total;
  if (refreshed) *refreshed = (long long)b->h_plan->refreshed_total;
  return 0;
}

int pcba_batch_linear_stats(const pcba_batch* b, long long* pairs, long long* full,
                            long long* coeffs) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (pairs) *pairs = (long long)b->h_plan->lin_pairs;
  if (full) *full = (long long)b->h_plan->lin_full;
  if (coeffs) *coeffs = b->lin ? (long long)b->desc[0].cg : 0;
  return 0;
}

int pcba_batch_set_stream(pcba_batch* b, void* stream) {
  if (!b) return fail(PCBA_ERR_INVALID, "batch is null");
  if (b->own_stream && b->stream) {
    PCBA_CK(cudaStreamSynchronize(b->stream));
    cudaStreamDestroy(b->stream);
    b->own_stream = false;
  }
  b->stream = (cudaStream_t)stream;
  return 0;
}

void pcba_batch_destroy(pcba_batch* b) { free_batch(b); }

int pcba_solve_batch(pcba_handle** hs, int n, double opt_tol, double eq_tol, int max_iters,
                     size_t mem_cap_total, const double* warm_start, pcba_result* out) {
  pcba_batch* b = nullptr;
  int rc = batch_create_impl(&b, hs, n, mem_cap_total, 0);
  if (rc) return rc;
  rc = batch_solve_impl(b, nullptr, opt_tol, eq_tol, max_iters, 0, warm_start, out);
  free_batch(b);
  return rc;
}

int pcba_get_list(pcba_handle* h, long long* K_out, double* cost, double* ineq, double* eq,
                  float* err, unsigned* index, int* level) {
  if (!h || !h->own) return fail(PCBA_ERR_INVALID, "no solve has run on this handle");
  pcba_batch* b = h->own;
  const ProbState& S = b->h_state[0];
  const ProbDesc& d = b->desc[0];
  const long long K = S.K;
  if (K_out) *K_out = K;
  if (level)
    for (int q = 0; q < d.l; ++q) level[q] = S.level[q];
  if (!cost && !ineq && !eq && !err && !index) return 0;
  std::vector<char> buf((size_t)(K * d.item_bytes));
  std::vector<unsigned> slot((size_t)std::max<long long>(K, 1));
  const long long nslots_total = b->nslots_total;
  PCBA_CK(cudaMemcpy(slot.data(), b->d_slots + 3 * nslots_total + d.slot_off,
                     sizeof(unsigned) * (size_t)K, cudaMemcpyDeviceToHost));
  for (long long k = 0; k < K; ++k)
    PCBA_CK(cudaMemcpy(buf.data() + k * d.item_bytes,
                       b->d_arena + d.list_off + (size_t)slot[(size_t)k] * d.item_bytes,
                       (size_t)d.item_bytes, cudaMemcpyDeviceToHost));
  const bool f32 = b->precision == PCBA_FP32;
  const int nerr = 1 + d.alpha + d.beta;
  // linear families: the copy of the shared patches the next step would read
  const int cpy = b->h_plan->steps_global & 1;
  const long long off_g = d.off_g + cpy * d.copy_g, off_eg = d.off_eg + cpy * d.copy_e;
  for (long long k = 0; k < K; ++k) {
    const char* it = buf.data() + k * d.item_bytes;
    if (index)
      for (int q = 0; q < d.l; ++q) index[k * d.l + q] = ((const unsigned*)it)[q];
    const double O = f32 ? *(const double*)(it + 32) : 0.0;
    auto val = [&](long long off, long long e) -> double {
      return f32 ? (double)((const float*)(it + off))[e] : ((const double*)(it + off))[e];
    };
    if (cost)
      for (int j = 0; j < d.cp; ++j) cost[k * d.cp + j] = f32 ? O + val(d.off_cost, j) : val(d.off_cost, j);
    if (ineq)
      for (int i = 0; i < d.alpha; ++i) {
        // FP32 patches are stored relative to an offset (linear families:
        // FP64, dense families: FP32)
        const double Oi = !f32 ? 0.0
                          : d.lin ? ((const double*)(it + off_eg + 4LL * d.apad))[i]
                                  : (double)((const float*)(it + d.off_og))[i];
        for (int j = 0; j < d.cg; ++j)
          ineq[(k * d.alpha + i) * d.cg + j] = Oi + val(off_g, (long long)j * d.apad + i);
      }
    if (eq)
      for (int i = 0; i < d.beta; ++i) {
        const double Oh = f32 && !d.lin ? (double)((const float*)(it + d.off_oh))[i] : 0.0;
        for (int j = 0; j < d.ch; ++j)
          eq[(k * d.beta + i) * d.ch + j] = Oh + val(d.off_h, (long long)j * d.bpad + i);
      }
    if (err) {
      float* e = err + k * nerr;
      if (f32) {
        e[0] = *(const float*)(it + 40);
        // the sign bit marks refresh candidates; the bound is the magnitude
        for (int i = 0; i < d.alpha; ++i) e[1 + i] = std::fabs(((const float*)(it + off_eg))[i]);
        for (int i = 0; i < d.beta; ++i)
          e[1 + d.alpha + i] = std::fabs(((const float*)(it + d.off_eh))[i]);
      } else {
        for (int i = 0; i < nerr; ++i) e[i] = 0.0f;
      }
    }
  }
  return 0;
}

int pcba_root_patches(pcba_handle* h, double* cost, double* ineq, double* eq) {
  if (!h) return fail(PCBA_ERR_INVALID, "handle is null");
  pcba_batch* b = nullptr;
  const size_t cap = h->own ? h->own_cap : (size_t)pcba_item_bytes(h) * 4;
  int rc = own_batch(h, cap, &b);
  if (rc) return rc;
  rc = batch_solve_impl(b, nullptr, 1.0, 1.0, 2, 1, nullptr, nullptr, true);
  if (rc) return rc;
  const HostProblem& P = h->prob;
  std::vector<double> raw((size_t)b->mono_doubles);
  PCBA_CK(cudaMemcpy(raw.data(), b->d_raw, sizeof(double) * raw.size(), cudaMemcpyDeviceToHost));
  if (cost) std::copy(raw.begin(), raw.begin() + P.cp, cost);
  if (ineq) std::copy(raw.begin() + P.cp, raw.begin() + P.cp + P.alpha * P.cg, ineq);
  if (eq)
    std::copy(raw.begin() + P.cp + P.alpha * P.cg,
              raw.begin() + P.cp + P.alpha * P.cg + P.beta * P.ch, eq);
  return 0;
}

}  // extern "C"
