// pcba_bernstein_convert_noalloc: monomial-to-Bernstein conversion that makes
// no device allocation (see include/pcba.h).
//
// The regular conversion (pcba_create / pcba_root_patches) keeps its per-axis
// transform matrices in a buffer the library allocates.  Here they live in a
// fixed file-scope device array instead, so the call only needs the caller's
// input and output buffers.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "pcba.h"

// set by this file's entry point; defined in pcba.cu
int pcba_internal_fail(int code, const std::string& msg);

namespace {

constexpr int kMaxDeg1 = PCBA_MAX_DEGREE + 1;   // 17 coefficients per fibre at most
constexpr int kMatDoubles = kMaxDeg1 * kMaxDeg1;  // one (d+1)^2 matrix
// One transform matrix T_r per axis.
constexpr int kScratchDoubles = PCBA_MAX_DIM * kMatDoubles;

// The scratch of every call on this device (18.5 KB).  Host code must not pass
// this name to a kernel: in host code it is only a stand-in for the symbol.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// The array's device address, per device, together with the unique ID of the
// CUDA context it was looked up in: a module is loaded once per context, so
// after cudaDeviceReset (a new primary context) or in another context of the
// same device the address is looked up again.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  unsigned long long ctx_id;
  double* ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

struct ConvArgs {
  int l;
  int C;
  int n_patches;
  int deg[PCBA_MAX_DIM];
  double lo[PCBA_MAX_DIM], hi[PCBA_MAX_DIM];
};

__device__ double nb_binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  if (k > n - k) k = n - k;
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
  return c;
}

__device__ double nb_pow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// One thread per (axis, row): T_r[i][j] = sum_k C(i,k)/C(n,k) C(j,k) lo^(j-k) w^k
// (power basis on [lo, lo+w] -> Bernstein basis, Sec. II-D, Assumption 1).
__global__ void nb_matrices(ConvArgs a, double* scratch) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.l * kMaxDeg1) return;
  const int r = t / kMaxDeg1, i = t % kMaxDeg1;
  const int n = a.deg[r];
  if (i > n) return;
  const double lo = a.lo[r], w = a.hi[r] - a.lo[r];
  double* T = scratch + (size_t)r * kMatDoubles;
  for (int j = 0; j <= n; ++j) {
    double s = 0.0;
    const int kmax = i < j ? i : j;
    for (int k = 0; k <= kmax; ++k)
      s += nb_binom(i, k) / nb_binom(n, k) * nb_binom(j, k) * nb_pow(lo, j - k) * nb_pow(w, k);
    T[i * (n + 1) + j] = s;
  }
}

// One warp per patch: l mode products in shared memory, then the output.
__global__ void nb_convert(ConvArgs a, const double* scratch, const double* mono, double* out) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31;
  double* sA = sm;
  double* sB = sm + a.C;
  double* sT = sB + a.C;
  for (int pidx = blockIdx.x; pidx < a.n_patches; pidx += gridDim.x) {
    const double* src = mono + (size_t)pidx * a.C;
    for (int j = lane; j < a.C; j += 32) sA[j] = src[j];
    __syncwarp();
    for (int r = 0; r < a.l; ++r) {
      const int n = a.deg[r];
      int stride = 1;
      for (int q = r + 1; q < a.l; ++q) stride *= a.deg[q] + 1;
      const double* T = scratch + (size_t)r * kMatDoubles;
      for (int e = lane; e < (n + 1) * (n + 1); e += 32) sT[e] = T[e];
      __syncwarp();
      const int blk = (n + 1) * stride;
      for (int o = lane; o < a.C; o += 32) {
        const int hp = o / blk;
        const int rem = o - hp * blk;
        const int i = rem / stride;
        const int in = rem - i * stride;
        const double* x = sA + hp * blk + in;
        double s = 0.0;
        for (int j = 0; j <= n; ++j) s = fma(sT[i * (n + 1) + j], x[j * stride], s);
        sB[o] = s;
      }
      __syncwarp();
      double* tmp = sA;
      sA = sB;
      sB = tmp;
    }
    double* dst = out + (size_t)pidx * a.C;
    for (int j = lane; j < a.C; j += 32) dst[j] = sA[j];
    __syncwarp();
  }
}

// Unique ID of the calling thread's current CUDA context (0 if there is none
// yet), through the driver entry points of the runtime (no link to libcuda).
int current_context_id(unsigned long long* id) {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000,
                                                      cudaEnableDefault, &q1);
    cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000,
                                                      cudaEnableDefault, &q2);
    if (e1 != cudaSuccess || e2 != cudaSuccess || !f1 || !f2 ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess)
      return pcba_internal_fail(PCBA_ERR_CUDA, "cuCtxGetCurrent / cuCtxGetId are not available");
    get_current = (PFN_cuCtxGetCurrent_v4000)f1;
    get_id = (PFN_cuCtxGetId_v12000)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS)
    return pcba_internal_fail(PCBA_ERR_CUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS)
    return pcba_internal_fail(PCBA_ERR_CUDA, "cuCtxGetId failed");
  return 0;
}

// Resolves the device address of the scratch array with the device current:
// once per device and CUDA context, cached for the later calls.
int scratch_for_current_device(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return pcba_internal_fail(PCBA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return pcba_internal_fail(PCBA_ERR_INVALID, "device ordinal beyond the supported 64");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc) return rc;
  if (id != 0 && g_scratch[dev].ptr && g_scratch[dev].ctx_id == id) {
    *ptr = g_scratch[dev].ptr;
    return 0;
  }
  // the lookup makes the device's primary context current if none was
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return pcba_internal_fail(PCBA_ERR_CUDA,
                              std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  rc = current_context_id(&id);
  if (rc) return rc;
  g_scratch[dev].ctx_id = id;
  g_scratch[dev].ptr = (double*)p;
  *ptr = (double*)p;
  return 0;
}

}  // namespace

extern "C" int pcba_bernstein_convert_noalloc(const double* d_mono, int n_patches, int nvars,
                                              const int* degree, const double* lo,
                                              const double* hi, double* d_out, void* stream) {
  if (!d_mono || !d_out || !degree || !lo || !hi)
    return pcba_internal_fail(PCBA_ERR_INVALID, "noalloc conversion: null argument");
  if (n_patches < 0) return pcba_internal_fail(PCBA_ERR_INVALID, "noalloc conversion: n_patches < 0");
  if (nvars < 1 || nvars > PCBA_MAX_DIM)
    return pcba_internal_fail(PCBA_ERR_INVALID,
                              "noalloc conversion: nvars must be 1..8 (scratch holds 8 axes)");
  ConvArgs a;
  a.l = nvars;
  a.n_patches = n_patches;
  long long C = 1;
  for (int r = 0; r < PCBA_MAX_DIM; ++r) {
    a.deg[r] = 0;
    a.lo[r] = 0.0;
    a.hi[r] = 1.0;
  }
  for (int r = 0; r < nvars; ++r) {
    if (degree[r] < 0 || degree[r] > PCBA_MAX_DEGREE)
      return pcba_internal_fail(PCBA_ERR_INVALID,
                                "noalloc conversion: degree must be 0..16 (scratch holds 17x17 "
                                "matrices per axis)");
    if (!(lo[r] < hi[r]) || !std::isfinite(lo[r]) || !std::isfinite(hi[r]))
      return pcba_internal_fail(PCBA_ERR_INVALID, "noalloc conversion: need finite lo < hi");
    a.deg[r] = degree[r];
    a.lo[r] = lo[r];
    a.hi[r] = hi[r];
    C *= degree[r] + 1;
  }
  if (C > PCBA_MAX_PATCH)
    return pcba_internal_fail(PCBA_ERR_INVALID, "noalloc conversion: patch larger than 8192");
  a.C = (int)C;
  if (n_patches == 0) return 0;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = (size_t)(2 * C + kMatDoubles) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(nb_convert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess)
    return pcba_internal_fail(PCBA_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  nb_matrices<<<(PCBA_MAX_DIM * kMaxDeg1 + 127) / 128, 128, 0, s>>>(a, scratch);
  const int grid = n_patches < 4096 ? n_patches : 4096;
  nb_convert<<<grid, 32, smem, s>>>(a, scratch, d_mono, d_out);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return pcba_internal_fail(PCBA_ERR_CUDA, std::string("noalloc launch: ") + cudaGetErrorString(e));
  return 0;
}
