// Host-side interface between the translation units of libpcba.
//
// The subdivision kernels (pcba_k2.cu, built once for FP32 and once for FP64)
// and the polish kernel (pcba_polish.cu) are compiled on their own, in
// parallel with the engine (pcba.cu); a kernel can only be launched from the
// unit that defines it, so each unit exports plain host functions that pick
// a kernel instance, set its attributes and launch it.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <string>
#include <vector>

#include "pcba_device.cuh"

// error reporting of the library (defined in pcba.cu)
int pcba_internal_fail(int code, const std::string& msg);

// One configuration of the subdivision kernel: TMA staging or not, warps per
// block, pipeline stages per warp, dynamic shared memory and grid size.
struct K2Cfg {
  bool tma;
  int wpb, stages;
  size_t smem;
  int grid;
};

// Everything the subdivision launcher needs about a batch.
struct K2Plan {
  int lin_k = 0;                     // linear families: shared patches per item (0: dense)
  int lin_cgmax = 1, lin_cpmax = 1;  // largest shared / cost patch of the batch
  int lin_split_grid = 1;            // blocks of the linear split kernel (256 threads)
  size_t lin_split_smem = 0;         // its dynamic shared memory
  int nmax = 16;  // degree class of the dense kernels (4, 8 or 16)
  int nfix = 0;   // every patch of the batch has this degree on every axis (4 or 6), else 0
  int tma_stage_elems = 0, tma_cpmax = 1;
  std::vector<K2Cfg> cfgs;  // index 0: direct loads (or the linear kernel), then TMA
};

// Fills the plan for the batch's problems (kernel variant, feasible
// configurations with their occupancy-sized grids); 0 or a PCBA_ERR_* code.
// Launches one of the per-step kernels (those that begin with pdl_begin),
// with programmatic stream serialization when pdl is set: it is scheduled
// as its predecessor in the stream finishes, and waits for it itself.  The
// environment variable PCBA_NO_PDL turns this off (plain launches).
template <typename... P, typename... A>
inline cudaError_t pcba_launch_step(bool pdl, void (*k)(P...), dim3 grid, dim3 block,
                                    size_t smem, cudaStream_t s, A... args) {
  static const bool no_pdl = std::getenv("PCBA_NO_PDL") != nullptr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = no_pdl || !pdl ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);
}

int pcba_k2_prepare_f32(K2Plan& g, const std::vector<ProbDesc>& desc, bool lin, int sms,
                        int smem_optin);
int pcba_k2_prepare_f64(K2Plan& g, const std::vector<ProbDesc>& desc, bool lin, int sms,
                        int smem_optin);
// Queues one subdivision launch (configuration cfg) on the stream.
void pcba_k2_launch_f32(const K2Plan& g, int cfg, const Engine& E, cudaStream_t s);
void pcba_k2_launch_f64(const K2Plan& g, int cfg, const Engine& E, cudaStream_t s);

// Queues k_polish<L> over grid problems (pcba_polish.cuh); 0 or a PCBA_ERR_* code.
int pcba_polish_launch(const Engine& E, int L, unsigned grid, cudaStream_t s, double* out,
                       double mu0, double gap, double eq_tol, int iters);
