// The subdivision kernels of libpcba (Alg. 2 + Alg. 3) and their launcher,
// compiled once per arithmetic: PCBA_K2_F64 = 0 builds the FP32 instances,
// 1 the FP64 ones (see pcba_host.h).  The kernels themselves are in
// pcba_subdivide.cuh (dense problems, direct or TMA-staged loads) and
// pcba_linear.cuh (linear-family problems).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <string>

#include "pcba.h"
#include "pcba_host.h"
#include "pcba_subdivide.cuh"
#include "pcba_linear.cuh"

// 1: the linear-family kernels are launched as dependent steps
#ifndef PCBA_PDL_K2
#define PCBA_PDL_K2 1
#endif
#ifndef PCBA_K2_F64
#define PCBA_K2_F64 0
#endif

namespace {

#if PCBA_K2_F64
using T = double;
#else
using T = float;
#endif

#define K2_CK(call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return pcba_internal_fail(PCBA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// The TMA subdivision kernel instance for a degree class / fixed degree.
const void* tma_kernel(int nmax, int nfix) {
  if (nfix == 6) return (const void*)k2_subdivide_tma<T, 8, 6>;
  if (nfix == 4) return (const void*)k2_subdivide_tma<T, 4, 4>;
  if (nmax <= 4) return (const void*)k2_subdivide_tma<T, 4>;
  if (nmax <= 8) return (const void*)k2_subdivide_tma<T, 8>;
  return (const void*)k2_subdivide_tma<T, 16>;
}

const void* direct_kernel(int nmax) {
  if (nmax <= 4) return (const void*)k2_subdivide<T, 4>;
  if (nmax <= 8) return (const void*)k2_subdivide<T, 8>;
  return (const void*)k2_subdivide<T, 16>;
}

// The linear-family kernels for K shared patches: the split (a thread per
// item) and the bound (a warp per item chunk).  K = 3 with every patch of
// degree 6 on every axis - the obstacle constraints of degree-(3,3) maps - has
// a fixed-degree split.
const void* lin_split_kernel(int K, int nfix) {
  if (K == 3 && nfix == 6) return (const void*)k2_lin_split<T, 3, 6>;
  switch (K) {
    case 1: return (const void*)k2_lin_split<T, 1, 0>;
    case 2: return (const void*)k2_lin_split<T, 2, 0>;
    case 3: return (const void*)k2_lin_split<T, 3, 0>;
    default: return (const void*)k2_lin_split<T, 4, 0>;
  }
}
const void* lin_bound_kernel(int K) {
  switch (K) {
    case 1: return (const void*)k2_lin_bound<T, 1>;
    case 2: return (const void*)k2_lin_bound<T, 2>;
    case 3: return (const void*)k2_lin_bound<T, 3>;
    default: return (const void*)k2_lin_bound<T, 4>;
  }
}

int prepare(K2Plan& g, const std::vector<ProbDesc>& desc, bool lin, int sms, int smem_optin) {
  long long cpmax = 1;
  for (const ProbDesc& d : desc) cpmax = std::max<long long>(cpmax, d.cp);
  // kernel variant by the largest degree
  int dmax = 0;
  for (const ProbDesc& d : desc)
    for (int r = 0; r < d.l; ++r) dmax = std::max(dmax, std::max(d.P[r], std::max(d.G[r], d.H[r])));
  g.nmax = dmax <= 4 ? 4 : (dmax <= 8 ? 8 : 16);
  {
    // a single degree on every axis of every patch of the batch: fixed-degree kernel
    int fixed = -1;
    bool uniform = true;
    auto see = [&](int n) {
      if (fixed < 0) fixed = n;
      else if (fixed != n) uniform = false;
    };
    for (const ProbDesc& d : desc)
      for (int r = 0; r < d.l; ++r) {
        see(d.P[r]);
        if (d.alpha > 0) see(d.G[r]);
        if (d.beta > 0) see(d.H[r]);
      }
    g.nfix = (uniform && (fixed == 4 || fixed == 6) && !std::getenv("PCBA_NO_FIXED_DEGREE"))
                 ? fixed : 0;
  }
  int occ = 0;
  g.cfgs.clear();
  if (lin) {
    // linear families: the split and bound kernels, no TMA staging
    g.lin_k = desc[0].alpha;
    g.lin_cpmax = (int)cpmax;
    g.lin_cgmax = 1;
    for (const ProbDesc& d : desc) g.lin_cgmax = std::max(g.lin_cgmax, d.cg);
    const size_t ws = lin_split_warp_bytes<T>(g.lin_cgmax, g.lin_cpmax);
    const size_t wbnd = lin_bound_warp_bytes<T>(g.lin_cgmax);
    if (8 * ws > (size_t)smem_optin || 8 * wbnd > (size_t)smem_optin)
      return pcba_internal_fail(PCBA_ERR_INVALID, "shared patches too large");
    const void* ks = lin_split_kernel(g.lin_k, g.nfix);
    K2_CK(cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * ws)));
    K2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ks, 256, 8 * ws));
    g.lin_split_grid = std::max(1, occ) * sms;
    g.lin_split_smem = 8 * ws;
    const void* kb = lin_bound_kernel(g.lin_k);
    K2_CK(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * wbnd)));
    K2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb, 256, 8 * wbnd));
    g.cfgs.push_back({false, 8, 1, 8 * wbnd, std::max(1, occ) * sms});
    return 0;
  }
  g.lin_k = 0;
  const size_t k2_smem = (size_t)(2 * cpmax) * sizeof(T);
  const void* k2 = direct_kernel(g.nmax);
  K2_CK(cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max<size_t>(k2_smem, 1)));
  K2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k2, PCBA_TPB, k2_smem));
  g.cfgs.push_back({false, 8, 1, k2_smem, std::max(1, occ) * sms});
  // TMA-staged configurations: per warp 'stages' copies of a [C][32] column
  // block (C <= 256, the TMA box limit)
  long long cstage = 1;
  bool fits = true;
  for (const ProbDesc& d : desc) {
    if (d.alpha > 0) cstage = std::max<long long>(cstage, d.cg);
    if (d.beta > 0) cstage = std::max<long long>(cstage, d.ch);
    if ((d.alpha > 0 && d.cg > 256) || (d.beta > 0 && d.ch > 256)) fits = false;
  }
  g.tma_stage_elems = (int)(cstage * 32);
  g.tma_cpmax = (int)cpmax;
  const size_t head_cap = ((size_t)64 + (size_t)cpmax * sizeof(T) + 32 + 127) / 128 * 128;
  const size_t stage_bytes = (size_t)g.tma_stage_elems * sizeof(T) + PCBA_ESTAGE_BYTES + head_cap;
  const int cand[][2] = {{8, 2}, {8, 3}, {4, 2}, {4, 3}, {2, 2}};
  const void* kt = tma_kernel(g.nmax, g.nfix);
  size_t smem_max = 0;
  for (const auto& c : cand) {
    const size_t wb = ((size_t)c[1] * stage_bytes + 2 * (size_t)cpmax * sizeof(T) + 127) / 128 * 128;
    const size_t total = (size_t)c[0] * wb + (size_t)c[0] * c[1] * 8;
    if (fits && total <= (size_t)smem_optin) {
      g.cfgs.push_back({true, c[0], c[1], total, 0});
      smem_max = std::max(smem_max, total);
    }
  }
  if (g.cfgs.size() > 1) {
    K2_CK(cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    for (auto& c : g.cfgs) {
      if (!c.tma) continue;
      K2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kt, 32 * c.wpb, c.smem));
      c.grid = std::max(1, occ) * sms;
    }
  }
  return 0;
}

void launch(const K2Plan& g, int cfg, const Engine& E, cudaStream_t s) {
  const K2Cfg& c = g.cfgs[cfg];
  const dim3 blk(32 * c.wpb);
  if (g.lin_k > 0) {
    // the split writes the children, then the bound reads them
    const int gs = g.lin_split_grid, cg = g.lin_cgmax, cp = g.lin_cpmax;
    const size_t ss = g.lin_split_smem;
    // (both begin with pdl_begin: launched as dependent steps)
    auto split = g.lin_k == 3 && g.nfix == 6 ? k2_lin_split<T, 3, 6>
                 : g.lin_k == 1             ? k2_lin_split<T, 1, 0>
                 : g.lin_k == 2             ? k2_lin_split<T, 2, 0>
                 : g.lin_k == 3             ? k2_lin_split<T, 3, 0>
                                            : k2_lin_split<T, 4, 0>;
    auto bound = g.lin_k == 1 ? k2_lin_bound<T, 1>
                 : g.lin_k == 2 ? k2_lin_bound<T, 2>
                 : g.lin_k == 3 ? k2_lin_bound<T, 3>
                                : k2_lin_bound<T, 4>;
    pcba_launch_step(PCBA_PDL_K2, split, gs, 256, ss, s, E, cg, cp);
    pcba_launch_step(PCBA_PDL_K2, bound, c.grid, blk, c.smem, s, E, cg);
    return;
  }
  if (c.tma) {
    const int st = c.stages, se = g.tma_stage_elems, cp = g.tma_cpmax;
    if (g.nfix == 6)
      k2_subdivide_tma<T, 8, 6><<<c.grid, blk, c.smem, s>>>(E, st, se, cp);
    else if (g.nfix == 4)
      k2_subdivide_tma<T, 4, 4><<<c.grid, blk, c.smem, s>>>(E, st, se, cp);
    else if (g.nmax <= 4)
      k2_subdivide_tma<T, 4><<<c.grid, blk, c.smem, s>>>(E, st, se, cp);
    else if (g.nmax <= 8)
      k2_subdivide_tma<T, 8><<<c.grid, blk, c.smem, s>>>(E, st, se, cp);
    else
      k2_subdivide_tma<T, 16><<<c.grid, blk, c.smem, s>>>(E, st, se, cp);
    return;
  }
  if (g.nmax <= 4) k2_subdivide<T, 4><<<c.grid, PCBA_TPB, c.smem, s>>>(E);
  else if (g.nmax <= 8) k2_subdivide<T, 8><<<c.grid, PCBA_TPB, c.smem, s>>>(E);
  else k2_subdivide<T, 16><<<c.grid, PCBA_TPB, c.smem, s>>>(E);
}

}  // namespace

#if PCBA_K2_F64
int pcba_k2_prepare_f64(K2Plan& g, const std::vector<ProbDesc>& desc, bool lin, int sms,
                        int smem_optin) {
  return prepare(g, desc, lin, sms, smem_optin);
}
void pcba_k2_launch_f64(const K2Plan& g, int cfg, const Engine& E, cudaStream_t s) {
  launch(g, cfg, E, s);
}
#else
int pcba_k2_prepare_f32(K2Plan& g, const std::vector<ProbDesc>& desc, bool lin, int sms,
                        int smem_optin) {
  return prepare(g, desc, lin, sms, smem_optin);
}
void pcba_k2_launch_f32(const K2Plan& g, int cfg, const Engine& E, cudaStream_t s) {
  launch(g, cfg, E, s);
}
#endif
