// The local polish of incumbents (pcba_polish.cuh), compiled on its own: one
// k_polish instance per number of variables, launched through
// pcba_polish_launch (pcba_host.h).
#include <cuda_runtime.h>

#include <string>

#include "pcba.h"
#include "pcba_host.h"
#include "pcba_polish.cuh"

int pcba_polish_launch(const Engine& E, int L, unsigned g, cudaStream_t s, double* out,
                       double mu0, double gap, double eq_tol, int iters) {
  switch (L) {
    case 1: k_polish<1><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
    case 2: k_polish<2><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
    case 3: k_polish<3><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
    case 4: k_polish<4><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
    case 5: k_polish<5><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
    case 6: k_polish<6><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
    case 7: k_polish<7><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
    default: k_polish<8><<<g, PCBA_POLISH_TPB, 0, s>>>(E, out, mu0, gap, eq_tol, iters); break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return pcba_internal_fail(PCBA_ERR_CUDA, std::string("k_polish launch: ") + cudaGetErrorString(e));
  return 0;
}
