// Measurement kernel: the FP64 FMA throughput of the GPU the library runs on, the peak the solver's
// FP64-bound phases are reported against (the paper has no counterpart).  Every thread runs CHAINS
// independent chains of dependent FP64 fused multiply-adds, so that the FP64 pipe, not the dependent
// latency, bounds the rate; the grid holds several blocks per SM on every SM.  The host takes the best of a
// few shapes (chains per thread, blocks per SM).
#include "kiops_kernels.h"

#include <cuda_runtime.h>

namespace {

constexpr int kProbeThreads = 256;

template <int CHAINS>
__global__ void __launch_bounds__(kProbeThreads) fp64_fma_kernel(int iters, double a, double b, double* out) {
  double x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  out[blockIdx.x * (size_t)kProbeThreads + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

namespace kiops_k {

int probe_threads() { return kProbeThreads; }

double probe_flops_per_thread(int chains, int iters) { return 2.0 * chains * (double)iters; }

cudaError_t launch_fp64_probe(int chains, int blocks, int iters, double* out, cudaStream_t st) {
  if (chains == 16) fp64_fma_kernel<16><<<blocks, kProbeThreads, 0, st>>>(iters, 0.9999999, 1e-7, out);
  else fp64_fma_kernel<8><<<blocks, kProbeThreads, 0, st>>>(iters, 0.9999999, 1e-7, out);
  return cudaGetLastError();
}

}  // namespace kiops_k
