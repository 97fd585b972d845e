// FP64-basis grid-engine kernels with one 512-thread block per SM (the other kernels use 256-thread blocks,
// two per SM).  Same source; its own namespace keeps the two block sizes apart.
#define KIOPS_THREADS 512
#define KIOPS_DEV_NS kiops_dev_wide
#include "kiops_device.cuh"
#include "kiops_kernels.h"

using namespace kiops_dev_wide;

namespace kiops_k {
void* solve_kernel_f64_wide(int kind) {
  if (kind == OP_CSR) return (void*)kiops_solve_kernel<double, OP_CSR, true>;
  if (kind == OP_ST2D) return (void*)kiops_solve_kernel<double, OP_ST2D, true>;
  return (void*)kiops_solve_kernel<double, OP_ST3D, true>;
}
int wide_threads() { return kThreads; }
}  // namespace kiops_k
