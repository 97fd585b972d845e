// Instantiations of the grid-engine kernel with the bulk-tensor-copy (TMA) several-tiles paths (2D stencils in
// either precision, 3D stencils with an FP32 basis), in their own translation unit (compiled in parallel with
// the others).
#include "kiops_device.cuh"
#include "kiops_kernels.h"

using namespace kiops_dev;

namespace kiops_k {
void* solve_kernel_tma(bool fp32) {
  if (fp32) return (void*)kiops_solve_kernel<float, OP_ST2D, true, kTmaGeneral>;
  return (void*)kiops_solve_kernel<double, OP_ST2D, true, kTmaGeneral>;
}
void* solve_kernel_tma3d() { return (void*)kiops_solve_kernel<float, OP_ST3D, true, kTmaGeneral>; }
}  // namespace kiops_k
