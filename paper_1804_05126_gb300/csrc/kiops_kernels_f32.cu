// FP32-basis kernel instantiations.
#include "kiops_device.cuh"
#include "kiops_kernels.h"

using namespace kiops_dev;

namespace kiops_k {
void* solve_kernel_f32(int kind) {
  if (kind == OP_CSR) return (void*)kiops_solve_kernel<float, OP_CSR, true>;
  if (kind == OP_ST2D) return (void*)kiops_solve_kernel<float, OP_ST2D, true>;
  return (void*)kiops_solve_kernel<float, OP_ST3D, true>;
}
void* team_kernel_f32(int kind) {
  if (kind == OP_CSR) return (void*)kiops_team_kernel<float, OP_CSR>;
  if (kind == OP_ST2D) return (void*)kiops_team_kernel<float, OP_ST2D>;
  return (void*)kiops_team_kernel<float, OP_ST3D>;
}
}  // namespace kiops_k
