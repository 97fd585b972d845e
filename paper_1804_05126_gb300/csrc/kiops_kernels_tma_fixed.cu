// The grid-engine kernel for 2D stencils with the bulk-tensor-copy several-tiles path compiled for one
// configuration: 32 x 16 tiles, two species, p = 3, FP32 basis (loop bounds, shared-memory offsets and the
// B-block loop are constants; ragged edge tiles run the whole box and mask what lies beyond the grid).
#include "kiops_device.cuh"
#include "kiops_kernels.h"

using namespace kiops_dev;

namespace kiops_k {
void* solve_kernel_tma_fixed() { return (void*)kiops_solve_kernel<float, OP_ST2D, true, kTmaFixed>; }
// 3D stencils, FP32 basis: the staged 3D tile path compiled for 32 x 8 x 4 tiles
void* solve_kernel_tma3d_fixed() { return (void*)kiops_solve_kernel<float, OP_ST3D, true, kTmaFixed>; }
}  // namespace kiops_k
