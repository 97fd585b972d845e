// Persistent serving kernel instantiation (dispatches on every operator kind and precision).
#include "kiops_device.cuh"
#include "kiops_kernels.h"

namespace kiops_k {
void* server_kernel() { return (void*)kiops_dev::kiops_server_kernel<0>; }
}  // namespace kiops_k
