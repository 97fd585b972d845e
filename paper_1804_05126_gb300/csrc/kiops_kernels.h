// Entry points of the kernel translation units (each compiled on its own, in parallel).
#pragma once

namespace kiops_k {
void* solve_kernel_f64(int kind);   // grid engine, FP64 basis
void* solve_kernel_f32(int kind);   // grid engine, FP32 basis
void* team_kernel_f64(int kind);    // batch team engine, FP64 basis
void* team_kernel_f32(int kind);    // batch team engine, FP32 basis
void* noalloc_kernel(int kind);     // single block, argument block by value (FP64)
void* server_kernel();              // persistent serving kernel (every kind and precision)
}  // namespace kiops_k
