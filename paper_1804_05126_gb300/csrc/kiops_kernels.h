// Entry points of the kernel translation units (each compiled on its own, in parallel).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kiops_k {
void* solve_kernel_f64(int kind);   // grid engine, FP64 basis
void* solve_kernel_f64_wide(int kind);  // grid engine, FP64 basis, 512-thread blocks (one per SM)
int wide_threads();                 // block size of solve_kernel_f64_wide
void* solve_kernel_f32(int kind);   // grid engine, FP32 basis
void* solve_kernel_tma(bool fp32);  // grid engine, 2D stencils, with the bulk-tensor-copy several-tiles path
void* solve_kernel_tma_fixed();     // the same, FP32, for 32 x 16 tiles, two species and p = 3
void* solve_kernel_tma3d();         // grid engine, 3D stencils, FP32 basis, 3D tiles staged by bulk tensor copies
void* solve_kernel_tma3d_fixed();   // the same compiled for 32 x 8 x 4 tiles
void* team_kernel_f64(int kind);    // batch team engine, FP64 basis
void* team_kernel_f32(int kind);    // batch team engine, FP32 basis
void* noalloc_kernel(int kind);     // single block, argument block by value (FP64)
void* server_kernel();              // persistent serving kernel (every kind and precision)

// Integrators (kiops_integrate.cu).  A test problem of section 4 on an n x n grid.
struct PdeDev {
  int kind;       // 0: 2D ADR (Neumann), 1: 2D Gray-Scott (periodic)
  int ns;         // species
  int bc;         // 1 periodic, 2 Neumann (reflection)
  int64_t n;      // points per dimension
  double dx;      // grid spacing
  double prm[4];  // ADR: eps, alpha, gamma; Gray-Scott: d_u, d_v, a, b
};
// Weights of r2 and r3 in b_3 and b_4: b_k = h (x_k r2 + y_k (r3 + z r2)).
struct SchemeDev {
  double x3, y3, x4, y4, z;
};
cudaError_t launch_pde_eval(const PdeDev& P, const double* u, double h, double* hf, double* const fields[4], int sms,
                            cudaStream_t st);
cudaError_t launch_stages(int64_t N, const double* u, const double* W2, double c2, const double* W3, double c3,
                          double* U2, double* U3, int sms, cudaStream_t st);
cudaError_t launch_remainder(const PdeDev& P, const double* un, const double* U, double h, double* out, int sms,
                             cudaStream_t st);
cudaError_t launch_assemble(const PdeDev& P, const double* un, const double* U2, const double* U3, double h,
                            const SchemeDev& S, double* b3, double* b4, int sms, cudaStream_t st);
cudaError_t launch_axpy2(int64_t N, double* y, double a1, const double* x1, double a2, const double* x2, int sms,
                         cudaStream_t st);
// FP64 FMA throughput probe (kiops_probe.cu): `blocks` blocks of probe_threads() threads, each thread
// running `chains` (8 or 16) FMA chains for probe_flops_per_thread(chains, iters) flops; out holds
// blocks * probe_threads() doubles.
int probe_threads();
double probe_flops_per_thread(int chains, int iters);
cudaError_t launch_fp64_probe(int chains, int blocks, int iters, double* out, cudaStream_t st);
}  // namespace kiops_k
