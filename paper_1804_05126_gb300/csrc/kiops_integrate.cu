// Pointwise kernels of the exponential integrators (section 4): the right-hand side f(u) = L u + R(u) of
// the paper's 2D ADR and Gray-Scott problems, the h-scaled Jacobian coupling fields, the stage vectors,
// the nonlinear remainders r(U) and the b vectors of the Task II call (eqs 9-11, 50, 51, 53).
//
// Every kernel is a grid-stride loop over grid points (a point carries both species of Gray-Scott), so
// each thread reads and writes only its own point except for the stencil neighbours of f.
#include "kiops_kernels.h"

#include <cuda_runtime.h>

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ int64_t wrap(int bc, int64_t i, int64_t n) {
  if (i >= 0 && i < n) return i;
  if (bc == 1) return i < 0 ? i + n : i - n;
  return i < 0 ? -i : 2 * (n - 1) - i;  // homogeneous Neumann: reflection
}

// Pointwise nonlinear part R and its Jacobian dR at one grid point (x[s] = species s at the point).
__device__ __forceinline__ void reaction(const kiops_k::PdeDev& P, const double* x, double* R, double (*dR)[2]) {
  if (P.kind == 0) {  // gamma u (u - 1/2)(1 - u)
    const double u = x[0], g = P.prm[2];
    R[0] = g * u * (u - 0.5) * (1.0 - u);
    if (dR) dR[0][0] = g * (-3.0 * u * u + 3.0 * u - 0.5);
  } else {  // Gray-Scott: -u v^2 + a (1 - u), u v^2 - (a + b) v
    const double u = x[0], v = x[1], a = P.prm[2], b = P.prm[3];
    R[0] = -u * v * v + a * (1.0 - u);
    R[1] = u * v * v - (a + b) * v;
    if (dR) {
      dR[0][0] = -v * v - a;
      dR[0][1] = -2.0 * u * v;
      dR[1][0] = v * v;
      dR[1][1] = 2.0 * u * v - (a + b);
    }
  }
}

// hf = h f(u); fields (if given) = h dR(u) in the operator's (r, c) layout.
__global__ void pde_eval_kernel(kiops_k::PdeDev P, const double* __restrict__ u, double h, double* __restrict__ hf,
                                double* f00, double* f01, double* f10, double* f11) {
  const int64_t n = P.n, npts = n * n;
  const double idx2 = 1.0 / (P.dx * P.dx), i2dx = 1.0 / (2.0 * P.dx);
  for (int64_t pt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pt < npts; pt += (int64_t)gridDim.x * blockDim.x) {
    const int64_t iy = pt / n, ix = pt - iy * n;
    const int64_t xw = wrap(P.bc, ix - 1, n), xe = wrap(P.bc, ix + 1, n);
    const int64_t ys = wrap(P.bc, iy - 1, n), yn = wrap(P.bc, iy + 1, n);
    double x[2], R[2], dR[2][2];
    for (int s = 0; s < P.ns; ++s) x[s] = u[s * npts + pt];
    reaction(P, x, R, f00 ? dR : nullptr);
    for (int s = 0; s < P.ns; ++s) {
      const double* z = u + s * npts;
      const double c = z[pt], w = z[iy * n + xw], e = z[iy * n + xe], so = z[ys * n + ix], no = z[yn * n + ix];
      const double lap = (w + e + so + no - 4.0 * c) * idx2;
      double lin;
      if (P.kind == 0) lin = P.prm[0] * lap - P.prm[1] * (((e - w) + (no - so)) * i2dx);
      else lin = P.prm[s] * lap;
      hf[s * npts + pt] = h * (lin + R[s]);
    }
    if (f00) {
      f00[pt] = h * dR[0][0];
      if (P.ns == 2) {
        f01[pt] = h * dR[0][1];
        f10[pt] = h * dR[1][0];
        f11[pt] = h * dR[1][1];
      }
    }
  }
}

// U2 = u + c2 W2, U3 = u + c3 W3
__global__ void stages_kernel(int64_t N, const double* __restrict__ u, const double* __restrict__ W2, double c2,
                              const double* __restrict__ W3, double c3, double* __restrict__ U2, double* __restrict__ U3) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double ui = u[i];
    U2[i] = ui + c2 * W2[i];
    U3[i] = ui + c3 * W3[i];
  }
}

// r(U) = R(U) - R(u) - dR(u) (U - u) at one point (the linear part L cancels exactly in the remainder
// defined below eq 2: f(U) - f(u) - J(u)(U - u) with f = L u + R(u) and J = L + dR(u))
__device__ __forceinline__ void remainder_at(const kiops_k::PdeDev& P, const double* un, const double* U, int64_t npts,
                                             int64_t pt, double* r) {
  double xu[2], xU[2], Ru[2], RU[2], dR[2][2];
  for (int s = 0; s < P.ns; ++s) {
    xu[s] = un[s * npts + pt];
    xU[s] = U[s * npts + pt];
  }
  reaction(P, xu, Ru, dR);
  reaction(P, xU, RU, nullptr);
  for (int s = 0; s < P.ns; ++s) {
    double lin = 0.0;
    for (int q = 0; q < P.ns; ++q) lin = fma(dR[s][q], xU[q] - xu[q], lin);
    r[s] = (RU[s] - Ru[s]) - lin;
  }
}

// out = h r(U)
__global__ void remainder_kernel(kiops_k::PdeDev P, const double* __restrict__ un, const double* __restrict__ U,
                                 double h, double* __restrict__ out) {
  const int64_t npts = P.n * P.n;
  for (int64_t pt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pt < npts; pt += (int64_t)gridDim.x * blockDim.x) {
    double r[2];
    remainder_at(P, un, U, npts, pt, r);
    for (int s = 0; s < P.ns; ++s) out[s * npts + pt] = h * r[s];
  }
}

// b3 = h (x3 r2 + y3 (r3 + z r2)), b4 = h (x4 r2 + y4 (r3 + z r2)) with r2 = r(U2), r3 = r(U3)
__global__ void assemble_kernel(kiops_k::PdeDev P, const double* __restrict__ un, const double* __restrict__ U2,
                                const double* __restrict__ U3, double h, kiops_k::SchemeDev S, double* __restrict__ b3,
                                double* __restrict__ b4) {
  const int64_t npts = P.n * P.n;
  for (int64_t pt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pt < npts; pt += (int64_t)gridDim.x * blockDim.x) {
    double r2[2], r3[2];
    remainder_at(P, un, U2, npts, pt, r2);
    remainder_at(P, un, U3, npts, pt, r3);
    for (int s = 0; s < P.ns; ++s) {
      const double d = r3[s] + S.z * r2[s];
      b3[s * npts + pt] = h * (S.x3 * r2[s] + S.y3 * d);
      b4[s * npts + pt] = h * (S.x4 * r2[s] + S.y4 * d);
    }
  }
}

// y += a1 x1 + a2 x2
__global__ void axpy2_kernel(int64_t N, double* __restrict__ y, double a1, const double* __restrict__ x1, double a2,
                             const double* __restrict__ x2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double v = y[i];
    if (x1) v += a1 * x1[i];
    if (x2) v += a2 * x2[i];
    y[i] = v;
  }
}

int grid_for(int64_t n, int sms) {
  const int64_t want = (n + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)sms * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

namespace kiops_k {

cudaError_t launch_pde_eval(const PdeDev& P, const double* u, double h, double* hf, double* const fields[4], int sms,
                            cudaStream_t st) {
  pde_eval_kernel<<<grid_for(P.n * P.n, sms), kBlock, 0, st>>>(P, u, h, hf, fields ? fields[0] : nullptr,
                                                                fields ? fields[1] : nullptr,
                                                                fields ? fields[2] : nullptr,
                                                                fields ? fields[3] : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_stages(int64_t N, const double* u, const double* W2, double c2, const double* W3, double c3,
                          double* U2, double* U3, int sms, cudaStream_t st) {
  stages_kernel<<<grid_for(N, sms), kBlock, 0, st>>>(N, u, W2, c2, W3, c3, U2, U3);
  return cudaGetLastError();
}

cudaError_t launch_remainder(const PdeDev& P, const double* un, const double* U, double h, double* out, int sms,
                             cudaStream_t st) {
  remainder_kernel<<<grid_for(P.n * P.n, sms), kBlock, 0, st>>>(P, un, U, h, out);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const PdeDev& P, const double* un, const double* U2, const double* U3, double h,
                            const SchemeDev& S, double* b3, double* b4, int sms, cudaStream_t st) {
  assemble_kernel<<<grid_for(P.n * P.n, sms), kBlock, 0, st>>>(P, un, U2, U3, h, S, b3, b4);
  return cudaGetLastError();
}

cudaError_t launch_axpy2(int64_t N, double* y, double a1, const double* x1, double a2, const double* x2, int sms,
                         cudaStream_t st) {
  axpy2_kernel<<<grid_for(N, sms), kBlock, 0, st>>>(N, y, a1, x1, a2, x2);
  return cudaGetLastError();
}

}  // namespace kiops_k
