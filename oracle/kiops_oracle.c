/*
 * KIOPS CPU oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, serial FP64 implementation of the KIOPS method of Gaudreault, Rainwater & Tokman,
 * "KIOPS: A fast adaptive Krylov subspace solver for exponential integrators", J. Comput. Phys. 372
 * (2018), with its corrigendum.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this code; the product path never does.  It shares no code, header, table or
 * helper with the CUDA implementation.
 *
 * The vector loops carry OpenMP work-sharing pragmas.  The parity oracle is compiled without OpenMP,
 * so they are ignored there and every loop runs serially in its written order; a second build with
 * -fopenmp serves only the all-core timing of the CPU baseline (its sums are then split over threads).
 *
 * Every function names the passage it follows.  The steps are taken in the paper's order:
 *   Theorem 1 (eqs 13-15, corrigendum eqs 18-19)  augmented matrix  Ã = [[A, B], [0, K]]
 *   Algorithm 1                                    substepping driver (Task II: one output time)
 *   Algorithm 2                                    incomplete orthogonalisation (MGS order, length m_o)
 *   eqs 33, 36-38                                  projection and a-posteriori error estimate
 *   eq 39                                          acceptance  omega <= 1.4
 *   Algorithm 4, sections 3.6.1 / 3.6.2            adaptive choice of tau and m
 *   section 3.7, eqs 47-49                         exact tail reset and power-of-two scaling of B
 *   section 3.3.1 ([47] = Higham 2005)             diagonal Pade approximant with scaling and squaring
 *
 * Readings of passages that are ambiguous or garbled (each is also a switch or a documented choice):
 *   R1  H~ used in the exponential has a zero last row (eq 37), not the slice H(1:j+1,1:j+1) that
 *       Algorithm 1 exponentiates; opts.literal_last_row=1 selects the literal slice instead.
 *   R2  eq 43 is applied as (q+1) = log(eps/eps_old) / log(tau/tau_old), the inverse of the printed
 *       ratio, so that it matches its own error model err ~ C tau^(q+1); q+1 = m/4 otherwise.
 *   R3  kappa (eq 45) and the order estimate (eq 43) are reset at each new substep and updated only
 *       when the current iteration is rejected right after a rejected one in the same substep.
 *   R4  m_new = ceil(m + log(omega/gamma)/log kappa), clipped to [floor(3m/4), ceil(4m/3)] and then
 *       to [m_min, m_max] (eq 46 and the text after it).
 *   R5  "remaining interval" is T_end - (T_now + tau) after an accepted step, T_end - T_now after a
 *       rejected one; a new substep starts with tau = min(tau, T_end - T_now).
 *   R6  happy breakdown when ||x|| <= breakdown_tol * ||A~ v_j|| (the breakdown test of Algorithm 2).
 *   R7  ||B||_1 is the matrix 1-norm (largest column sum); nu = mu = 1 when it is 0 or p = 0.
 *   R16 Task I: the intermediate outputs of Algorithm 3 use beta, the substep's start-vector norm, as scale.
 *   R9  Cost model (eqs 40-42), evaluated after every iteration that did not break down.  Scenario A
 *       keeps m and takes tau_A from eq 44 (gamma = 0.9 after an accepted iteration, 0.6 after a
 *       rejected one, clipped as in Algorithm 4's m = m_max branch); scenario B keeps tau and takes m_B from
 *       eq 46 as in R4.  t_end - t_now is the remaining interval of R5 (cost 0 when none is left).
 *       nz(A~) in eq 41 counts the operator's stored nonzeros only (the B block is the separate
 *       (2p-1)N + p term): CSR nnz, 5 (2D) or 7 (3D) per unknown for a stencil plus one per unknown
 *       and coupling field, n^2 dense.  N_mult in eq 42 is the multiplication count of [47] for a
 *       matrix of the 1-norm of tau H~ (scaled by tau_A/tau for scenario A): pi_m = 2, 3, 4, 5, 6
 *       for Pade degrees 3, 5, 7, 9, 13 plus the s squarings.  With opts.scenario = 1 the cheaper
 *       scenario replaces Algorithm 4's choice in its branch that varies m (ties keep scenario B).
 *       The paper prints no cost values; the pieces are pinned by values worked out by hand from eqs 40-42,
 *       from [47]'s degree thresholds and from the operators' nonzero counts (tests/golden/cost_model.txt),
 *       and the scenario inputs tau_A (eq 44) and m_B (eq 46) by the hand-worked Algorithm 4 sequences
 *       (tests/golden/alg4_scripted.txt); the composition per iteration follows R9 and is checked against
 *       the paper's statement that scenario B is almost always the cheaper completion, and the
 *       cheaper-scenario mode against the exact dense exponential.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------------
 * Operator descriptions (the matrix A of eq 12).  All arrays are host arrays owned by the caller.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  int kind;                 /* 0 CSR, 1 five-point 2D stencil, 2 seven-point 3D stencil, 3 dense */
  int64_t n;                /* number of unknowns N */
  /* CSR */
  const int32_t* rowptr;
  const int32_t* colind;
  const double* vals;
  /* stencils: grid sizes, species count (2D only), boundary type */
  int64_t nx, ny, nz;
  int nspecies;             /* 1 or 2 (2D); species-blocked unknown ordering [u; v] */
  int bc;                   /* 0: homogeneous Dirichlet, 1: periodic, 2: homogeneous Neumann */
  double coef[2][7];        /* per species: centre, -x, +x, -y, +y, (-z, +z) */
  const double* diag[2][2]; /* diag[r][c][pt]: pointwise coupling from species c into species r; NULL = 0 */
  /* dense (row-major n x n) */
  const double* dense;
} oracle_op;

typedef struct {
  int m_min, m_max, m_o;
  int normalize;            /* section 3.7 scaling of B (1 = on) */
  double breakdown_tol;     /* R6 */
  int64_t max_substeps;
  int64_t max_iterations;
  int literal_last_row;     /* R1 switch */
  int scenario;             /* R9: 0 Algorithm 4, 1 the cheaper scenario of eq 40 */
} oracle_opts;

typedef struct {
  int64_t substep;
  int j;
  double tau, t_now, eps, omega;
  int accepted, breakdown;
  int m_new;
  double tau_new;
  double cost_a, cost_b;    /* eq 40 for scenario A (tau_A, m) and B (tau, m_B) (R9); 0 on breakdown */
  double hnorm;             /* ||tau H~||_1 of the iteration's exponential */
} oracle_trace;

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOMEM = 2, ORACLE_ENOTCONV = 3 };

/* y = A x for the operator; follows the definitions of the test problems' Jacobians (section 4). */
static double stencil_x(const oracle_op* A, const double* x, int s, int64_t ix, int64_t iy, int64_t iz) {
  int64_t nx = A->nx, ny = A->ny, nz = A->kind == 2 ? A->nz : 1;
  if (A->bc == 1) {
    ix = (ix + nx) % nx;
    iy = (iy + ny) % ny;
    iz = (iz + nz) % nz;
  } else if (A->bc == 2) {
    /* homogeneous Neumann, second-order ghost point: the value one step outside equals the value one
       step inside (x(-1) = x(1), x(n) = x(n-2)) */
    if (ix < 0) ix = -ix;
    if (ix >= nx) ix = 2 * (nx - 1) - ix;
    if (iy < 0) iy = -iy;
    if (iy >= ny) iy = 2 * (ny - 1) - iy;
    if (nz > 1) {
      if (iz < 0) iz = -iz;
      if (iz >= nz) iz = 2 * (nz - 1) - iz;
    }
  } else if (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= nz) {
    return 0.0;
  }
  return x[(int64_t)s * nx * ny * nz + (iz * ny + iy) * nx + ix];
}

void oracle_apply(const oracle_op* A, const double* x, double* y) {
  if (A->kind == 0) {
#pragma omp parallel for
    for (int64_t i = 0; i < A->n; ++i) {
      double acc = 0.0;
      for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) acc += A->vals[k] * x[A->colind[k]];
      y[i] = acc;
    }
  } else if (A->kind == 1 || A->kind == 2) {
    int64_t nx = A->nx, ny = A->ny, nz = A->kind == 2 ? A->nz : 1;
    int ns = A->kind == 2 ? 1 : A->nspecies;
    int64_t npts = nx * ny * nz;
#pragma omp parallel for collapse(3)
    for (int s = 0; s < ns; ++s)
      for (int64_t iz = 0; iz < nz; ++iz)
        for (int64_t iy = 0; iy < ny; ++iy)
          for (int64_t ix = 0; ix < nx; ++ix) {
            int64_t pt = (iz * ny + iy) * nx + ix;
            const double* c = A->coef[s];
            double acc = c[0] * stencil_x(A, x, s, ix, iy, iz);
            acc += c[1] * stencil_x(A, x, s, ix - 1, iy, iz);
            acc += c[2] * stencil_x(A, x, s, ix + 1, iy, iz);
            acc += c[3] * stencil_x(A, x, s, ix, iy - 1, iz);
            acc += c[4] * stencil_x(A, x, s, ix, iy + 1, iz);
            if (A->kind == 2) {
              acc += c[5] * stencil_x(A, x, s, ix, iy, iz - 1);
              acc += c[6] * stencil_x(A, x, s, ix, iy, iz + 1);
            }
            for (int r = 0; r < ns; ++r)
              if (A->diag[s][r]) acc += A->diag[s][r][pt] * x[(int64_t)r * npts + pt];
            y[(int64_t)s * npts + pt] = acc;
          }
  } else {
#pragma omp parallel for
    for (int64_t i = 0; i < A->n; ++i) {
      double acc = 0.0;
      for (int64_t k = 0; k < A->n; ++k) acc += A->dense[i * A->n + k] * x[k];
      y[i] = acc;
    }
  }
}

/* ------------------------------------------------------------------------------------------------
 * Dense matrix exponential: diagonal Pade approximant with scaling and squaring (section 3.3.1,
 * reference [47]: N. J. Higham, SIAM J. Matrix Anal. Appl. 26 (2005) 1179-1193).  The degree is the
 * smallest of 3, 5, 7, 9 whose published threshold theta_m bounds ||A||_1; otherwise degree 13 after
 * scaling by 2^-s with s = ceil(log2(||A||_1 / theta_13)).  The Pade coefficients come from the closed
 * form c_k = (2m-k)! m! / ((2m)! k! (m-k)!).  p(X) and q(X) = p(-X) are evaluated by plain Horner
 * steps, q R = p is solved by Gaussian elimination with partial pivoting, and R is squared s times.
 * ---------------------------------------------------------------------------------------------- */
static void matmul(int n, const double* a, const double* b, double* c) {
#pragma omp parallel for
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double s = 0.0;
      for (int l = 0; l < n; ++l) s += a[i * n + l] * b[l * n + k];
      c[i * n + k] = s;
    }
}

static double norm1(int n, const double* a) {
  double best = 0.0;
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fabs(a[i * n + k]);
    if (s > best) best = s;
  }
  return best;
}

/* ceil(log2(x)) for x > 0, exact: x = f 2^e with f in [0.5, 1). */
static int ceil_log2(double x) {
  int e;
  double f = frexp(x, &e);
  return f == 0.5 ? e - 1 : e;
}

static double pade_coef(int m, int k) {
  /* (2m-k)! m! / ((2m)! k! (m-k)!) as a product of ratios */
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c *= (double)(m - k + i) / ((double)i * (double)(2 * m - k + i));
  return c;
}

/* Solve Q R = P in place (P becomes R); Gaussian elimination with partial pivoting. */
static int lu_solve(int n, double* q, double* p) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = fabs(q[col * n + col]);
    for (int r = col + 1; r < n; ++r)
      if (fabs(q[r * n + col]) > best) { best = fabs(q[r * n + col]); piv = r; }
    if (best == 0.0) return -1;
    if (piv != col) {
      for (int k = 0; k < n; ++k) {
        double t = q[col * n + k]; q[col * n + k] = q[piv * n + k]; q[piv * n + k] = t;
        t = p[col * n + k]; p[col * n + k] = p[piv * n + k]; p[piv * n + k] = t;
      }
    }
    for (int r = col + 1; r < n; ++r) {
      double f = q[r * n + col] / q[col * n + col];
      if (f == 0.0) continue;
      for (int k = col; k < n; ++k) q[r * n + k] -= f * q[col * n + k];
      for (int k = 0; k < n; ++k) p[r * n + k] -= f * p[col * n + k];
    }
  }
  for (int col = n - 1; col >= 0; --col) {
    for (int k = 0; k < n; ++k) {
      double s = p[col * n + k];
      for (int l = col + 1; l < n; ++l) s -= q[col * n + l] * p[l * n + k];
      p[col * n + k] = s / q[col * n + col];
    }
  }
  return 0;
}

int oracle_expm(int n, const double* a, double* f) {
  static const int degs[5] = {3, 5, 7, 9, 13};
  /* theta_m of Higham (2005), Table 2.3 (double precision) */
  static const double theta[5] = {1.495585217958292e-2, 2.539398330063230e-1, 9.504178996162932e-1,
                                  2.097847961257068e0, 5.371920351148152e0};
  if (n <= 0) return 0;
  size_t nn = (size_t)n * n;
  double* x = (double*)malloc(nn * sizeof(double));
  double* pm = (double*)malloc(nn * sizeof(double));
  double* qm = (double*)malloc(nn * sizeof(double));
  double* t = (double*)malloc(nn * sizeof(double));
  if (!x || !pm || !qm || !t) { free(x); free(pm); free(qm); free(t); return ORACLE_ENOMEM; }
  double nrm = norm1(n, a);
  int deg = 13, s = 0;
  for (int d = 0; d < 4; ++d)
    if (nrm <= theta[d]) { deg = degs[d]; break; }
  if (deg == 13 && nrm > theta[4]) s = ceil_log2(nrm / theta[4]);
  if (s < 0) s = 0;
  double scale = ldexp(1.0, -s);
  for (size_t i = 0; i < nn; ++i) x[i] = a[i] * scale;
  /* Horner: P = c_m I; P = P X + c_k I for k = m-1..0; Q likewise with (-1)^k c_k */
  for (size_t i = 0; i < nn; ++i) { pm[i] = 0.0; qm[i] = 0.0; }
  for (int i = 0; i < n; ++i) {
    pm[i * n + i] = pade_coef(deg, deg);
    qm[i * n + i] = (deg % 2 ? -1.0 : 1.0) * pade_coef(deg, deg);
  }
  for (int k = deg - 1; k >= 0; --k) {
    double ck = pade_coef(deg, k);
    matmul(n, pm, x, t);
    memcpy(pm, t, nn * sizeof(double));
    for (int i = 0; i < n; ++i) pm[i * n + i] += ck;
    matmul(n, qm, x, t);
    memcpy(qm, t, nn * sizeof(double));
    for (int i = 0; i < n; ++i) qm[i * n + i] += (k % 2 ? -1.0 : 1.0) * ck;
  }
  int rc = lu_solve(n, qm, pm);
  for (int i = 0; i < s && rc == 0; ++i) {
    matmul(n, pm, pm, t);
    memcpy(pm, t, nn * sizeof(double));
  }
  memcpy(f, pm, nn * sizeof(double));
  free(x); free(pm); free(qm); free(t);
  return rc == 0 ? ORACLE_OK : ORACLE_EINVAL;
}

/* ------------------------------------------------------------------------------------------------
 * Cost model of section 3.2 (eqs 40-42), reading R9.
 * ---------------------------------------------------------------------------------------------- */
static double op_nonzeros(const oracle_op* A) {
  if (A->kind == 0) return (double)A->rowptr[A->n];
  if (A->kind == 3) return (double)A->n * (double)A->n;
  double npts = (double)A->nx * (double)A->ny * (double)(A->kind == 2 ? A->nz : 1);
  int ns = A->kind == 2 ? 1 : A->nspecies;
  double nz = (A->kind == 2 ? 7.0 : 5.0) * npts * ns;
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c)
      if (A->diag[r][c]) nz += npts;
  return nz;
}

/* multiplications of the scaling-and-squaring Pade method of [47] for a matrix of 1-norm x */
static double n_mult(double x) {
  static const double theta[5] = {1.495585217958292e-2, 2.539398330063230e-1, 9.504178996162932e-1,
                                  2.097847961257068e0, 5.371920351148152e0};
  static const double pi_m[5] = {2, 3, 4, 5, 6};
  for (int d = 0; d < 4; ++d)
    if (x <= theta[d]) return pi_m[d];
  int s = x > theta[4] ? ceil_log2(x / theta[4]) : 0;
  return pi_m[4] + (s > 0 ? s : 0);
}

static double cost_iop(double m, double N, double p, double nz) { /* eq 41 */
  return m * ((2.0 * nz + (2.0 * p - 1.0) * N + p) + 8.0 * (N + p)) - 4.0 * (N + p) + 3.0 * (N + p) * m;
}

static double cost_exp(double nmult, double m, double p) { /* eq 42 */
  return nmult * (2.0 * (m + p) - 1.0) * (m + p) * (m + p);
}

/* eq 40: the cost of finishing the remaining interval rem with steps tau and dimension m */
static double cost_remaining(double rem, double tau, double m, double N, double p, double nz, double nmult) {
  if (!(rem > 0.0) || !(tau > 0.0)) return 0.0;
  return ceil(rem / tau) * (cost_iop(m, N, p, nz) + cost_exp(nmult, m, p));
}

/* The cost model's pieces as exported entry points (for the pins of the tests): eq 40 with eqs 41-42,
 * the N_mult of [47] and nz(A~) of reading R9. */
double oracle_cost_eq40(double rem, double tau, double m, double N, double p, double nz, double nmult) {
  return cost_remaining(rem, tau, m, N, p, nz, nmult);
}
double oracle_n_mult(double x) { return n_mult(x); }
double oracle_op_nonzeros(const oracle_op* A) { return op_nonzeros(A); }

/* ------------------------------------------------------------------------------------------------
 * Augmented matrix-vector product (Algorithm 2; Theorem 1 with B = [b_p, ..., b_1]).
 * x has N + p entries: x[0:N] the state, x[N+t] (t = 0..p-1) the tail; tail row t pairs with
 * column t of B, which is b_{p-t}.  nu scales B (section 3.7).
 * ---------------------------------------------------------------------------------------------- */
static void aug_matvec(const oracle_op* A, int p, const double* const* b, double nu, const double* x,
                       double* y) {
  int64_t N = A->n;
  oracle_apply(A, x, y);
  for (int t = 0; t < p; ++t) {
    const double* col = b[p - t];
    double c = nu * x[N + t];
#pragma omp parallel for
    for (int64_t i = 0; i < N; ++i) y[i] += col[i] * c;
  }
  for (int t = 0; t + 1 < p; ++t) y[N + t] = x[N + t + 1];
  if (p >= 1) y[N + p - 1] = 0.0;
}

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* ------------------------------------------------------------------------------------------------
 * Algorithm 2 generalised to length m_o: extends V, H from j to m columns.  V is (m_max+1) columns of
 * length M = N + p (column c holds v_{c+1}); H is (m_max+2) x (m_max+2) row-major, 1-based H(i,k) at
 * h[(i-1)*ldh + (k-1)].  Returns 1 on happy breakdown.
 * ---------------------------------------------------------------------------------------------- */
static int iop(const oracle_op* A, int p, const double* const* b, double nu, double* V, double* h, int ldh,
               int* jp, int m, int m_o, double bd_tol, double* x, int64_t* matvecs) {
  int64_t M = A->n + p;
  int j = *jp;
  while (j < m) {
    j = j + 1;
    aug_matvec(A, p, b, nu, V + (size_t)(j - 1) * M, x);
    *matvecs += 1;
    double pre = sqrt(dot(x, x, M));
    int i0 = j - m_o + 1 < 1 ? 1 : j - m_o + 1;
    for (int i = i0; i <= j; ++i) {
      const double* vi = V + (size_t)(i - 1) * M;
      double hij = dot(vi, x, M);
      h[(i - 1) * ldh + (j - 1)] = hij;
#pragma omp parallel for
      for (int64_t r = 0; r < M; ++r) x[r] -= hij * vi[r];
    }
    double s = sqrt(dot(x, x, M));
    if (s <= bd_tol * pre) {
      *jp = j;
      return 1;
    }
    h[j * ldh + (j - 1)] = s;
    double inv = 1.0 / s;
    double* vn = V + (size_t)j * M;
#pragma omp parallel for
    for (int64_t r = 0; r < M; ++r) vn[r] = inv * x[r];
  }
  *jp = j;
  return 0;
}

/* Standalone IOP of Algorithm 2 from a given start vector (for invariant checks of eq 30 / Thm 2). */
int oracle_iop(const oracle_op* A, int p, const double* b_flat, const double* v_start, int m, int m_o,
               double bd_tol, double* V_out, double* H_out, int* j_out, int* breakdown_out) {
  int64_t N = A->n, M = N + p;
  const double* b[8];
  if (p < 0 || p > 7 || m < 1) return ORACLE_EINVAL;
  for (int k = 0; k <= p; ++k) b[k] = b_flat + (size_t)k * N;
  int ldh = m + 2;
  double* x = (double*)malloc((size_t)M * sizeof(double));
  if (!x) return ORACLE_ENOMEM;
  double beta = sqrt(dot(v_start, v_start, M));
  for (int64_t r = 0; r < M; ++r) V_out[r] = v_start[r] / beta;
  memset(H_out, 0, sizeof(double) * (size_t)ldh * ldh);
  int j = 0;
  int64_t mv = 0;
  *breakdown_out = iop(A, p, b, 1.0, V_out, H_out, ldh, &j, m, m_o, bd_tol, x, &mv);
  *j_out = j;
  free(x);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Algorithm 4 (with eq 39, section 3.6.1 eqs 43-44 and section 3.6.2 eqs 45-46) for one iteration,
 * as a pure function of the iteration's outcome and the adaptivity memory of the current substep.
 *   eq 39        omega = T_end eps / (tau tol); accepted iff omega <= delta = 1.4; omega = 0 on breakdown
 *   R3           kappa (eq 45) and the order estimate (eq 43 read as R2) start from their defaults at each
 *                new substep and are updated when this iteration is rejected right after a rejected one:
 *                kappa = (omega/omega_old)^(1/(m_old - m)) when m changed and tau did not (kappa <= 1 or
 *                non-finite -> 2); q+1 = log(eps/eps_old)/log(tau/tau_old) when tau changed and m did not
 *                (<= 0 or non-finite -> m/4, section 3.6.1's q = m/4 - 1)
 *   breakdown    tau_new = min(tau, remaining), m_new = m
 *   j == m_max   rejected: m_new = j, tau_new = tau (gamma_max/omega)^(1/(q+1)) clipped to [tau/5, remaining];
 *                accepted: eq 44 with gamma = 0.9, clipped to [tau/5, 5 tau] and remaining
 *   otherwise    tau kept, m_new from eq 46 (R4)
 * "remaining" is R5's: T_end - (T_now + tau) after an accepted iteration, T_end - T_now after a rejected one.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  int have_prev, prev_j;   /* the previous iteration of this substep was rejected (R3) */
  double prev_tau, prev_omega, prev_eps;
  double kappa;            /* eq 45 estimate (default 2, section 3.6.2) */
  double qp1_est;          /* eq 43 estimate of q+1 (0 = none yet) */
} oracle_alg4_state;

typedef struct {
  double omega;
  int accepted;
  double kappa, qp1;       /* the values this iteration's decision used */
  double remaining;
  double tau_new;
  int m_new;
} oracle_alg4_out;

void oracle_alg4(oracle_alg4_state* st, int new_substep, int j, int m, int m_min, int m_max, double tau,
                 double t_now, double T_end, double tol, double eps, int breakdown, oracle_alg4_out* out) {
  const double delta = 1.4, gamma = 0.9, gamma_max = 0.6; /* section 3.5, Algorithm 4 */
  if (new_substep) {
    st->have_prev = 0; st->prev_j = 0;
    st->prev_tau = st->prev_omega = st->prev_eps = 0.0;
    st->kappa = 2.0; st->qp1_est = 0.0;
  }
  const double omega = breakdown ? 0.0 : T_end * eps / (tau * tol); /* eq 39; 0 on a breakdown */
  const int accepted = omega <= delta;
  const double remaining = T_end - (accepted ? t_now + tau : t_now);
  if (!accepted && st->have_prev) { /* R3 */
    if (j != st->prev_j && tau == st->prev_tau) {
      double k = pow(omega / st->prev_omega, 1.0 / (double)(st->prev_j - j)); /* eq 45 */
      st->kappa = (isfinite(k) && k > 1.0) ? k : 2.0;
    } else if (j == st->prev_j && tau != st->prev_tau) {
      double e = log(eps / st->prev_eps) / log(tau / st->prev_tau); /* eq 43, read as R2 */
      st->qp1_est = (isfinite(e) && e > 0.0) ? e : 0.0;
    }
  }
  const double qp1 = st->qp1_est > 0.0 ? st->qp1_est : (double)j / 4.0; /* section 3.6.1: q = m/4 - 1 */
  double tau_new;
  int m_new;
  if (breakdown) { /* tau and m kept */
    tau_new = tau < remaining ? tau : remaining;
    m_new = m;
  } else if (j == m_max) { /* tau varies */
    if (omega > delta) {
      m_new = j;
      tau_new = tau * pow(gamma_max / omega, 1.0 / qp1);
      if (tau_new < tau / 5.0) tau_new = tau / 5.0;
      if (tau_new > remaining) tau_new = remaining;
    } else { /* section 3.6.1, eq 44 */
      m_new = m;
      tau_new = tau * pow(gamma / omega, 1.0 / qp1);
      if (!(tau_new <= 5.0 * tau)) tau_new = 5.0 * tau;
      if (tau_new < tau / 5.0) tau_new = tau / 5.0;
      if (tau_new > remaining) tau_new = remaining;
    }
  } else { /* m varies: section 3.6.2, eq 46, R4 */
    tau_new = tau;
    double mn = (double)m + log(omega / gamma) / log(st->kappa);
    double lo = floor(0.75 * (double)m), hi = ceil(4.0 * (double)m / 3.0);
    if (!(mn >= lo)) mn = lo;
    if (mn > hi) mn = hi;
    mn = ceil(mn);
    if (mn < m_min) mn = m_min;
    if (mn > m_max) mn = m_max;
    m_new = (int)mn;
  }
  if (!accepted) { /* a rejection keeps the basis; this iteration becomes the "old" one (R3) */
    st->have_prev = 1; st->prev_j = j; st->prev_tau = tau; st->prev_omega = omega; st->prev_eps = eps;
  }
  out->omega = omega; out->accepted = accepted; out->kappa = st->kappa; out->qp1 = qp1;
  out->remaining = remaining; out->tau_new = tau_new; out->m_new = m_new;
}

/* ------------------------------------------------------------------------------------------------
 * Algorithm 1 with Algorithms 2-4.
 *   T, n_steps  output times T(1) < ... < T(end) (Task II: one time)
 *   task1       Task I: outputs at every T(l), scaled by (1/T(l))^p (Algorithm 1)
 *   b_flat      (p+1) vectors b_0..b_p of length N, contiguous, natural order
 *   W           n_steps columns of N entries (column l: the result at T(l))
 *   stats       [substeps, rejected, matvecs, m_last, iterations]
 * Reading R16: the intermediate outputs of Algorithm 3 are scaled by beta, the norm of the
 * substep's start vector; the printed ||w(:,l)|| would read a column the previous output has overwritten.
 * ---------------------------------------------------------------------------------------------- */
static int kiops_core(const oracle_op* A, const double* T, int n_steps, int task1, int p, const double* b_flat,
                      double tol, int m_init, const oracle_opts* o, double* W, int64_t* stats,
                      oracle_trace* trace, int64_t trace_cap, int64_t* trace_len) {
  const double T_end = T[n_steps - 1];
  int ell = 0;  /* current output column (Algorithm 1) */
  const double gamma = 0.9, gamma_max = 0.6; /* Algorithm 4 (scenario A of the cost model, R9) */
  int64_t N = A->n, M = N + p;
  int m_min = o->m_min, m_max = o->m_max, m_o = o->m_o;
  const double* b[8];
  if (p < 0 || p > 7 || N < 1 || !(tol > 0) || m_init < 1 || m_min < 1 || m_max < m_min || m_o < 1 ||
      T_end < 0 || !isfinite(T_end) || n_steps < 1)
    return ORACLE_EINVAL;
  for (int l = 0; l + 1 < n_steps; ++l)
    if (!(T[l] > 0.0) || !(T[l] < T[l + 1])) return ORACLE_EINVAL;
  for (int k = 0; k <= p; ++k) b[k] = b_flat + (size_t)k * N;
  if (trace_len) *trace_len = 0;
  for (int k = 0; k < 5; ++k) stats[k] = 0;
  memcpy(W, b[0], (size_t)N * sizeof(double)); /* Algorithm 1: w = b_0 */
  if (T_end == 0.0) { stats[3] = m_init; return ORACLE_OK; }

  /* section 3.7, eqs 48-49 */
  double nu = 1.0, mu = 1.0;
  if (p >= 1 && o->normalize) {
    double nb = 0.0;
    for (int k = 1; k <= p; ++k) {
      double s = 0.0;
      for (int64_t i = 0; i < N; ++i) s += fabs(b[k][i]);
      if (s > nb) nb = s;
    }
    if (nb > 0.0) {
      int e = ceil_log2(nb);
      nu = ldexp(1.0, -e);
      mu = ldexp(1.0, e);
    }
  }

  int ldh = m_max + 2, nmax = m_max + 1;
  double* V = (double*)calloc((size_t)(m_max + 1) * M, sizeof(double));
  double* h = (double*)calloc((size_t)ldh * ldh, sizeof(double));
  double* x = (double*)malloc((size_t)M * sizeof(double));
  double* ht = (double*)malloc((size_t)nmax * nmax * sizeof(double));
  double* F = (double*)malloc((size_t)nmax * nmax * sizeof(double));
  if (!V || !h || !x || !ht || !F) { free(V); free(h); free(x); free(ht); free(F); return ORACLE_ENOMEM; }

  int m = m_min > (m_init < m_max ? m_init : m_max) ? m_min : (m_init < m_max ? m_init : m_max); /* m_init clipped to [m_min, m_max] */
  double tau = T_end, t_now = 0.0, beta = 0.0;
  int j = 0, rc = ORACLE_OK;
  int64_t substeps = 0, rejected = 0, matvecs = 0, iters = 0;
  /* adaptivity memory of the current substep (R3), reset by the first iteration of every substep */
  oracle_alg4_state a4;
  int new_sub = 1;

  while (t_now < T_end) {
    if (iters >= o->max_iterations || substeps >= o->max_substeps) { rc = ORACLE_ENOTCONV; break; }
    if (j == 0) { /* new substep: start vector */
      if (tau > T_end - t_now) tau = T_end - t_now; /* R5 */
      memcpy(V, W + (size_t)ell * N, (size_t)N * sizeof(double));
      for (int t = 0; t < p; ++t) { /* tail (corrigendum), eq 47, times mu */
        int e = p - 1 - t;
        double v = 1.0;
        for (int i = 1; i <= e; ++i) v *= t_now / (double)i;
        V[N + t] = mu * v;
      }
      beta = sqrt(dot(V, V, M));
      if (beta == 0.0) { /* v = 0: the exponential maps it to 0 */
        memset(W + (size_t)ell * N, 0, (size_t)(n_steps - ell) * N * sizeof(double));
        break;
      }
      double inv = 1.0 / beta;
#pragma omp parallel for
      for (int64_t r = 0; r < M; ++r) V[r] *= inv; /* V_1 = [w; tail] / beta */
      memset(h, 0, (size_t)ldh * ldh * sizeof(double));
      new_sub = 1;
    }
    int breakdown = iop(A, p, b, nu, V, h, ldh, &j, m, m_o, o->breakdown_tol, x, &matvecs); /* Algorithm 2 */

    /* the exponential, eq 37 (R1): H~ = [[H_j, e_1], [0, 0]] */
    int n = j + 1;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) ht[r * n + c] = 0.0;
    for (int r = 1; r <= j; ++r)
      for (int c = 1; c <= j; ++c) ht[(r - 1) * n + (c - 1)] = tau * h[(r - 1) * ldh + (c - 1)];
    ht[0 * n + j] = tau * 1.0;
    if (o->literal_last_row)
      for (int c = 1; c <= j; ++c) ht[j * n + (c - 1)] = tau * h[j * ldh + (c - 1)];
    const double hnorm = norm1(n, ht); /* ||tau H~||_1, for the cost model (R9) */
    if (oracle_expm(n, ht, F) != ORACLE_OK) { rc = ORACLE_ENOTCONV; break; }

    /* eqs 36, 38 */
    double eps = 0.0;
    if (!breakdown) eps = beta * h[j * ldh + (j - 1)] * fabs(F[(j - 1) * n + j]);
    /* eq 39 and Algorithm 4 */
    oracle_alg4_out d;
    oracle_alg4(&a4, new_sub, j, m, m_min, m_max, tau, t_now, T_end, tol, eps, breakdown, &d);
    new_sub = 0;
    const double omega = d.omega, remaining = d.remaining, qp1 = d.qp1, kappa = d.kappa;
    const int accepted = d.accepted;
    double t_next = accepted ? t_now + tau : t_now;
    double tau_new = d.tau_new;
    int m_new = d.m_new;

    /* R9: eq 40 for both scenarios; opts.scenario = 1 takes the cheaper one where Algorithm 4 varies m */
    double cost_a = 0.0, cost_b = 0.0;
    if (!breakdown) {
      double tau_a = tau * pow((accepted ? gamma : gamma_max) / omega, 1.0 / qp1);
      if (accepted && !(tau_a <= 5.0 * tau)) tau_a = 5.0 * tau;
      if (!(tau_a >= tau / 5.0)) tau_a = tau / 5.0;
      if (tau_a > remaining) tau_a = remaining;
      double mb = (double)m + log(omega / gamma) / log(kappa);
      double lo = floor(0.75 * (double)m), hi = ceil(4.0 * (double)m / 3.0);
      if (!(mb >= lo)) mb = lo;
      if (mb > hi) mb = hi;
      mb = ceil(mb);
      if (mb < m_min) mb = m_min;
      if (mb > m_max) mb = m_max;
      const double nz = op_nonzeros(A);
      cost_a = cost_remaining(remaining, tau_a, (double)m, (double)N, (double)p, nz, n_mult(hnorm * (tau_a / tau)));
      cost_b = cost_remaining(remaining, tau, mb, (double)N, (double)p, nz, n_mult(hnorm));
      if (o->scenario == 1 && j < m_max && cost_a < cost_b) {
        tau_new = tau_a;
        m_new = m;
      }
    }

    if (trace && trace_len && *trace_len < trace_cap) {
      oracle_trace* tr = &trace[*trace_len];
      tr->substep = substeps; tr->j = j; tr->tau = tau; tr->t_now = t_now; tr->eps = eps; tr->omega = omega;
      tr->accepted = accepted; tr->breakdown = breakdown; tr->m_new = m_new; tr->tau_new = tau_new;
      tr->cost_a = cost_a; tr->cost_b = cost_b; tr->hnorm = hnorm;
      *trace_len += 1;
    }
    iters++;

    if (accepted) { /* accepted: Algorithm 3 */
      if (task1) { /* Algorithm 3: outputs strictly inside this substep */
        int n_tau = 0;
        for (int k = ell; k < n_steps; ++k)
          if (fabs(T[k]) < fabs(t_now + tau)) n_tau++;
        if (n_tau > 0) {
          memcpy(W + (size_t)(ell + n_tau) * N, W + (size_t)ell * N, (size_t)N * sizeof(double)); /* running state carried to the next column */
          double* h2 = (double*)malloc((size_t)j * j * sizeof(double));
          double* F2 = (double*)malloc((size_t)j * j * sizeof(double));
          if (!h2 || !F2) { free(h2); free(F2); rc = ORACLE_ENOMEM; break; }
          for (int k = 0; k < n_tau; ++k) {
            const double tt = T[ell + k] - t_now;
            for (int r = 0; r < j; ++r)
              for (int cc = 0; cc < j; ++cc) h2[r * j + cc] = tt * h[r * ldh + cc];
            if (oracle_expm(j, h2, F2) != ORACLE_OK) { rc = ORACLE_ENOTCONV; break; } /* exp((T(k) - T_now) H_j) */
            double* wk = W + (size_t)(ell + k) * N;
            for (int64_t r = 0; r < N; ++r) { /* beta V F(:, 1), R16 */
              double sacc = 0.0;
              for (int cc = 0; cc < j; ++cc) sacc += V[(size_t)cc * M + r] * F2[cc * j + 0];
              wk[r] = beta * sacc;
            }
          }
          free(h2);
          free(F2);
          if (rc != ORACLE_OK) break;
          ell += n_tau;
        }
      }
      double* wl = W + (size_t)ell * N; /* Algorithm 3, the Task II update: w = beta V(1:N,1:j) F(1:j,1) */
#pragma omp parallel for
      for (int64_t r = 0; r < N; ++r) {
        double s = 0.0;
        for (int c = 0; c < j; ++c) s += V[(size_t)c * M + r] * F[c * n + 0];
        wl[r] = beta * s;
      }
      if (tau >= T_end - t_now || t_next >= T_end) t_now = T_end;
      else t_now = t_next;
      j = 0;
      substeps++;
    } else { /* rejected: keep the basis */
      rejected++;
    }
    tau = tau_new;
    m = m_new;
  }
  if (task1 && rc == ORACLE_OK) /* Algorithm 1: outputs scaled by (1/T(l))^p */
    for (int l = 0; l < n_steps; ++l) {
      double sc = 1.0;
      for (int k = 0; k < p; ++k) sc *= 1.0 / T[l];
      for (int64_t r = 0; r < N; ++r) W[(size_t)l * N + r] *= sc;
    }
  stats[0] = substeps; stats[1] = rejected; stats[2] = matvecs; stats[3] = m; stats[4] = iters;
  free(V); free(h); free(x); free(ht); free(F);
  return rc;
}

/* Task II (one output time T_end): sum_k T_end^k phi_k(T_end A) b_k. */
int oracle_kiops(const oracle_op* A, double T_end, int p, const double* b_flat, double tol, int m_init,
                 const oracle_opts* o, double* w_out, int64_t* stats, oracle_trace* trace,
                 int64_t trace_cap, int64_t* trace_len) {
  return kiops_core(A, &T_end, 1, 0, p, b_flat, tol, m_init, o, w_out, stats, trace, trace_cap, trace_len);
}

/* Task I: W(:, l) = (1/T(l))^p e^{T(l) A~} v (top N entries), l = 1..n_steps (Algorithm 1). */
int oracle_kiops_task1(const oracle_op* A, const double* T, int n_steps, int p, const double* b_flat, double tol,
                       int m_init, const oracle_opts* o, double* W, int64_t* stats, oracle_trace* trace,
                       int64_t trace_cap, int64_t* trace_len) {
  return kiops_core(A, T, n_steps, 1, p, b_flat, tol, m_init, o, W, stats, trace, trace_cap, trace_len);
}
