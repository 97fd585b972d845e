/*
 * kiops.h — C ABI of the GB300 (sm_103a) KIOPS solver.
 *
 * Computes  w = sum_{k=0}^{p} tau^k phi_k(tau A) b_k                        (paper eq 12 / eq 20)
 * with the adaptive Krylov method KIOPS of Gaudreault, Rainwater & Tokman, "KIOPS: A fast adaptive
 * Krylov subspace solver for exponential integrators", J. Comput. Phys. 372 (2018):
 *   - one exponential of the augmented matrix A~ = [[A, B], [0, K]], B = [b_p..b_1]   (Theorem 1, eq 13)
 *   - Krylov basis by incomplete orthogonalisation of length m_o                      (Algorithm 2)
 *   - projection beta V_m exp(tau H~) e_1 with H~ = [[H_m, e_1], [0, 0]]             (eqs 33, 37, 38)
 *   - a-posteriori estimate and acceptance omega <= 1.4                              (eqs 36, 39)
 *   - adaptive substep tau and Krylov dimension m                                    (Alg 1, Alg 4, 3.6)
 *   - exact tail reset and power-of-two scaling of B                                 (section 3.7)
 * Only Task II (a single output time, eq 12) is provided.
 *
 * Conventions for every entry point
 *   - Return value: KIOPS_OK or an error status; kiops_last_error(ctx) holds a message for the most
 *     recent failure on that context.  No entry point aborts the process.
 *   - "device" pointers are CUDA device (or managed) addresses on the context's device; "host" pointers
 *     are ordinary host memory.  The caller owns every input and output buffer; the library borrows
 *     them for the duration of the call (operators borrow theirs until kiops_op_destroy).
 *   - Vectors of length N are contiguous FP64 arrays in the operator's unknown ordering.
 *   - The context owns its device workspace (Krylov basis, small dense matrices, barrier words).  It is
 *     allocated with cudaMalloc on first use and grown on demand, unless the caller attaches a buffer
 *     with kiops_attach_workspace.
 *   - A context is used by one host thread at a time.  Work is issued on cfg.stream; calls return after
 *     the work has completed (they synchronise that stream).
 */
#ifndef KIOPS_H
#define KIOPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KIOPS_MAX_P 16   /* largest p (number of phi terms beyond phi_0) */
#define KIOPS_MAX_M 256  /* largest m_max (Krylov dimension cap) */
#define KIOPS_MAX_TIMES 32  /* largest number of Task I output times */

typedef enum {
  KIOPS_OK = 0,
  KIOPS_EINVAL = 1,    /* invalid argument (NULL pointer, p out of range, tol <= 0, tau < 0, ...) */
  KIOPS_ENOMEM = 2,    /* device memory or attached workspace too small */
  KIOPS_ENOTCONV = 3,  /* max_substeps / max_iterations reached before T_end */
  KIOPS_ETIMEOUT = 4,  /* a device-side wait exceeded cfg.timeout_s; the result is invalid */
  KIOPS_ECUDA = 5,     /* a CUDA runtime call failed; see kiops_last_error */
  KIOPS_EBUSY = 6      /* the context is in use */
} kiops_status;

typedef enum {
  KIOPS_FP64 = 0,        /* basis, matvec and all reductions in FP64 */
  KIOPS_FP32_BASIS = 1   /* basis and matvec in FP32; dot products, norms, H, exponential and control in FP64 */
} kiops_precision;

typedef enum {
  KIOPS_ENGINE_AUTO = 0, /* grid engine for large N, single-CTA engine for small N */
  KIOPS_ENGINE_GRID = 1, /* one persistent cooperative kernel over the whole GPU per solve */
  KIOPS_ENGINE_CTA = 2   /* one thread block per solve (used for batches) */
} kiops_engine;

typedef struct {
  int device;              /* CUDA device ordinal (default 0) */
  void* stream;            /* cudaStream_t to issue work on; NULL = the legacy default stream */
  int m_min, m_max;        /* Krylov dimension bounds (Algorithm 1 defaults 10, 128); m_max <= KIOPS_MAX_M */
  int normalize_B;         /* section 3.7 power-of-two scaling of B (default 1); applied with an FP64
                              basis only (with an FP32 basis it would make the tail dominate the basis) */
  double breakdown_tol;    /* happy breakdown when ||x|| <= breakdown_tol * ||A~ v_j|| (default 1e-12) */
  int64_t max_substeps;    /* accepted substeps before KIOPS_ENOTCONV (default 1e6) */
  int64_t max_iterations;  /* accepted + rejected iterations before KIOPS_ENOTCONV (default 1e5) */
  double timeout_s;        /* limit on any single device-side wait (default 10 s) */
  int engine;              /* kiops_engine (default AUTO) */
  int grid_blocks;         /* grid engine block count; 0 = as many as are co-resident */
  int profile;             /* 1: fill kiops_stats.phase_cycles (device cycle counters, rank-0 view) */
  int fuse_stencil;        /* 1 (default): 2D stencils on the grid engine normalise v_{j+1} inside the next
                              step's tiles (one grid barrier per Krylov step), and so do 3D stencils with an
                              FP32 basis on grids with more 3D tiles than blocks (tma > 0); 0: separate
                              normalise pass */
  int batch_team_blocks;   /* kiops_solve_batch: blocks per team (0 = automatic, 1 = one block per request) */
  int fused_smem;          /* tiled 2D path: shared-memory extras, a bitmask of 1 = the finalised tiles of the
                              last m_o + 1 basis vectors, 2 = the next raw tile prefetched (cp.async) during
                              the cross-block sum, 4 = the tile's B columns and coupling fields; -1 (default) =
                              automatic.  A combination that would lower the co-resident block count is
                              dropped, and grids with more tiles than blocks (each block takes several
                              tiles in turn) use none.  Results are bit-identical for every value. */
  int scenario;            /* 0 (default): Algorithm 4 chooses the next m and tau.  1: after an iteration in
                              Algorithm 4's vary-m branch the cheaper of the two scenarios of section 3.2 is
                              taken, by the cost of eq 40 with eqs 41-42: A keeps m and takes tau from eq 44
                              (gamma 0.9 after an accepted, 0.6 after a rejected iteration), B keeps tau and
                              takes m from eq 46 (ties keep B).  nz(A~) counts the operator's stored nonzeros
                              (CSR nnz; 5 or 7 per unknown for stencils plus one per unknown and coupling
                              field); N_mult is the multiplication count of Higham's scaling-and-squaring Pade
                              method for the 1-norm of tau H~.  Both costs are in every trace record. */
  int block_threads;       /* grid engine, FP64 basis: 256 = two blocks of 256 threads per SM, 512 = one block
                              of 512 threads per SM (half the blocks to reduce over and to synchronise),
                              0 (default) = automatic: one block of 512 threads per SM for N <= 65536, one
                              block of 256 threads per SM for N <= 2^19, else two blocks of 256.  Other
                              engines and the FP32 basis use two blocks of 256 threads per SM. */
  int tma;                 /* grid engine, 2D stencils whose grid has more tiles than blocks: stage each tile's
                              operands in shared memory with bulk tensor copies (TMA), ahead of the tile being
                              computed.  1 (default) = with an FP32 basis only (FP64 steps are bound by the FP64
                              pipe and run faster with per-element loads), 2 = with either basis, 0 = never.
                              Used where the row length and the plane size are multiples of 16 bytes. */
  int tile_w, tile_h;      /* that path's tile shape (points; tile_w a multiple of 4); 0, 0 (default) =
                              automatic.  A shape that does not fit the shared memory at the launch's block
                              count is replaced by the automatic choice. */
  int tma_stages;          /* that path's tiles in flight per block (2 to 6; 0 = 2) */
  int tma_prefetch;        /* that path's L2 lookahead: tiles fetched into L2 (bulk prefetch, no shared memory)
                              this many tiles before their shared-memory copy is issued; 0 = none, -1 (default)
                              = automatic (none: measured slower with it) */
  int tma_fixed;           /* that path with an FP32 basis, 32 x 16 tiles, two species and p = 3: 1 (default) =
                              run the kernel compiled for exactly that configuration (constant loop bounds and
                              offsets), 0 = the general one */
} kiops_config;

typedef struct {
  int64_t substeps;        /* accepted substeps */
  int64_t rejected;        /* rejected iterations */
  int64_t matvecs;         /* applications of A~ (Algorithm 2), basis extensions included */
  int64_t iterations;      /* accepted + rejected */
  int64_t expm_calls;      /* small dense exponentials (one per iteration) */
  int m_last;              /* Krylov dimension suggested for the next call (warm start, section 3.6) */
  int engine;              /* engine that ran the solve */
  int grid_blocks;         /* blocks of the launch */
  int status;              /* kiops_status of the device run */
  double err_est;          /* last error estimate eps_m (eq 36) */
  /* SM cycles by phase when cfg.profile is set (rank-0 view): 0 setup, 1 start vector, 2 step matvec+dots
   * and block reduction, 3 step cross-block sum, 4 step coefficients, 5 step normalise, 6 expm powers,
   * 7 expm Horner, 8 expm squarings, 9 control, 10 update, 11 grid barrier waits, 12 tiled path:
   * finalisation of v_j, 13 tiled path: A~ v_j and dots, 14 tiled path with bulk tensor copies: waits for a
   * tile's copies (and the issue of the next ones), 15 that path: the block barrier that ends a tile (waits
   * for the block's last products); other entries 0. */
  int64_t phase_cycles[16];
  /* 2D stencils on the grid engine: how the Krylov step ran.  tile_path 0 = not tiled (or one tile per
   * block), 1 = several tiles per block with per-element loads, 2 = several tiles per block staged by bulk
   * tensor copies, 3 = as 2 with the kernel compiled for 32 x 16 tiles, two species and p = 3; 3D stencils
   * with an FP32 basis: 4 = 3D tiles staged by bulk tensor copies with lagged normalisation (no separate
   * normalise pass); tile_w, tile_h = the tile's x and y extent for paths 1 to 4 (0 otherwise). */
  int tile_path, tile_w, tile_h;
} kiops_stats;

/* One record per iteration (accepted or rejected) when a trace buffer is given. */
typedef struct {
  int64_t substep;
  int j;                   /* Krylov dimension of the iteration */
  int accepted;
  int breakdown;
  int m_new;               /* Algorithm 4 suggestion (or the cost model's, cfg.scenario = 1) */
  double tau, t_now, eps, omega, tau_new;
  double cost_a, cost_b;   /* eq 40 for scenario A (keep m, tau from eq 44) and B (keep tau, m from eq 46); see
                              kiops_config.scenario; 0 on breakdown or when no interval is left */
  double hnorm;            /* ||tau H~||_1 of the iteration's exponential (eq 37) */
} kiops_trace_rec;

typedef struct kiops_ctx kiops_ctx;
typedef struct kiops_op kiops_op;

/* Boundary treatment of the stencil operators: the value of x at an index just outside the grid.
 * KIOPS_BC_DIRICHLET: 0 (homogeneous Dirichlet); KIOPS_BC_PERIODIC: the index wraps;
 * KIOPS_BC_NEUMANN: reflection about the boundary point, x(-1) = x(1) and x(n) = x(n-2) (homogeneous
 * Neumann with the second-order ghost point; needs n >= 2 in every dimension). */
enum { KIOPS_BC_DIRICHLET = 0, KIOPS_BC_PERIODIC = 1, KIOPS_BC_NEUMANN = 2 };

/* 5-point 2D stencil (1 or 2 species) with a pointwise coupling block: unknowns species-blocked
 * [u; v], each x-fastest (index = s*nx*ny + iy*nx + ix).  For species s:
 *   (A x)_s(ix,iy) = coef[s][0] x_s(ix,iy) + coef[s][1] x_s(ix-1,iy) + coef[s][2] x_s(ix+1,iy)
 *                  + coef[s][3] x_s(ix,iy-1) + coef[s][4] x_s(ix,iy+1) + sum_r diag[s][r][pt] x_r(ix,iy)
 * with x outside the grid given by bc.  diag[s][r] are device pointers of nx*ny FP64 values or NULL
 * (= 0).  This covers the Jacobians of the paper's 2D ADR and Gray-Scott test problems (section 4).
 *
 * Shared coupling fields (optional; zero the members below when not used, e.g. by memset of the whole
 * descriptor).  With nfields = 1 or 2 the entries of the pointwise block are affine in fields that several
 * entries share, and diag must be all NULL:
 *   diag[s][r](pt) = fma(dweight[s][r], field[dfield[s][r]][pt], dconst[s][r])   if dfield[s][r] >= 0,
 *   diag[s][r](pt) = dconst[s][r]                                                 if dfield[s][r] = -1,
 * evaluated in FP64 (one rounding).  field[f] are device pointers of nx*ny FP64 values, borrowed like diag.
 * The Gray-Scott Jacobian of section 4 has this form with the two fields v0^2 and 2 u0 v0 (entries
 * -F - v0^2, -2 u0 v0, v0^2 and 2 u0 v0 - (F + k)).  The operator writes the entries once into device
 * memory it owns (8 bytes per point and nonzero entry, freed by kiops_op_destroy) for the paths that read
 * whole entries; the staged several-tiles step (kiops_stats.tile_path 2 or 3, by default with an FP32
 * basis only) reads the nfields planes instead and forms the entries in the basis precision (with an FP32
 * basis its results differ from those of the same block given by diag by the FP32 rounding of the
 * entries).  Errors: KIOPS_EINVAL for nfields outside 0..2, a
 * NULL field, diag given as well, or dfield outside -1..nfields-1 on an entry of the block; KIOPS_ENOMEM
 * or KIOPS_ECUDA if the entries cannot be allocated or written. */
typedef struct {
  int64_t nx, ny;
  int nspecies;            /* 1 or 2 */
  int bc;                  /* KIOPS_BC_* */
  double coef[2][5];
  const double* diag[2][2];
  int nfields;             /* 0 (diag gives the block), 1 or 2 */
  int dfield[2][2];
  double dconst[2][2];
  double dweight[2][2];
  const double* field[2];
} kiops_stencil2d_desc;

/* 7-point 3D stencil, one species, x-fastest (index = (iz*ny + iy)*nx + ix):
 *   (A x)(i) = c[0] x(i) + c[1] x(i-ex) + c[2] x(i+ex) + c[3] x(i-ey) + c[4] x(i+ey) + c[5] x(i-ez)
 *            + c[6] x(i+ez) + diag[i] x(i);  diag is a device pointer of N FP64 values or NULL. */
typedef struct {
  int64_t nx, ny, nz;
  int bc;                  /* KIOPS_BC_* */
  double coef[7];
  const double* diag;
} kiops_stencil3d_desc;

/* One solve of a batch (kiops_solve_batch). */
typedef struct {
  const kiops_op* A;
  double tau;
  int p;
  const double* const* b;  /* host array of p+1 device pointers b_0..b_p (natural order) */
  double tol;
  int m_init;
  int m_o;
  kiops_precision prec;
  double* w;               /* device, N */
} kiops_request;

/* Defaults: m_min 10, m_max 128, normalize_B 1, breakdown_tol 1e-12 (Algorithm 1, section 3.7). */
kiops_status kiops_config_default(kiops_config* cfg);

/* Constants of the method as implemented: out[0..5] = delta (eq 39), gamma (eq 44), gamma_max
 * (Algorithm 4), kappa default (section 3.6.2), tau clip factor 5 (section 3.6.1), m_o default 2. */
kiops_status kiops_constants(double out[6]);

/* Create a context on cfg->device (cfg == NULL: defaults).  *ctx is set on success. */
kiops_status kiops_create(kiops_ctx** ctx, const kiops_config* cfg);
kiops_status kiops_destroy(kiops_ctx* ctx);
const char* kiops_last_error(const kiops_ctx* ctx);
const char* kiops_status_string(kiops_status s);

/* Attach a caller-owned device buffer of `bytes` bytes as the workspace (NULL detaches; the context then
 * allocates its own).  kiops_workspace_size reports the bytes a solve needs. */
kiops_status kiops_attach_workspace(kiops_ctx* ctx, void* dptr, size_t bytes);
kiops_status kiops_workspace_size(kiops_ctx* ctx, const kiops_op* A, int p, int m_o, kiops_precision prec,
                                  size_t* bytes);

/* Operators (the matrix A of eq 12, applied matrix-free, Algorithm 2).
 * CSR: n x n, rowptr[n+1], colind[nnz] (int32), vals[nnz] (FP64), all device pointers, borrowed. */
kiops_status kiops_op_csr(kiops_ctx* ctx, kiops_op** op, int64_t n, int64_t nnz, const int32_t* rowptr,
                          const int32_t* colind, const double* vals);
kiops_status kiops_op_stencil2d(kiops_ctx* ctx, kiops_op** op, const kiops_stencil2d_desc* desc);
kiops_status kiops_op_stencil3d(kiops_ctx* ctx, kiops_op** op, const kiops_stencil3d_desc* desc);
kiops_status kiops_op_destroy(kiops_op* op);
int64_t kiops_op_size(const kiops_op* op);

/* y = A x (device vectors of length N) — the operator alone, for checks. */
kiops_status kiops_op_apply(kiops_ctx* ctx, const kiops_op* A, const double* x, double* y);

/* The solve (Algorithm 1, Task II, T = [tau]).
 *   tau     >= 0 (tau == 0 returns w = b_0 without any matvec)
 *   p       0..KIOPS_MAX_P
 *   b       host array of p+1 DEVICE pointers b_0..b_p, each N FP64 values (natural order)
 *   tol     > 0, absolute tolerance of eq 39
 *   m_init  >= 1, first Krylov dimension (clipped to [m_min, m_max], Algorithm 1)
 *   m_o     >= 1, orthogonalisation length (2 = the paper's IOP; >= m_max = full Arnoldi)
 *   prec    KIOPS_FP64 or KIOPS_FP32_BASIS
 *   w       DEVICE output of N FP64 values (may alias b[0])
 *   stats   host, may be NULL
 * Errors: EINVAL for bad arguments, ENOMEM, ENOTCONV, ETIMEOUT, ECUDA. */
kiops_status kiops_solve(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b, double tol,
                         int m_init, int m_o, kiops_precision prec, double* w, kiops_stats* stats);

/* kiops_solve with a per-iteration trace (host buffer of trace_cap records; *trace_len = records written). */
kiops_status kiops_solve_traced(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b,
                                double tol, int m_init, int m_o, kiops_precision prec, double* w,
                                kiops_stats* stats, kiops_trace_rec* trace, int64_t trace_cap,
                                int64_t* trace_len);

/* Task I (Algorithm 1 with Algorithm 3): one adaptive run to T[n_times-1] that also returns
 *   w[l] = (1/T[l])^p * sum_k T[l]^k phi_k(T[l] A) b_k,   l = 0..n_times-1,
 * i.e. phi_p(T[l] A) b_p for every l when b_0..b_{p-1} are zero (the use the paper makes of it in
 * exponential integrators).  T: host array of increasing positive times (n_times <= KIOPS_MAX_TIMES);
 * w: host array of n_times DEVICE output pointers (N FP64 values each).  Outputs strictly inside an
 * accepted substep come from exp((T[l] - T_now) H_j) on that substep's basis (Algorithm 3);
 * the substep sizes are not shortened to hit them. */
kiops_status kiops_solve_task1(kiops_ctx* ctx, const kiops_op* A, const double* T, int n_times, int p,
                               const double* const* b, double tol, int m_init, int m_o, kiops_precision prec,
                               double* const* w, kiops_stats* stats);

/* Same as kiops_solve but b (p+1 pointers to N values each) and w are HOST buffers; the host-device
 * copies happen inside the call (pinned staging owned by the context). */
kiops_status kiops_solve_host(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b_host,
                              double tol, int m_init, int m_o, kiops_precision prec, double* w_host,
                              kiops_stats* stats);

/* Independent solves in one cooperative launch per (precision, operator kind) group.  The launch is split
 * into teams of cfg.batch_team_blocks blocks (0 = automatic); each team runs a list of requests one after
 * another with its own barrier, partial sums and workspace.  The lists are planned on the host: requests
 * sorted by an estimated work (N times a step count from a Gershgorin bound of ||tau A||) and each given to
 * the least-loaded team.  With 1 block per team every request runs on its own block.  Results do not
 * depend on the team a request lands on only up to the team size (reduction order follows the block count).
 * stats: host array of `count` entries or NULL.  Every request's operator must belong to ctx. */
kiops_status kiops_solve_batch(kiops_ctx* ctx, int count, const kiops_request* reqs, kiops_stats* stats);

/* Set cfg.batch_team_blocks of a live context (used by the batch autotuner). */
kiops_status kiops_set_batch_team_blocks(kiops_ctx* ctx, int team_blocks);

/* The configuration of a live context, and a new one for the solves that follow (used by the autotuner of
 * the engine's launch shapes).  The device and the stream cannot change (EINVAL); a context that runs a server
 * keeps its configuration (EBUSY).  Results depend on the shape settings (tile_w, tile_h, block_threads,
 * grid_blocks, tma) only through the order in which partial sums are added. */
kiops_status kiops_get_config(const kiops_ctx* ctx, kiops_config* cfg);
kiops_status kiops_set_config(kiops_ctx* ctx, const kiops_config* cfg);

/* Dense exponential F = exp(A) of an n x n row-major FP64 matrix (device pointers), n <= KIOPS_MAX_M + 1,
 * computed by the same on-device scaling-and-squaring code the solver uses for exp(tau H~). */
kiops_status kiops_expm(kiops_ctx* ctx, int n, const double* a, double* f);

/* ---- Serving: continuous batching of independent solves (one server per context).
 *
 * kiops_server_start launches a persistent cooperative kernel whose teams of blocks take requests from
 * device-visible queues as soon as they finish the previous one; requests submitted while others run are
 * admitted whenever a queue slot and workspace inside the HBM budget are free, and their work overlaps on
 * the device.  Requests with an estimated work (see kiops_solve_batch) above large_work_threshold go to the
 * "large" class (large_teams teams of large_team_blocks blocks), the others to teams of small_team_blocks
 * blocks.  A request's result depends on its class's team size only, not on the other requests.
 * While the server kernel runs it occupies the GPU: other solves on the device wait until it exits (it
 * exits after idle_timeout_s without work and is relaunched by the next submit or poll).  The paper has no
 * counterpart; this is the execution model of the build. */
typedef struct {
  double hbm_budget_bytes;      /* admission budget for request workspaces, allocated at start (120e9) */
  int queue_slots;              /* request slots per class (512) */
  int small_team_blocks;        /* blocks per small team (8) */
  int large_team_blocks;        /* blocks per large team (0 = the large teams share half of the co-resident blocks) */
  int large_teams;              /* number of large teams (2; 0 = every request is small) */
  double large_work_threshold;  /* estimated work above which a request is large (2e8) */
  double idle_timeout_s;        /* the kernel exits after this long without work; must be < cfg.timeout_s (2) */
  double solo_min_unknowns;     /* requests with at least this many unknowns run alone on the whole GPU (the grid
                                   engine of kiops_solve) between launches of the server kernel: the server stops
                                   admitting, lets the requests in flight finish, runs them in arrival order and
                                   resumes.  A team's share of the GPU is slower for such sizes.  0 = never
                                   (default 1e6) */
} kiops_server_config;

kiops_status kiops_server_config_default(kiops_server_config* cfg);
kiops_status kiops_server_start(kiops_ctx* ctx, const kiops_server_config* cfg);
/* Queue one request (same fields as kiops_solve; tau > 0).  b and w are borrowed until kiops_poll reports
 * it done.  *ticket identifies it.  Errors: EINVAL, ENOMEM if it cannot fit the budget even alone. */
kiops_status kiops_submit(kiops_ctx* ctx, const kiops_request* req, uint64_t* ticket);
/* Wait up to timeout_s (0 = just check) for a ticket; *done = 1 and stats filled once it has finished.  Requests
 * that run alone (solo_min_unknowns) are run inside this call, so one call can take as long as such a solve. */
kiops_status kiops_poll(kiops_ctx* ctx, uint64_t ticket, double timeout_s, int* done, kiops_stats* stats);
/* info[0..7] = pending (not yet admitted), in flight, reserved workspace bytes, small teams, large teams,
 * blocks per large team, requests the small and the large teams have claimed since the server started. */
kiops_status kiops_server_info(kiops_ctx* ctx, int64_t info[8]);
/* Self-test of the server's recovery from a device-side wait that gave up (the paper has no counterpart):
 * raises the server's abort word from the host, as such a wait does.  Running teams stop at their next
 * check of the word and the kernel exits; requests they had claimed finish with KIOPS_ETIMEOUT (reported
 * by kiops_poll), requests not yet claimed stay queued, and the next launch clears the word and serves
 * them.  EINVAL without a server. */
kiops_status kiops_server_selftest_abort(kiops_ctx* ctx);
/* Stop the server after the queued work (waits for the kernel), free its memory. */
kiops_status kiops_server_stop(kiops_ctx* ctx);

/* ---- Exponential integrators (section 4) ------------------------------------------------------------
 * Constant-step integration of the paper's nonlinear 2D test problems with the stiffly accurate schemes of
 * section 4 in their grouped ("mixed") form of section 2: per step one Task I call gives both stage
 * vectors (phi_1 at the two stage nodes), one Task II call (eqs 10-11, A = h J_n, tau = 1) gives u_{n+1};
 * EXPRB5s3 adds a Task I call for the phi_3 terms of its third stage.  Each call starts from the Krylov
 * dimension its counterpart ended with in the previous step (section 3.6).  All in FP64.
 *   EPIRK4s3  (eq 50): nodes 1/8, 1/9; b_3 = h(1892 r2 + 1458 (r3 - 2 r2)), b_4 = h(-42336 r2 - 34992 (r3 - 2 r2))
 *   EPIRK4s3A (eq 51): nodes 1/2, 2/3; b_3 = h(32 r2 - 27/2 r3), b_4 = h(-144 r2 + 81 r3)
 *   EXPRB5s3  (eq 53): nodes 1/2, 9/10; third stage + (27/25 phi_3(A/2) + 729/125 phi_3(9A/10)) h r2;
 *                      b_3 = h(18 r2 - 250/81 r3), b_4 = h(-60 r2 + 500/27 r3)
 * with r2 = r(U_n2), r3 = r(U_n3) and r(U) = f(U) - f(u_n) - J_n (U - u_n) (section 2). */
enum { KIOPS_PDE_ADR2D = 0, KIOPS_PDE_GRAY_SCOTT2D = 1 };
enum { KIOPS_EPIRK4S3 = 0, KIOPS_EPIRK4S3A = 1, KIOPS_EXPRB5S3 = 2 };

/* KIOPS_PDE_ADR2D: u_t = eps Lap u - alpha (u_x + u_y) + gamma u (u - 1/2)(1 - u) on [0,1]^2, homogeneous
 *   Neumann, n x n vertex grid including the boundary (spacing 1/(n-1)); param = {eps, alpha, gamma}
 *   (section 4: 1/100, -10, 100).  N = n^2.
 * KIOPS_PDE_GRAY_SCOTT2D: u_t = d_u Lap u - u v^2 + a (1 - u), v_t = d_v Lap v + u v^2 - (a + b) v on the
 *   periodic unit square, grid x = i/n; param = {d_u, d_v, a, b} (section 4: 0.2, 0.1, 0.04, 0.06).
 *   N = 2 n^2, species-blocked [u; v].
 * Second-order centred differences, x fastest. */
typedef struct {
  int kind;                 /* KIOPS_PDE_* */
  int64_t n;                /* points per dimension (>= 2) */
  double param[4];
} kiops_pde;

typedef struct {
  int64_t steps;            /* time steps taken */
  int64_t kiops_calls;      /* phi-function solves */
  int64_t matvecs, substeps, rejected;  /* summed over the solves */
  int m_last[3];            /* final Krylov dimension of each call slot of the last step */
} kiops_integrate_stats;

/* f = f(u) of the test problem (device vectors of N FP64 values).  Waits for the context's stream. */
kiops_status kiops_pde_rhs(kiops_ctx* ctx, const kiops_pde* pde, const double* u, double* f);

/* Integrate from t0 to t1 > t0 in nsteps equal steps with the scheme KIOPS_EPIRK4S3 / _EPIRK4S3A /
 * _EXPRB5S3; u (device, N FP64) holds u(t0) on entry and u(t1) on return.  tol is each solve's tolerance,
 * m_init the first step's starting Krylov dimension.  The context allocates its integrator workspace
 * (about 16 N FP64 values) on first use.  Errors of a solve are returned as they are (stats then count
 * the steps completed). */
kiops_status kiops_integrate(kiops_ctx* ctx, const kiops_pde* pde, int scheme, double t0, double t1, int64_t nsteps,
                             double tol, int m_init, double* u, kiops_integrate_stats* stats);

/* Self-test of the bounded device-side waits (the paper has no counterpart): one thread block of a two-block
 * team enters the team barrier that every solve uses; the second arrival never comes, so after timeout_s
 * (0 < timeout_s <= 5) the wait gives up, raises the abort flag and the kernel returns.  Returns
 * KIOPS_ETIMEOUT when that happened as designed (the context stays usable), KIOPS_ECUDA otherwise. */
kiops_status kiops_selftest_wait_timeout(kiops_ctx* ctx, double timeout_s);

/* Measured FP64 throughput of the context's GPU in flop/s (the paper has no counterpart: the peak the
 * FP64-bound phases of the solver are reported against).  Two or four blocks of 256 threads per SM, every
 * thread running 8 or 16 independent chains of dependent FP64 fused multiply-adds (2 flops each); the best
 * of three timed launches of each shape after a warm-up, on the context's stream.  Allocates and frees a
 * small result buffer. */
kiops_status kiops_probe_fp64(kiops_ctx* ctx, double* flops_per_s);

/* Size of the fixed device scratch used by kiops_solve_noalloc (bytes). */
#define KIOPS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* kiops_solve without any memory allocation.  Some callers cannot let a library allocate device memory
 * while they run: applications whose device memory is owned by their own pool or allocator (a cudaMalloc
 * behind their back escapes their accounting, fragments their pool and synchronises the whole device),
 * and real-time or embedded hosts that forbid allocation after start-up (cudaMalloc may block for an
 * unbounded time).  This entry point serves them.  (The paper has no counterpart: it is an interface
 * property, not part of the method.)
 *
 * Same arguments and result as kiops_solve with prec = KIOPS_FP64; the solve runs on one thread block.
 * Instead of the context's cudaMalloc'd workspace it uses one file-scope device array of
 * KIOPS_NOALLOC_SCRATCH_BYTES, which every GPU that loads this library holds until the process exits.
 * The caller still passes b and w.  Requests whose workspace (Krylov basis of (m_max+1) x (N+p) FP64
 * values, Hessenberg and exponential work matrices) does not fit are rejected with KIOPS_EINVAL and a
 * message giving the bytes needed; with m_max = 128 roughly N + p <= 30000 fits.
 * Set-up: the first call on a device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture.  Every call shares the one array and
 * it keeps the previous call's contents (the counters it needs are cleared on each call): calls whose
 * GPU work overlaps (from several streams, threads or contexts on the same device) race and give
 * undefined results.  The call copies the stats back and waits for its stream before returning. */
kiops_status kiops_solve_noalloc(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b,
                                 double tol, int m_init, int m_o, double* w, kiops_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* KIOPS_H */
