// Device side of the KIOPS solver for GB300 (sm_103a).
//
// One kernel template runs Algorithm 1 (Task II) of Gaudreault, Rainwater & Tokman (JCP 372, 2018)
// end to end on the device: setup (section 3.7), start vector (Algorithm 1), IOP steps
// (Algorithm 2), the small exponential of tau H~ (eqs 37-38), the estimate and acceptance (eqs 36, 39),
// Algorithm 4 with sections 3.6.1-3.6.2, and the update w = beta V F(:,1) (Algorithm 3, Task II).
//
// Two execution "teams" share that code:
//   GridTeam  one persistent cooperative launch spreads every vector phase over all blocks of the GPU;
//             phases are separated by a counter barrier with a deadline; every block reduces the
//             published per-block partial sums in the same fixed order, so every block holds bitwise
//             identical scalars and takes identical control decisions without broadcasting them.
//   CtaTeam   one thread block owns a whole solve (batches of independent problems, small problems).
//
// Nothing here is a dense contraction over the large dimension, so no tensor cores are used: the vector
// phases are bandwidth / FP64-pipe bound and the small exponential is an FP64 dense computation spread
// over the blocks of the team.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

// A translation unit that builds the kernels with another block size (KIOPS_THREADS) also gives them their
// own namespace (KIOPS_DEV_NS), so that no kernel or device function of one size shadows the other.
#ifndef KIOPS_DEV_NS
#define KIOPS_DEV_NS kiops_dev
#endif
namespace KIOPS_DEV_NS {

#ifndef KIOPS_THREADS
#define KIOPS_THREADS 256
#endif
constexpr int kThreads = KIOPS_THREADS;  // threads per block (256 or 512)
constexpr int kWarps = kThreads / 32;
// Kernel variants of the 2D several-tiles path with bulk tensor copies: none, any tile shape / species
// count / p, or compiled for 32 x 16 tiles, two species and p = 3.
constexpr int kTmaNone = 0, kTmaGeneral = 1, kTmaFixed = 2;
// blocks per SM the register budget is sized for (two of 256 threads or one of 512: 128 registers a thread)
constexpr int kMinBlocks = kThreads <= 256 ? 2 : 1;
constexpr int kMaxM = 256;                 // largest m_max
constexpr int kMaxN = kMaxM + 1;           // largest exponential size n = j + 1
constexpr int kMaxP = 16;                  // largest p
constexpr int kRegK = 8;                   // accumulators per thread per reduction pass
constexpr int kChunk = 3;                  // window vectors handled per pass (2*3 + 1 <= kRegK)
constexpr int kMaxWin = kMaxM + 1;         // largest orthogonalisation window
constexpr int kMaxRed = 2 * kMaxWin + 1;   // largest reduction width
constexpr int kTile = 8;                   // dense matmul tile edge
constexpr int kMaxDeg = 8;                 // entries of the Taylor degree table
constexpr int kGramRing = 8;               // Gram rows kept in shared memory (m_o <= kGramRing)
// elements per pass of the several-tiles 2D loops, which read global memory (the loads of a pass are
// issued together): products (six values an element) and finalisation (three or four)
template <typename T>
constexpr int kBatch = sizeof(T) == 4 ? 4 : 2;
template <typename T>
constexpr int kBatchFin = sizeof(T) == 4 ? 8 : 4;
constexpr int kMaxTimes = 32;              // Task I: largest number of output times

enum : int { ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ENOTCONV = 3, ST_ETIMEOUT = 4, ST_ECUDA = 5 };
enum : int { OP_CSR = 0, OP_ST2D = 1, OP_ST3D = 2 };

struct OpDesc {
  int kind;
  int64_t n;
  const int32_t* rowptr;
  const int32_t* colind;
  const double* vals;
  int64_t nx, ny, nz;
  int nspecies;
  int bc;                    // 0 homogeneous Dirichlet, 1 periodic, 2 homogeneous Neumann (reflection)
  double coef[2][7];
  float coef_f[2][7];        // the same coefficients rounded to FP32 (FP32 basis)
  const double* diag[2][2];
  // 2D stencils with shared coupling fields: entry (s, q) of the pointwise block is
  // fma(dweight[s][q], field[dfield[s][q]], dconst[s][q]) (dconst alone for dfield -1); diag then points at
  // these entries as the operator wrote them, and the staged tile path reads the nfields planes instead.
  int nfields;
  int dfield[2][2];
  double dconst[2][2], dweight[2][2];
  const double* field[2];
};

// Stencil coefficients in the basis precision (FP64 -> FP32 conversions run at the FP64 rate on this GPU,
// so the FP32 copies are made once on the host).
template <typename T>
__device__ __forceinline__ const T* coef_ptr(const OpDesc& op, int s) {
  if constexpr (sizeof(T) == 4) return op.coef_f[s];
  else return op.coef[s];
}

// Truncated Taylor degrees evaluated by Paterson-Stockmeyer: deg = r*q - 1 with r-1 matmuls for the
// powers X^2..X^r and q-1 Horner matmuls in X^r; theta = largest ||X||_1 whose truncation tail
// sum_{k > deg} theta^k / k! stays below the unit roundoff 2^-53.
struct TaylorTable {
  int count;
  int deg[kMaxDeg];
  int r[kMaxDeg];
  int q[kMaxDeg];
  double theta[kMaxDeg];
  double invfact[64];  // 1/k! by repeated division (k <= largest degree)
};

struct TraceRec {
  int64_t substep;
  int j, accepted, breakdown, m_new;
  double tau, t_now, eps, omega, tau_new;
  double cost_a, cost_b;
  double hnorm;
};

struct SolveArgs {
  OpDesc op;
  int64_t N;
  int p;
  int64_t ldv;               // stride between basis vectors (elements)
  double T_end, tol;
  int m_init, m_min, m_max, m_o;
  int normalize;
  double bd_tol;
  int64_t max_substeps, max_iters;
  const double* b[kMaxP + 1];
  double* w;
  void* V;                   // (m_max + 1) vectors of ldv elements (double or float)
  double* H;                 // (m_max + 2)^2, row-major, 1-based H(i,k) at [(i-1)*(m_max+2) + k-1]
  double* gram;              // (m_max + 1) * m_o : <v_i, v_{i-o}> at [(i-1)*m_o + o]
  double* mats;              // expm work: (r_max + 2) matrices of (m_max+1)^2
  double* fvec;              // F(:,1) in [0, m_max+1), F(j, j+1) at [m_max+1]
  double* partials;          // 2 * grid * kMaxRed (grid engine only)
  unsigned int* bar;         // barrier counter (grid engine only)
  int* abort_flag;           // nonzero: a block gave up waiting (grid engine only)
  long long timeout_ns;
  int64_t* stats;            // substeps, rejected, matvecs, iterations, expm_calls, m_last, status
  double* stats_d;           // err_est
  TraceRec* trace;
  int64_t trace_cap;
  int64_t* trace_len;
  long long* prof;           // non-NULL: cycles spent per phase, rank 0 view (16 counters)
  TaylorTable tt;
  int scenario;              // 1: the cheaper scenario of eq 40 replaces Algorithm 4's change of m
  double nz_op;              // stored nonzeros of A (nz in eq 41)
  // 2D stencils: lagged normalisation on 2D tiles (one barrier per Krylov step), see fused_st2d_phase
  int fused;                 // 1: use the tiled lagged path
  int tile_gx, tile_gy, tile_w, tile_h;
  // fused path, dynamic shared memory (all of it reused by the exponential, which invalidates it):
  //   [ring: max(ring_n, 1) halo'd tiles][stage: one halo'd tile][table: one code per halo'd tile point]
  //   [cache: (p + ns) values per tile point]
  int ring_n;                // finalised tiles of the last ring_n basis vectors (0: only v_j's tile is kept)
  int stage_on;              // prefetch the raw x_{j+1} tile + halo with cp.async (needs the table)
  int cache_on;              // keep the tile's B columns and coupling fields in shared memory
  int sm_stage, sm_tbl, sm_cache;  // offsets (doubles) in dynamic shared memory
  void* raw;                 // two raw vectors x_{j+1} of ldv elements (ring, fused path only)
  float* bf;                 // FP32 basis: B columns as floats, column t = b_{p-t} at bf + t*ldv
  float* df;                 // FP32 basis: pointwise coupling fields as floats, (s*ns + q)*npts (stencils)
  int prec;                  // 0 FP64 basis, 1 FP32 basis (runtime dispatch in the server kernel)
  int n_times;               // Task I: output times (0 = Task II, the single result in w)
  double times[kMaxTimes];   // Task I: T(1) < ... < T(end) = T_end
  double* wout[kMaxTimes];   // Task I: outputs (wout[n_times-1] == w holds the running state)
  unsigned long long ticket; // serving: written to the completion word when the solve is done
  int expm_only;             // 1: compute exp(a) of an n x n matrix only (kiops_expm)
  int expm_n;
  const double* expm_in;
  double* expm_out;
  // several-tiles 2D path with bulk tensor (TMA) staging of each tile's operands (grid engine only), see
  // fused_st2d_tma.  The tile shape is tile_w x tile_h; halo'd operands are copied as boxes of tma_bw x
  // tma_bh points per species starting at (x0 - tma_pad, y0 - 1), so that the box's x coordinate stays
  // 16-byte aligned; own-point operands as tile_w x tile_h boxes.
  int tma_on;
  int tma_stages;            // tiles in flight per block (shared-memory stages)
  int tma_prefetch;          // issue(k) also fetches tile k + tma_prefetch into L2 (0: none; > tma_stages)
  int tma_pad;               // 16 bytes of elements (4 FP32, 2 FP64)
  int tma_bw, tma_bh;
  int tma_nf;                // coupling-field planes staged per tile
  int tma_fidx[2][2];        // plane of the coupling field (s, q) among the staged ones, -1 if none
  // per species, in the basis precision: the centre coefficient plus the constant of the own entry, the weight
  // of the own entry's plane, the constant and the weight of the other species' entry (a plane given as the
  // entry itself: the centre coefficient, 1, 0, 1)
  alignas(16) float tma_aff_f[2][4];
  alignas(16) double tma_aff_d[2][4];
  int tma_stage_bytes, tma_box_bytes, tma_off_f, tma_off_b, tma_off_d, tma_bar_off;
  int tma_side_off;          // kThreads x 4 elements: per-thread landing slots of an edge tile's wrapped halo
  int tile_d, tile_gz, tma_bd;  // 3D stencils: tile depth, tiles along z, box depth (tile_d + 2)
  const void* tmaps;         // the kernel parameter's tensor maps (basis, raw ring, B columns, coupling fields)
  void* tma_b;               // B columns b_{p-t} at t * ldv in the basis precision (FP32: bf; FP64: a copy)
  void* tma_f;               // coupling fields in the basis precision, tma_nf planes of nx * ny points
};

// ------------------------------------------------------------------------------------------------
// low-level helpers
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// ceil(log2(x)) for x > 0, exact (frexp gives x = f 2^e, f in [0.5, 1)).
__device__ __forceinline__ int ceil_log2(double x) {
  int e;
  double f = frexp(x, &e);
  return f == 0.5 ? e - 1 : e;
}

// Cost model of section 3.2.  Multiplications of Higham's scaling-and-squaring Pade method (the
// algorithm the paper cites for its exponential) for a matrix of 1-norm x: pi_m = 2, 3, 4, 5, 6 for
// the degrees 3, 5, 7, 9, 13 chosen by the thresholds theta_m of Higham (2005, Table 2.3), plus the
// squarings of the degree-13 branch.
__device__ __forceinline__ double pade_mults(double x) {
  const double theta[5] = {1.495585217958292e-2, 2.539398330063230e-1, 9.504178996162932e-1, 2.097847961257068e0,
                           5.371920351148152e0};
  for (int d = 0; d < 4; ++d)
    if (x <= theta[d]) return (double)(2 + d);
  const int s = x > theta[4] ? ceil_log2(x / theta[4]) : 0;
  return 6.0 + (s > 0 ? s : 0);
}

// eq 40 with eq 41 (m Krylov steps) and eq 42 (the exponential); 0 when no interval is left.
__device__ __forceinline__ double scenario_cost(double rem, double tau, double m, double N, double p, double nz,
                                                double nmult) {
  if (!(rem > 0.0) || !(tau > 0.0)) return 0.0;
  const double iop = m * ((2.0 * nz + (2.0 * p - 1.0) * N + p) + 8.0 * (N + p)) - 4.0 * (N + p) + 3.0 * (N + p) * m;
  const double ex = nmult * (2.0 * (m + p) - 1.0) * (m + p) * (m + p);
  return ceil(rem / tau) * (iop + ex);
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------------------------------------
// Teams
// ------------------------------------------------------------------------------------------------
struct GridTeam {
  int rank, size;
  unsigned int* ctr;
  int* abort_flag;
  long long timeout_ns;
  unsigned int epoch;
  // Counter barrier: every block adds 1 (release) and waits (acquire) until the counter reaches
  // size * epoch.  A wait longer than timeout_ns raises the abort flag; every waiter also leaves when it
  // sees the flag.  Returns false when the team must stop.
  __device__ bool sync(int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
      epoch += 1;
      red_release_add(ctr, 1u);  // release: orders this block's writes (bar.sync above) before the arrival
      const unsigned int target = epoch * (unsigned int)size;
      const long long t0 = global_ns();
      int ok = 1;
      unsigned int spins = 0;
      while ((int)(ld_acquire(ctr) - target) < 0) {
        if (((++spins) & 63u) == 0u) {
          if (ld_volatile_int(abort_flag)) { ok = 0; break; }
          if (global_ns() - t0 > timeout_ns) {
            atomicExch(abort_flag, ST_ETIMEOUT);
            ok = 0;
            break;
          }
        }
      }
      *s_flag = ok;  // the acquire load above orders the reads that follow the bar.sync below
    }
    __syncthreads();
    return *s_flag != 0;
  }
};

struct CtaTeam {
  int rank = 0, size = 1;
  __device__ bool sync(int*) {
    __syncthreads();
    return true;
  }
};

// ------------------------------------------------------------------------------------------------
// Shared control state: identical in every block of a grid team.
// ------------------------------------------------------------------------------------------------
struct Ctl {
  double t_now, tau, beta, nu, mu, s, s2, rs, eps_last, nx2_pre;
  double kappa, qp1_est, prev_tau, prev_omega, prev_eps;
  int m, j, i0, nwin, breakdown, recompute, accepted, done, status, have_prev, prev_j, sync_ok;
  int64_t substeps, rejected, matvecs, iters, expm_calls;
  // expm selection
  int deg_i, n_exp, s_sq;
  double xscale;
  double hcoef[kMaxWin];        // MGS coefficients h(i0..j, j)
  double colabs[kMaxM + 2];     // 1-based: sum_i |h(i,k)| over the window entries of column k
  double sub[kMaxM + 2];        // 1-based: h(k+1, k)
  double tail[kMaxP];           // tail of the vector being multiplied
  double fin_h[kChunk];         // fused path: MGS coefficients and 1/s that finalise the pending raw vector
  double fin_rs;
  int fin_pending, fin_i0, fin_nwin;
  float yhi[kMaxN], ylo[kMaxN];  // FP32 basis: update weights split into float hi + lo
  double yint[kMaxN];           // Task I: first column of exp(tau~ H_j) for an intermediate output
  double t_sub, tau_sub;        // start time and step of the substep that was just accepted
  int ring_lo;                  // fused path: v_ring_lo .. v_j are in the shared-memory ring
  double hnorm;                 // ||tau H~||_1 of the last exponential (cost model)
  int pre_j;                    // fused path: the stage holds raw x_{pre_j} (0: nothing staged)
  int cache_ok;                 // fused path: the B / coupling cache is filled
  int tbl_ok;                   // fused path: the halo index table is filled
  double vtail[kGramRing][kMaxP];  // fused path: tail of v_k (basis precision) in row k % kGramRing
  int ell;                      // Task I: next output index (Algorithm 1)
  double ntail[kMaxP];          // nu * tail (the B-block weights of the step)
  float ntail_f[kMaxP];         // the same weights rounded to FP32 (FP32 basis)
  double gram[kGramRing][kGramRing];  // row i % kGramRing: <v_i, v_{i-o}>, o = 0..m_o-1 (m_o <= kGramRing)
  double hc[kMaxP + 1];         // Horner epilogue coefficients
  double red[kMaxRed];          // results of the last all-reduce
  double blk[kMaxRed];          // this block's partial sums
  double wred[kWarps][kRegK];
  float wff[kWarps][kRegK][2];  // FP32 basis: per-warp float-float sums of the step's dots
  long long prof[16];           // cycles by phase (rank 0, thread 0) when profiling
  long long prof_last;
  unsigned int tma_seq;         // TMA path: tile loads this block has issued and consumed (barrier phases)
  int tma_init;                 // TMA path: the stage barriers are initialised
};

// Phase profiling: thread 0 of rank 0 charges the cycles since the previous tick to a category.
// The step's B-block weights in the basis precision.
template <typename T>
__device__ __forceinline__ const T* ntail_ptr(const Ctl& c) {
  if constexpr (sizeof(T) == 4) return c.ntail_f;
  else return c.ntail;
}

#define KIOPS_TICK(cat)                          \
  do {                                           \
    if (prof_on && threadIdx.x == 0) {           \
      const long long t_ = clock64();            \
      c.prof[(cat)] += t_ - c.prof_last;         \
      c.prof_last = t_;                          \
    }                                            \
  } while (0)

// Sum eight per-lane values over a warp with a transpose (butterfly) reduction: at the exchange with
// lane ^ 16 each lane keeps half of the values and adds its partner's copy of that half, then halves
// again at ^ 8 and ^ 4; two plain exchanges (^ 2, ^ 1) finish.  9 double adds per warp instead of the
// 40 of eight separate shuffle trees (a warp-wide FP64 add is expensive on this GPU).  On return lane l
// holds the sum of value index 4*b4 + 2*b3 + b2 (bits of l); the order of additions is fixed.
__device__ __forceinline__ double warp_transpose_sum8(const double (&v)[kRegK]) {
  const int lane = threadIdx.x & 31;
  const bool h1 = lane & 16, h2 = lane & 8, h3 = lane & 4;
  double a[4], b2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double send = h1 ? v[i] : v[i + 4];
    const double keep = h1 ? v[i + 4] : v[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double send = h2 ? a[i] : a[i + 2];
    const double keep = h2 ? a[i + 2] : a[i];
    b2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const double send = h3 ? b2[0] : b2[1];
  const double keep = h3 ? b2[1] : b2[0];
  double r = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

// Reduce acc[0..K) (K <= kRegK) over the first `nwarps` warps of the block into dst[0..K) (shared).
// Fixed order: butterfly within each warp, then warps 0, 1, 2, ... in sequence.
// Destination of slot k of the step's dot accumulators (<v_i, x> in slots 0..kChunk-1, <v_j, v_i> in
// kChunk.., ||x||^2 in 2 kChunk) in the compact all-reduce layout [<v_i, x>: nwin][||x||^2][<v_j, v_i>: nwin];
// -1 for unused slots.  nwin < 0 keeps slot k at k.
__device__ __forceinline__ int compact_slot(int k, int nwin) {
  if (nwin < 0) return k;
  if (k < nwin) return k;
  if (k == 2 * kChunk) return nwin;
  if (k >= kChunk && k < kChunk + nwin) return nwin + 1 + (k - kChunk);
  return -1;
}

__device__ __forceinline__ void block_reduce_to(Ctl& c, const double (&acc)[kRegK], int K, double* dst,
                                                int nwarps = kWarps, int nwin = -1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < nwarps) {
    const double r = warp_transpose_sum8(acc);
    if ((lane & 3) == 0) c.wred[warp][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = r;
  }
  __syncthreads();
  if (threadIdx.x < K) {  // pairwise tree over the warps (fixed shape for a given nwarps)
    double v[kWarps];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) v[w] = w < nwarps ? c.wred[w][threadIdx.x] : 0.0;
#pragma unroll
    for (int st = 1; st < kWarps; st <<= 1)
#pragma unroll
      for (int w = 0; w + st < kWarps; w += 2 * st) v[w] += v[w + st];
    const int d = compact_slot(threadIdx.x, nwin);
    if (d >= 0) dst[d] = v[0];
  }
  __syncthreads();
}
__device__ __forceinline__ void block_reduce(Ctl& c, const double (&acc)[kRegK], int K, int off) {
  block_reduce_to(c, acc, K, c.blk + off);
}

// Finish an all-reduce of blk[0..K) into red[0..K).  Grid: publish, barrier, then every block sums the
// published partials over ranks 0..size-1 in the same order.  Returns false if the team must stop.
template <class Team>
__device__ bool finish_reduce(Team& team, Ctl& c, double* partials, int& parity, int K, bool prof_on = false);

template <>
__device__ inline bool finish_reduce<CtaTeam>(CtaTeam& team, Ctl& c, double*, int&, int K, bool) {
  for (int k = threadIdx.x; k < K; k += kThreads) c.red[k] = c.blk[k];
  __syncthreads();
  return true;
}

// Sum the published partials of all ranks into red[0..K): value k of rank r is at buf[k * size + r] (a
// warp's loads of one value are contiguous); thread t loads rank t's partials (ranks t + kThreads, ...
// added on top), then the fixed block tree over only as many warps as hold ranks.
__device__ inline void grid_sum_partials(GridTeam& team, Ctl& c, const double* buf, int K) {
  const int nw = team.size >= kThreads ? kWarps : (team.size + 31) / 32;
  for (int k0 = 0; k0 < K; k0 += kRegK) {
    const int cnt = K - k0 < kRegK ? K - k0 : kRegK;
    double acc[kRegK];
    const int r = threadIdx.x;
    const double* src = buf + (size_t)k0 * team.size;  // value k of rank r at src[k * size + r]
#pragma unroll
    for (int k = 0; k < kRegK; ++k) acc[k] = (r < team.size && k < cnt) ? src[(size_t)k * team.size + r] : 0.0;
    for (int r2 = r + kThreads; r2 < team.size; r2 += kThreads) {
#pragma unroll
      for (int k = 0; k < kRegK; ++k)
        if (k < cnt) acc[k] += src[(size_t)k * team.size + r2];
    }
    block_reduce_to(c, acc, cnt, c.red + k0, nw);
  }
}

template <>
__device__ inline bool finish_reduce<GridTeam>(GridTeam& team, Ctl& c, double* partials, int& parity, int K,
                                        bool prof_on) {
  double* buf = partials + (size_t)parity * team.size * kMaxRed;
  for (int k = threadIdx.x; k < K; k += kThreads) buf[(size_t)k * team.size + team.rank] = c.blk[k];
  if (!team.sync(&c.sync_ok)) return false;
  KIOPS_TICK(11);
  grid_sum_partials(team, c, buf, K);
  parity ^= 1;
  return true;
}

// finish_reduce followed by work that needs the barrier but not the sums (the fused path issues its
// prefetch of the next raw tile there, overlapping the coefficient computation).
template <class Team, class Hook>
__device__ __forceinline__ bool finish_reduce_hook(Team& team, Ctl& c, double* partials, int& parity, int K,
                                                   bool prof_on, Hook&& hook) {
  if constexpr (std::is_same<Team, GridTeam>::value) {
    double* buf = partials + (size_t)parity * team.size * kMaxRed;
    for (int k = threadIdx.x; k < K; k += kThreads) buf[(size_t)k * team.size + team.rank] = c.blk[k];
    if (!team.sync(&c.sync_ok)) return false;
    KIOPS_TICK(11);
    grid_sum_partials(team, c, buf, K);
    hook();
    parity ^= 1;
    return true;
  } else {
    if (!finish_reduce<Team>(team, c, partials, parity, K, prof_on)) return false;
    hook();
    return true;
  }
}

// ------------------------------------------------------------------------------------------------
// Operators: row r of A x (matrix-free; Algorithm 2 applies A to the first N entries).
// ------------------------------------------------------------------------------------------------
// Index just outside [0, n) under the operator's boundary rule; returns -1 where the value is 0.
__device__ __forceinline__ int64_t bc_index(int bc, int64_t i, int64_t n) {
  if (i >= 0 && i < n) return i;
  if (bc == 1) return i < 0 ? i + n : i - n;
  if (bc == 2) return i < 0 ? -i : 2 * (n - 1) - i;
  return -1;
}

template <typename T>
__device__ __forceinline__ T st_val(const OpDesc& op, const T* x, int s, int64_t ix, int64_t iy, int64_t iz,
                                    int64_t nz) {
  ix = bc_index(op.bc, ix, op.nx);
  iy = bc_index(op.bc, iy, op.ny);
  iz = bc_index(op.bc, iz, nz);
  if (ix < 0 || iy < 0 || iz < 0) return T(0);
  return x[(int64_t)s * op.nx * op.ny * nz + (iz * op.ny + iy) * op.nx + ix];
}

template <typename T, int KIND>
__device__ __forceinline__ T apply_row(const OpDesc& op, const T* x, int64_t r) {
  if (KIND == OP_CSR) {
    T acc = T(0);
    const int32_t k1 = __ldg(op.rowptr + r + 1);
    for (int32_t k = __ldg(op.rowptr + r); k < k1; ++k) acc += T(__ldg(op.vals + k)) * x[__ldg(op.colind + k)];
    return acc;
  } else if (KIND == OP_ST2D) {
    const int64_t npts = op.nx * op.ny;
    const int s = (int)(r / npts);
    const int64_t pt = r - (int64_t)s * npts;
    const int64_t iy = pt / op.nx, ix = pt - iy * op.nx;
    const T* c = coef_ptr<T>(op, s);
    T acc = c[0] * x[r];
    acc += c[1] * st_val<T>(op, x, s, ix - 1, iy, 0, 1);
    acc += c[2] * st_val<T>(op, x, s, ix + 1, iy, 0, 1);
    acc += c[3] * st_val<T>(op, x, s, ix, iy - 1, 0, 1);
    acc += c[4] * st_val<T>(op, x, s, ix, iy + 1, 0, 1);
    for (int q = 0; q < op.nspecies; ++q)
      if (op.diag[s][q]) acc += T(__ldg(op.diag[s][q] + pt)) * x[(int64_t)q * npts + pt];
    return acc;
  } else {
    const int64_t nxy = op.nx * op.ny;
    const int64_t iz = r / nxy, rem = r - iz * nxy;
    const int64_t iy = rem / op.nx, ix = rem - iy * op.nx;
    const T* c = coef_ptr<T>(op, 0);
    T acc = c[0] * x[r];
    acc += c[1] * st_val<T>(op, x, 0, ix - 1, iy, iz, op.nz);
    acc += c[2] * st_val<T>(op, x, 0, ix + 1, iy, iz, op.nz);
    acc += c[3] * st_val<T>(op, x, 0, ix, iy - 1, iz, op.nz);
    acc += c[4] * st_val<T>(op, x, 0, ix, iy + 1, iz, op.nz);
    acc += c[5] * st_val<T>(op, x, 0, ix, iy, iz - 1, op.nz);
    acc += c[6] * st_val<T>(op, x, 0, ix, iy, iz + 1, op.nz);
    if (op.diag[0][0]) acc += T(__ldg(op.diag[0][0] + r)) * x[r];
    return acc;
  }
}

// Per-thread accumulation of the step's dot products.  FP64 basis: fused multiply-adds in FP64.  FP32
// basis: compensated float-float accumulation (TwoProduct with fmaf and TwoSum; Ogita, Rump & Oishi,
// SIAM J. Sci. Comput. 26 (2005), algorithm Dot2), which returns the sum as if accumulated in about twice
// the FP32 precision; the per-thread results are then reduced across threads and blocks in FP64.  On this
// GPU an FP64 operation costs as much pipe time as ~60 FP32 operations.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double v[kRegK];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < kRegK; ++k) v[k] = 0.0;
  }
  __device__ __forceinline__ void add(int k, double a, double b) { v[k] = fma(a, b, v[k]); }
  __device__ __forceinline__ void add_sum(int k, double s) { v[k] += s; }
  // the W products of one 16-byte item (the same as W calls of add)
  template <int W>
  __device__ __forceinline__ void add_item(int k, const double* a, const double* b) {
#pragma unroll
    for (int u = 0; u < W; ++u) v[k] = fma(a[u], b[u], v[k]);
  }
  __device__ __forceinline__ void to_double(double (&out)[kRegK]) const {
#pragma unroll
    for (int k = 0; k < kRegK; ++k) out[k] = v[k];
  }
};
template <>
struct DotAcc<float> {
  float hi[kRegK], lo[kRegK];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < kRegK; ++k) hi[k] = lo[k] = 0.0f;
  }
  __device__ __forceinline__ void add(int k, float a, float b) {
    const float pr = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -pr);  // a*b = pr + pe exactly
    const float t = __fadd_rn(hi[k], pr);
    const float z = __fsub_rn(t, hi[k]);
    const float se = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(t, z)), __fsub_rn(pr, z));  // hi + pr = t + se exactly
    hi[k] = t;
    lo[k] = __fadd_rn(lo[k], __fadd_rn(se, pe));
  }
  // s (a sum of products formed in FP32) added without error: TwoSum into (hi, lo)
  __device__ __forceinline__ void add_sum(int k, float s) {
    const float t = __fadd_rn(hi[k], s);
    const float z = __fsub_rn(t, hi[k]);
    lo[k] = __fadd_rn(lo[k], __fadd_rn(__fsub_rn(hi[k], __fsub_rn(t, z)), __fsub_rn(s, z)));
    hi[k] = t;
  }
  // The W products of one 16-byte item (W = 4 consecutive points): their sum s is formed in FP32 by a
  // chain of FMAs (at most W - 1 roundings, each relative to a partial sum of W terms), then added to
  // (hi, lo) without error as above.  The sum's error is at most about (W - 1) u sum |a b| over the item,
  // and these item errors do not grow with the number of items as a plain FP32 sum's would; it takes
  // 11 FP32 operations per item instead of 10 per product.
  template <int W>
  __device__ __forceinline__ void add_item(int k, const float* a, const float* b) {
    float s = __fmul_rn(a[0], b[0]);
#pragma unroll
    for (int u = 1; u < W; ++u) s = __fmaf_rn(a[u], b[u], s);
    const float t = __fadd_rn(hi[k], s);
    const float z = __fsub_rn(t, hi[k]);
    const float se = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(t, z)), __fsub_rn(s, z));
    hi[k] = t;
    lo[k] = __fadd_rn(lo[k], se);
  }
  __device__ __forceinline__ void to_double(double (&out)[kRegK]) const {
#pragma unroll
    for (int k = 0; k < kRegK; ++k) out[k] = (double)hi[k] + (double)lo[k];
  }
};

// (h, l) += (bh, bl) in float-float arithmetic: TwoSum of the high parts, the low parts added to its error,
// then renormalised (Fast2Sum).
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  const float s = __fadd_rn(h, bh);
  const float bb = __fsub_rn(s, h);
  float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// Block reduction of the step's dot accumulators into blk[0..K).  FP64 basis: block_reduce.  FP32 basis:
// each warp sums its lanes' float-float pairs with float-float additions over a fixed xor tree (FP32
// pipe only: an FP64 operation costs the FP64 pipe as much as ~60 FP32 ones on this GPU), then K threads
// add the warps' pairs in FP64 in warp order.
template <typename T>
__device__ __forceinline__ void block_reduce_dots(Ctl& c, const DotAcc<T>& d, int K, int nwin = -1) {
  if constexpr (sizeof(T) == 8) {
    double acc[kRegK];
    d.to_double(acc);
    block_reduce_to(c, acc, K, c.blk, kWarps, nwin);
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kRegK; ++k)
      if (k < K) {
        float h = d.hi[k], l = d.lo[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float bh = __shfl_xor_sync(0xffffffffu, h, o), bl = __shfl_xor_sync(0xffffffffu, l, o);
          ff_add(h, l, bh, bl);
        }
        if (lane == 0) {
          c.wff[warp][k][0] = h;
          c.wff[warp][k][1] = l;
        }
      }
    __syncthreads();
    if (threadIdx.x < K) {
      double sum = 0.0;
      for (int w = 0; w < kWarps; ++w) sum += (double)c.wff[w][threadIdx.x][0] + (double)c.wff[w][threadIdx.x][1];
      const int dst = compact_slot(threadIdx.x, nwin);
      if (dst >= 0) c.blk[dst] = sum;
    }
    __syncthreads();
  }
}

// B column t (= b_{p-t}) and pointwise coupling entry in the basis precision.
template <typename T>
__device__ __forceinline__ T bcol(const SolveArgs& a, int t, size_t r) {
  if constexpr (sizeof(T) == 4) return a.bf[(size_t)t * a.ldv + r];
  else return __ldg(a.b[a.p - t] + r);
}
// xv + sum_t ntail[t] * B(r, t) in the order t = 0..p-1, with every B value loaded before the first
// product so that the loads overlap (p is a run-time count, the loads would otherwise be serialised).
template <typename T>
__device__ __forceinline__ T add_btail(const SolveArgs& a, const T* ntail, int p, size_t r, T xv) {
  constexpr int kB = 4;
  T bv[kB];
#pragma unroll
  for (int t = 0; t < kB; ++t) bv[t] = t < p ? bcol<T>(a, t, r) : T(0);
#pragma unroll
  for (int t = 0; t < kB; ++t)
    if (t < p) xv = fma(ntail[t], bv[t], xv);
  for (int t = kB; t < p; ++t) xv = fma(ntail[t], bcol<T>(a, t, r), xv);
  return xv;
}

// Asynchronous global -> shared copies of one element (completed by cp_async_wait_all).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Asynchronous global -> shared copy of 16 bytes, cached in L2 only (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// ---- bulk tensor copies (TMA) completed through shared-memory barriers --------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// the initialised barriers become visible to the copy engine's (async) proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the barrier phase of the given parity to complete; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = global_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity))
    if (((++spins) & 63u) == 0u && global_ns() - t0 > timeout_ns) return false;
  return true;
}
// generic-proxy accesses of shared memory are ordered before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// global data written by other blocks before a gpu-scope barrier becomes visible to this block's bulk copies
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void tma_load_4d(void* dst, const void* map, int x, int y, int z, int w, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}
// the box of a 4D / 3D tensor map into L2 only (no shared memory, no completion to wait for)
__device__ __forceinline__ void tma_prefetch_4d(const void* map, int x, int y, int z, int w) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(map), "r"(x), "r"(y),
               "r"(z), "r"(w)
               : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const void* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(map), "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <typename T>
__device__ __forceinline__ T diag_val(const SolveArgs& a, int sp, int q, uint32_t pt) {
  if constexpr (sizeof(T) == 4) {
    const uint32_t npts = (uint32_t)(a.op.nx * a.op.ny * (a.op.kind == OP_ST3D ? a.op.nz : 1));
    return a.df[(size_t)(sp * a.op.nspecies + q) * npts + pt];
  } else {
    return __ldg(a.op.diag[sp][q] + pt);
  }
}

// Row r of the 3D 7-point operator at grid point (ix, iy, iz), r = ix + nx (iy + ny iz).
template <typename T>
__device__ __forceinline__ T apply_row_3d(const SolveArgs& a, const T* __restrict__ x, uint32_t r, uint32_t ix,
                                          uint32_t iy, uint32_t iz) {
  const OpDesc& op = a.op;
  const uint32_t nx = (uint32_t)op.nx, ny = (uint32_t)op.ny, nz = (uint32_t)op.nz, nxy = nx * ny;
  T xm, xp, ym, yp, zm, zp;
  if (op.bc == 2) {
    xm = x[ix == 0 ? r + 1 : r - 1];
    xp = x[ix + 1 == nx ? r - 1 : r + 1];
    ym = x[iy == 0 ? r + nx : r - nx];
    yp = x[iy + 1 == ny ? r - nx : r + nx];
    zm = x[iz == 0 ? r + nxy : r - nxy];
    zp = x[iz + 1 == nz ? r - nxy : r + nxy];
  } else if (op.bc == 1) {
    xm = x[ix == 0 ? r + nx - 1 : r - 1];
    xp = x[ix + 1 == nx ? r + 1 - nx : r + 1];
    ym = x[iy == 0 ? r + nxy - nx : r - nx];
    yp = x[iy + 1 == ny ? r + nx - nxy : r + nx];
    zm = x[iz == 0 ? r + (nz - 1) * nxy : r - nxy];
    zp = x[iz + 1 == nz ? r - (nz - 1) * nxy : r + nxy];
  } else {
    xm = ix > 0 ? x[r - 1] : T(0);
    xp = ix + 1 < nx ? x[r + 1] : T(0);
    ym = iy > 0 ? x[r - nx] : T(0);
    yp = iy + 1 < ny ? x[r + nx] : T(0);
    zm = iz > 0 ? x[r - nxy] : T(0);
    zp = iz + 1 < nz ? x[r + nxy] : T(0);
  }
  const T* c = coef_ptr<T>(op, 0);
  T acc = c[0] * x[r];
  acc = fma(c[1], xm, acc);
  acc = fma(c[2], xp, acc);
  acc = fma(c[3], ym, acc);
  acc = fma(c[4], yp, acc);
  acc = fma(c[5], zm, acc);
  acc = fma(c[6], zp, acc);
  if (op.diag[0][0]) acc = fma(diag_val<T>(a, 0, 0, r), x[r], acc);
  return acc;
}

// Grid coordinates of a row of a 3D stencil, advanced by a fixed number of rows with carries (mixed radix
// nx, ny): the step loops walk rows without a division per row.
struct Coord3 {
  uint32_t ix, iy, iz;
  __device__ __forceinline__ void set(uint32_t r, uint32_t nx, uint32_t nxy) {
    iz = r / nxy;
    const uint32_t rem = r - iz * nxy;
    iy = rem / nx;
    ix = rem - iy * nx;
  }
  // this += s, for s.ix < nx and s.iy < ny (as set() gives)
  __device__ __forceinline__ void add(const Coord3& s, uint32_t nx, uint32_t ny) {
    ix += s.ix;
    uint32_t cy = ix >= nx ? 1u : 0u;
    ix -= cy ? nx : 0u;
    iy += s.iy + cy;
    const uint32_t cz = iy >= ny ? 1u : 0u;
    iy -= cz ? ny : 0u;
    iz += s.iz + cz;
  }
};

// Row r of A x with 32-bit index arithmetic (stencil grids hold fewer than 2^31 points).
template <typename T, int KIND>
__device__ __forceinline__ T apply_row_fast(const SolveArgs& a, const T* __restrict__ x, uint32_t r) {
  const OpDesc& op = a.op;
  if (KIND == OP_CSR) {
    return apply_row<T, KIND>(op, x, (int64_t)r);
  } else if (KIND == OP_ST2D) {
    const uint32_t nx = (uint32_t)op.nx, ny = (uint32_t)op.ny, npts = nx * ny;
    uint32_t sp = 0, pt = r;
    if (op.nspecies == 2 && r >= npts) { sp = 1; pt = r - npts; }
    const uint32_t iy = pt / nx, ix = pt - iy * nx;
    const T* xs = x + (size_t)sp * npts;
    T w, e, so, no;
    if (op.bc == 1) {
      w = xs[ix == 0 ? pt + nx - 1 : pt - 1];
      e = xs[ix + 1 == nx ? pt + 1 - nx : pt + 1];
      so = xs[iy == 0 ? pt + npts - nx : pt - nx];
      no = xs[iy + 1 == ny ? pt + nx - npts : pt + nx];
    } else if (op.bc == 2) {  // reflection: the missing neighbour is the opposite one
      w = xs[ix == 0 ? pt + 1 : pt - 1];
      e = xs[ix + 1 == nx ? pt - 1 : pt + 1];
      so = xs[iy == 0 ? pt + nx : pt - nx];
      no = xs[iy + 1 == ny ? pt - nx : pt + nx];
    } else {
      w = ix > 0 ? xs[pt - 1] : T(0);
      e = ix + 1 < nx ? xs[pt + 1] : T(0);
      so = iy > 0 ? xs[pt - nx] : T(0);
      no = iy + 1 < ny ? xs[pt + nx] : T(0);
    }
    const T* c = coef_ptr<T>(op, (int)sp);
    T acc = c[0] * xs[pt];
    acc = fma(c[1], w, acc);
    acc = fma(c[2], e, acc);
    acc = fma(c[3], so, acc);
    acc = fma(c[4], no, acc);
    for (int q = 0; q < op.nspecies; ++q)
      if (op.diag[sp][q]) acc = fma(diag_val<T>(a, sp, q, pt), x[(size_t)q * npts + pt], acc);
    return acc;
  } else {
    const uint32_t nx = (uint32_t)op.nx, nxy = nx * (uint32_t)op.ny;
    const uint32_t iz = r / nxy, rem = r - iz * nxy;
    const uint32_t iy = rem / nx, ix = rem - iy * nx;
    return apply_row_3d<T>(a, x, r, ix, iy, iz);
  }
}

// ------------------------------------------------------------------------------------------------
// Small dense exponential exp(tau H~) (section 3.3.1, eqs 37-38), spread over the team's blocks.
//
// Scaling and squaring with a truncated Taylor polynomial in Paterson-Stockmeyer form.  The paper uses a
// diagonal Pade approximant; its linear solve is a chain of n dependent pivot steps, each of which would
// need a team-wide barrier, while the Taylor form is made of matrix products only (one barrier each).
// Both approximate exp to the unit roundoff for ||X|| <= theta.
// ------------------------------------------------------------------------------------------------
struct MmEpi {
  int nterms;          // Horner epilogue: + sum_t hc[t] * P_t(i,k), P_0 = I
  const double* pw;    // P_1 at pw, P_t at pw + (t-1) * ldm
  size_t ldm;
};

// Structure of every matrix of the exponential phase: a band (lower bandwidth lo, upper bandwidth up)
// plus a dense last column, and a last row that is zero except its diagonal entry.  tau H~ has lo = 1,
// up = m_o - 1 (Algorithm 2 writes rows j-m_o+1..j+1 of column j) and e_1 in its last column; products
// keep the form with bandwidths added.  Every matrix is written in full (zeros outside the structure), so
// a product only needs the inner index range where both factors can be nonzero.
struct Band {
  int lo, up;
};

__device__ __forceinline__ Band band_product(Band a, Band b, int n) {
  Band c{a.lo + b.lo, a.up + b.up};
  if (c.lo > n - 1) c.lo = n - 1;
  if (c.up > n - 1) c.up = n - 1;
  return c;
}

// C = A B (+ epilogue) for n x n row-major matrices; tiles of kTile x kTile distributed over ranks.
// Tiles outside the band of C are written as zeros without arithmetic.
static __device__ __noinline__ void mm_team(const double* A, Band bA, const double* B, Band bB, double* C, int n, int rank, int size,
                        const Ctl& c, const MmEpi& epi, double* sA, double* sB) {
  const Band bC = band_product(bA, bB, n);
  const int nt = (n + kTile - 1) / kTile;
  constexpr int kParts = kThreads / (kTile * kTile);  // threads per output entry (inner-range stripes)
  static_assert(kParts * kTile * kTile == kThreads && kParts <= 32 && (kParts & (kParts - 1)) == 0, "tile map");
  const int out = threadIdx.x / kParts, part = threadIdx.x % kParts;
  const int ti_l = out / kTile, tk_l = out % kTile;
  for (int tile = rank; tile < nt * nt; tile += size) {
    const int ti = tile / nt, tk = tile - ti * nt;
    const int i0 = ti * kTile, i1 = min(n, i0 + kTile), k0 = tk * kTile, k1 = min(n, k0 + kTile);
    const bool lastcol = k1 == n;
    const bool inband = lastcol || (k0 - (i1 - 1) <= bC.up && i0 - (k1 - 1) <= bC.lo);
    const int row = i0 + ti_l, col = k0 + tk_l;
    if (!inband) {
      if (part == 0 && row < n && col < n) C[(size_t)row * n + col] = 0.0;
      continue;
    }
    // inner range: A(i, l) != 0 needs l in [i - lo, i + up] (or l = n-1, which only meets B's last row,
    // zero outside the last column); B(l, k) != 0 needs l in [k - up, k + lo]
    int l0 = 0, l1 = n - 1;
    if (!lastcol) {
      l0 = max(0, max(i0 - bA.lo, k0 - bB.up));
      l1 = min(n - 1, min(i1 - 1 + bA.up, k1 - 1 + bB.lo));
    }
    const int nl = l1 - l0 + 1;
    for (int e = threadIdx.x; e < kTile * nl; e += kThreads) {
      const int rr = e / nl, l = l0 + (e - rr * nl);
      const int ra = i0 + rr;
      sA[rr * kMaxN + (l - l0)] = ra < n ? A[(size_t)ra * n + l] : 0.0;
      const int l2 = e / kTile, cc = e - l2 * kTile;
      const int cb = k0 + cc;
      sB[l2 * kTile + cc] = cb < n ? B[(size_t)(l0 + l2) * n + cb] : 0.0;
    }
    __syncthreads();
    // four independent chains per thread (FP64 dependent latency is 64 cycles on this GPU)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int l = part;
    for (; l + 3 * kParts < nl; l += 4 * kParts) {
      s0 = fma(sA[ti_l * kMaxN + l], sB[l * kTile + tk_l], s0);
      s1 = fma(sA[ti_l * kMaxN + l + kParts], sB[(l + kParts) * kTile + tk_l], s1);
      s2 = fma(sA[ti_l * kMaxN + l + 2 * kParts], sB[(l + 2 * kParts) * kTile + tk_l], s2);
      s3 = fma(sA[ti_l * kMaxN + l + 3 * kParts], sB[(l + 3 * kParts) * kTile + tk_l], s3);
    }
    for (; l < nl; l += kParts) s0 = fma(sA[ti_l * kMaxN + l], sB[l * kTile + tk_l], s0);
    double s = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = 1; o < kParts; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (part == 0 && row < n && col < n) {
      double e = 0.0;
      if (epi.nterms > 0) {
        e = row == col ? c.hc[0] : 0.0;
        for (int t = 1; t < epi.nterms; ++t) e = fma(c.hc[t], epi.pw[(size_t)(t - 1) * epi.ldm + (size_t)row * n + col], e);
      }
      C[(size_t)row * n + col] = s + e;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// Lagged normalisation for 2D stencils (one barrier per Krylov step).
//
// Step j of Algorithm 2 needs v_j = (1/s)(x_j - sum_i h_i v_i) at this block's points and at their grid
// neighbours.  Instead of a separate normalise pass followed by a grid barrier, each block finalises v_j on
// its 2D tile plus a one-point halo into shared memory (halo points are recomputed by every neighbouring
// block with the same arithmetic), writes the tile's v_j to the basis, and applies A~ from shared memory.
// Raw vectors x_{j+1} go to a two-slot ring so that no block overwrites a value a neighbour still reads.
// The arithmetic of every value is the same as in the unfused path.
// Coordinates (s, y, x) of the flat index e over ns planes of w x h points, stepped by kThreads without
// divisions (one division each at the start).
struct TileWalk {
  int w, h, dx, dy, x, y, s;
  __device__ __forceinline__ TileWalk(int e, int w_, int h_) : w(w_), h(h_) {
    const int plane = w * h;
    s = e / plane;
    const int rem = e - s * plane;
    y = rem / w;
    x = rem - y * w;
    dy = kThreads / w;
    dx = kThreads - dy * w;
  }
  __device__ __forceinline__ void next() {
    x += dx;
    y += dy;
    if (x >= w) {
      x -= w;
      ++y;
    }
    while (y >= h) {
      y -= h;
      ++s;
    }
  }
};

// Fused step on grids with more tiles than blocks: block `rank` finalises and applies tiles rank,
// rank + nblk, ... in turn in one tile buffer, without the shared-memory extras (every operand comes from
// global memory).  The loops take kBatchFin<T> (finalisation) or kBatch<T> (products) elements per pass
// and issue all their loads before the first store (the stores to V and to raw x_{j+1} could alias the loads for the compiler, which would otherwise
// wait for each element's loads in turn); per element the arithmetic and its order, and the order of the
// elements, are those of the one-tile form in fused_st2d_phase.
template <typename T>
__device__ __forceinline__ void fused_st2d_tiles(const SolveArgs& a, Ctl& c, int rank, int nblk, int j, int i0,
                                                 int nwin, T* V, size_t ldv, double* smem, DotAcc<T>& acc,
                                                 bool prof_on) {
  constexpr int U = kBatch<T>;
  constexpr int kB = 4;  // B columns loaded with the pass's other loads (the rest at their use)
  const OpDesc& op = a.op;
  const uint32_t nx = (uint32_t)op.nx, ny = (uint32_t)op.ny, npts = nx * ny;
  const int ns = op.nspecies;
  const int p = a.p;
  const int tid = threadIdx.x;
  const int bc = op.bc;
  T* raw = (T*)a.raw;
  const bool pend = c.fin_pending != 0;
  const T* src = pend ? raw + (size_t)((j - 1) & 1) * ldv : V + (size_t)(j - 1) * ldv;  // v_j before finalising
  T* vj = V + (size_t)(j - 1) * ldv;
  T* xo = raw + (size_t)(j & 1) * ldv;  // raw x_{j+1}
  const int fnw = pend ? c.fin_nwin : 0;
  const T fh0 = fnw > 0 ? T(c.fin_h[0]) : T(0), fh1 = fnw > 1 ? T(c.fin_h[1]) : T(0),
          fh2 = fnw > 2 ? T(c.fin_h[2]) : T(0);
  const T frs = pend ? T(c.fin_rs) : T(1);
  const T* f0 = V + (size_t)((pend ? c.fin_i0 : 1) - 1) * ldv;
  const T* f1 = V + (size_t)((pend ? c.fin_i0 : 1) + (fnw > 1 ? 1 : 0) - 1) * ldv;
  const T* f2 = V + (size_t)((pend ? c.fin_i0 : 1) + (fnw > 2 ? 2 : 0) - 1) * ldv;
  const T* w0 = V + (size_t)(i0 - 1) * ldv;  // dot window of step j (v_j itself comes from the tile buffer)
  const T* w1 = V + (size_t)(i0 + (nwin > 1 ? 1 : 0) - 1) * ldv;
  const T* nt = ntail_ptr<T>(c);
  T* st = (T*)smem;
  const int ntiles = a.tile_gx * a.tile_gy;
  for (int tile = rank; tile < ntiles; tile += nblk) {
    if (tile != rank) __syncthreads();  // the previous tile's products have read the tile buffer
    const int x0 = (tile % a.tile_gx) * a.tile_w, y0 = (tile / a.tile_gx) * a.tile_h;
    const int tw = min(a.tile_w, (int)nx - x0), th = min(a.tile_h, (int)ny - y0);
    const int hw = tw + 2, hh = th + 2, plane = hw * hh, tot = ns * plane, E = ns * tw * th;
    // v_j = (x_j - sum h v) / s over the tile and its one-point halo (halo points recomputed, not stored)
    {
      constexpr int UF = kBatchFin<T>;
      TileWalk wk(tid, hw, hh);
      for (int eb = tid; eb < tot; eb += UF * kThreads) {
        unsigned code[UF];
        T v[UF], a0[UF], a1[UF], a2[UF];
#pragma unroll
        for (int u = 0; u < UF; ++u) {
          const int e = eb + u * kThreads;
          code[u] = ~0u;
          v[u] = a0[u] = a1[u] = a2[u] = T(0);
          if (e < tot) {
            const int sp = wk.s, hy = wk.y, hx = wk.x;
            wk.next();
            int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
            gx = (int)bc_index(bc, gx, nx);
            gy = (int)bc_index(bc, gy, ny);
            const unsigned own = (hx >= 1 && hx <= tw && hy >= 1 && hy <= th) ? 1u : 0u;
            if (gx >= 0 && gy >= 0) {
              code[u] = 2u * ((unsigned)sp * npts + (unsigned)gy * nx + (unsigned)gx) + own;
              const size_t r = code[u] >> 1;
              v[u] = src[r];
              if (pend) {
                a0[u] = f0[r];
                if (fnw > 1) a1[u] = f1[r];
                if (fnw > 2) a2[u] = f2[r];
              }
            }
          }
        }
#pragma unroll
        for (int u = 0; u < UF; ++u) {
          const int e = eb + u * kThreads;
          if (e < tot) {
            T x = v[u];
            if (code[u] != ~0u && pend) {
              x = fma(-fh0, a0[u], x);
              if (fnw > 1) x = fma(-fh1, a1[u], x);
              if (fnw > 2) x = fma(-fh2, a2[u], x);
              x = x * frs;
              if (code[u] & 1u) vj[code[u] >> 1] = x;
            }
            st[e] = x;
          }
        }
      }
    }
    __syncthreads();
    KIOPS_TICK(12);
    // A~ v_j on the tile's own points and the step's dots
    {
      TileWalk wk(tid, tw, th);
      for (int eb = tid; eb < E; eb += U * kThreads) {
        int hu[U];       // index in the tile buffer; species = hu >= plane
        uint32_t ru[U];  // row of x
        T dov[U], dtv[U], bv[U][kB], g0v[U], g1v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * kThreads;
          hu[u] = 0;
          ru[u] = 0;
          dov[u] = dtv[u] = g0v[u] = g1v[u] = T(0);
#pragma unroll
          for (int t = 0; t < kB; ++t) bv[u][t] = T(0);
          if (e < E) {
            const int sp = wk.s, ly = wk.y, lx = wk.x;
            wk.next();
            const uint32_t pt = (uint32_t)(y0 + ly) * nx + (uint32_t)(x0 + lx);
            const uint32_t r = (uint32_t)sp * npts + pt;
            hu[u] = sp * plane + (ly + 1) * hw + (lx + 1);
            ru[u] = r;
            const int qo = 1 - sp;
            if (op.diag[sp][sp] != nullptr) dov[u] = diag_val<T>(a, sp, sp, pt);
            if (ns == 2 && op.diag[sp][qo] != nullptr) dtv[u] = diag_val<T>(a, sp, qo, pt);
#pragma unroll
            for (int t = 0; t < kB; ++t)
              if (t < p) bv[u][t] = bcol<T>(a, t, r);
            if (i0 != j) g0v[u] = w0[r];
            if (nwin > 1 && i0 + 1 != j) g1v[u] = w1[r];
          }
        }
        // FP32 basis: the batch's U elements are one item of the dot accumulators (DotAcc::add_item, one
        // FP32 sum per dot; elements beyond E contribute zeros).  FP64: each element's products are added
        // as they come (the order of fused_st2d_phase's one-tile loop).
        constexpr bool kItem = sizeof(T) == 4;
        T xq[U], cq[U], v0q[U], v1q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          xq[u] = cq[u] = v0q[u] = v1q[u] = T(0);
          if (eb + u * kThreads < E) {
            const int h = hu[u];
            const int sp = h >= plane ? 1 : 0;
            const size_t r = ru[u];
            const int qo = 1 - sp;
            const bool has_own = op.diag[sp][sp] != nullptr, has_oth = ns == 2 && op.diag[sp][qo] != nullptr;
            const T* cf = coef_ptr<T>(op, sp);
            const T ctr = st[h];
            const T cc = has_own ? cf[0] + dov[u] : cf[0];
            T xv = cc * ctr;
            xv = fma(cf[1], st[h - 1], xv);
            xv = fma(cf[2], st[h + 1], xv);
            xv = fma(cf[3], st[h - hw], xv);
            xv = fma(cf[4], st[h + hw], xv);
            if (has_oth) xv = fma(dtv[u], st[h + (qo - sp) * plane], xv);
#pragma unroll
            for (int t = 0; t < kB; ++t)
              if (t < p) xv = fma(nt[t], bv[u][t], xv);
            for (int t = kB; t < p; ++t) xv = fma(nt[t], bcol<T>(a, t, r), xv);
            xo[r] = xv;
            const T v0 = (i0 == j) ? ctr : g0v[u];
            const T v1 = (nwin > 1 && i0 + 1 != j) ? g1v[u] : ctr;
            if constexpr (kItem) {
              xq[u] = xv;
              cq[u] = ctr;
              v0q[u] = v0;
              v1q[u] = nwin > 1 ? v1 : T(0);
            } else {
              acc.add(0, v0, xv);
              acc.add(kChunk, ctr, v0);
              if (nwin > 1) {
                acc.add(1, v1, xv);
                acc.add(kChunk + 1, ctr, v1);
              }
              if (nwin > 2) {  // i0 + 2 == j
                acc.add(2, ctr, xv);
                acc.add(kChunk + 2, ctr, ctr);
              }
              acc.add(2 * kChunk, xv, xv);
            }
          }
        }
        if constexpr (kItem) {
          acc.template add_item<U>(0, v0q, xq);
          acc.template add_item<U>(kChunk, cq, v0q);
          if (nwin > 1) {
            acc.template add_item<U>(1, v1q, xq);
            acc.template add_item<U>(kChunk + 1, cq, v1q);
          }
          if (nwin > 2) {  // i0 + 2 == j
            acc.template add_item<U>(2, cq, xq);
            acc.template add_item<U>(kChunk + 2, cq, cq);
          }
          acc.template add_item<U>(2 * kChunk, xq, xq);
        }
      }
    }
    KIOPS_TICK(13);
  }
}

// 16 bytes of basis-precision values (4 FP32 or 2 FP64): the unit of work of the TMA path's loops.
template <typename T>
struct alignas(16) Vec16 {
  static constexpr int W = 16 / (int)sizeof(T);
  T e[16 / sizeof(T)];
};
template <typename T>
__device__ __forceinline__ Vec16<T> ld16(const T* p) {
  return *(const Vec16<T>*)p;
}
template <typename T>
__device__ __forceinline__ void st16(T* p, const Vec16<T>& v) {
  *(Vec16<T>*)p = v;
}
// 16-byte store to global memory (cached in L2 only: the next step reads it through the copy engine)
__device__ __forceinline__ void stg16(float* p, const Vec16<float>& v) {
  __stcg((float4*)p, make_float4(v.e[0], v.e[1], v.e[2], v.e[3]));
}
__device__ __forceinline__ void stg16(double* p, const Vec16<double>& v) {
  __stcg((double2*)p, make_double2(v.e[0], v.e[1]));
}

// The staged path's centre and coupling constants of species sp (SolveArgs::tma_aff_*), one 16-byte
// shared-memory read (two with an FP64 basis).
template <typename T>
struct Aff4 {
  T cc, wo, ct, wt;
};
template <typename T>
__device__ __forceinline__ Aff4<T> tma_aff(const SolveArgs& a, int sp) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *(const float4*)a.tma_aff_f[sp];
    return {v.x, v.y, v.z, v.w};
  } else {
    const double2 u = *(const double2*)a.tma_aff_d[sp], v = *(const double2*)(a.tma_aff_d[sp] + 2);
    return {u.x, u.y, v.x, v.y};
  }
}

// Fused step on grids with more tiles than blocks, operands staged by bulk tensor copies (TMA).  Block `rank`
// takes tiles rank, rank + nblk, ... in turn; one thread issues each tile's copies into one of tma_stages
// shared-memory stages (completed through that stage's barrier), tma_stages tiles ahead of the tile being
// computed, so the copies of the next tiles overlap the finalisation and products of this one.  Per tile:
//   halo'd boxes (tile + one-point halo, widened in x to a 16-byte aligned start): the vector v_j is built
//   from (raw x_j, or v_j itself on the first step of a substep) and the window vectors of its finalisation
//   (which contain the dot window of step j);
//   own-point boxes: the B columns and the coupling fields.
// Points outside the grid arrive as zeros from the copy, which is the Dirichlet value; for periodic and
// reflected boundaries the halo points the stencil reads there (one row above or below the tile, one column
// left or right of it) take the finalised value at their mapped index in a separate pass over the edge tiles
// only (so that the main loops carry no boundary test): from the tile's own box where the mapped point lies
// in it, else from per-thread slots that cp.async copies fill before the tile's wait.
// The loops take 16 bytes of consecutive points per item (tile widths are multiples of that): 128-bit
// shared-memory loads and global stores, coefficients and B-block weights held in registers.  Per element
// the arithmetic and its order are those of fused_st2d_tiles; the step's dots take each item's products as
// one sum (DotAcc::add_item), accumulated in another order.
// CTW, CTH, CNS, CP > 0 (CP >= 0) fix the tile shape, the species count and p at compile time (a kernel
// instantiation of its own): the loop bounds, the shared-memory offsets and the B-block loop are then
// constants, and a ragged tile at the grid's right or bottom edge runs the whole box with the points beyond
// the grid left out of the stores and the dots.  0 (CP = -1): taken from the arguments.
template <typename T, int CTW = 0, int CTH = 0, int CNS = 0, int CP = -1>
__device__ __forceinline__ void fused_st2d_tma(const SolveArgs& a, Ctl& c, int rank, int nblk, int j, int i0,
                                               int nwin, T* V, size_t ldv, double* smem, DotAcc<T>& acc,
                                               bool prof_on) {
  constexpr int W = Vec16<T>::W;
  constexpr bool kFixed = CTW > 0 && CTH > 0 && CNS > 0;
  const OpDesc& op = a.op;
  const int nx = (int)op.nx, ny = (int)op.ny;
  const uint32_t npts = (uint32_t)nx * (uint32_t)ny;
  const int ns = CNS > 0 ? CNS : op.nspecies;
  const int p = CP >= 0 ? CP : a.p;
  const int tid = threadIdx.x;
  const int bc = op.bc;
  T* raw = (T*)a.raw;
  const bool pend = c.fin_pending != 0;
  T* vj = V + (size_t)(j - 1) * ldv;
  T* xo = raw + (size_t)(j & 1) * ldv;  // raw x_{j+1}
  const int fnw = pend ? c.fin_nwin : 0;
  const T fh0 = fnw > 0 ? T(c.fin_h[0]) : T(0), fh1 = fnw > 1 ? T(c.fin_h[1]) : T(0),
          fh2 = fnw > 2 ? T(c.fin_h[2]) : T(0);
  const T frs = pend ? T(c.fin_rs) : T(1);
  // window boxes: the finalisation window (pending) or the dot window below v_j (first step)
  const int fbase = pend ? c.fin_i0 : i0;
  const int nfb = pend ? fnw : nwin - 1;
  const int wslot0 = i0 - fbase, wslot1 = i0 + 1 - fbase;  // window entries i0, i0 + 1 (when below j)
  // loop invariants in registers (the shared-memory stores of the finalisation go through generic pointers,
  // so values read from shared memory inside the loops would be read again after each store)
  T cfr[2][5], ntr[4];
  int fo_s[2], ft_s[2];
  for (int sp = 0; sp < 2; ++sp) {
    const T* cf = coef_ptr<T>(op, sp < ns ? sp : 0);
#pragma unroll
    for (int k = 0; k < 5; ++k) cfr[sp][k] = cf[k];
    fo_s[sp] = sp < ns ? a.tma_fidx[sp][sp] : -1;
    ft_s[sp] = ns == 2 ? a.tma_fidx[sp][1 - sp] : -1;
  }
  {
    const T* nt = ntail_ptr<T>(c);
#pragma unroll
    for (int t = 0; t < 4; ++t) ntr[t] = t < p ? nt[t] : T(0);
  }
  const T* ntp = ntail_ptr<T>(c);
  const int S = a.tma_stages, A = W;
  const int TW = kFixed ? CTW : a.tile_w, TH = kFixed ? CTH : a.tile_h;
  const int BW = kFixed ? CTW + 2 * W : a.tma_bw, BH = kFixed ? CTH + 2 : a.tma_bh;
  const int bplane = BW * BH, bsz = ns * bplane;  // elements of one halo'd box (all species)
  // elements between window boxes (box bytes rounded up to 128)
  const int fst = kFixed ? (bsz * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T) : a.tma_box_bytes / (int)sizeof(T);
  const int oplane = TW * TH;
  const int gxn = a.tile_gx, ntiles = a.tile_gx * a.tile_gy;
  const int K = rank < ntiles ? (ntiles - rank + nblk - 1) / nblk : 0;
  const int nwin_l = nwin, i0_l = i0, j_l = j;
  // stages and barriers from the first 128-byte aligned shared address (the launch reserves the slack)
  char* sm = (char*)smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
  uint64_t* bars = (uint64_t*)(sm + a.tma_bar_off);
  char* sm_side = sm + a.tma_side_off;
  const char* maps = (const char*)a.tmaps;  // 128 bytes each: basis, raw ring, B columns, fields
  const int tma_nf = a.tma_nf, off_f = a.tma_off_f, off_b = a.tma_off_b, off_d = a.tma_off_d;
  const int stage_bytes = a.tma_stage_bytes;
  const long long timeout_ns = a.timeout_ns;
  const unsigned expect = (unsigned)(bsz * (int)sizeof(T) * (1 + nfb)) +
                          (p > 0 ? (unsigned)(p * ns * oplane * (int)sizeof(T)) : 0u) +
                          (tma_nf > 0 ? (unsigned)(tma_nf * oplane * (int)sizeof(T)) : 0u);
  if (tid == 0 && !c.tma_init) {
    for (int s = 0; s < S; ++s) mbar_init(bars + s, 1);
    mbar_init_fence();
    c.tma_init = 1;
  }
  // raw x_j and v_j - 1 were written by every block before the barrier that opened this step
  fence_proxy_async_all();
  __syncthreads();
  const unsigned q0 = c.tma_seq;
  const int PF = a.tma_prefetch;
  auto prefetch = [&](int k) {  // thread 0: this block's k-th tile of the step into L2
    const int tile = rank + k * nblk;
    const int x0 = (tile % gxn) * TW, y0 = (tile / gxn) * TH;
    if (pend) tma_prefetch_4d(maps + 128, x0 - A, y0 - 1, 0, (j_l - 1) & 1);
    else tma_prefetch_4d(maps, x0 - A, y0 - 1, 0, j_l - 1);
    for (int u = 0; u < nfb; ++u) tma_prefetch_4d(maps, x0 - A, y0 - 1, 0, fbase + u - 1);
    if (p > 0) tma_prefetch_4d(maps + 256, x0, y0, 0, 0);
    if (tma_nf > 0) tma_prefetch_3d(maps + 384, x0, y0, 0);
  };
  auto issue = [&](int k) {  // thread 0: the copies of this block's k-th tile of the step
    if (k + PF < K) prefetch(k + PF);
    const int tile = rank + k * nblk;
    const int st = (int)((q0 + (unsigned)k) % (unsigned)S);
    char* base = sm + (size_t)st * stage_bytes;
    uint64_t* bar = bars + st;
    const int x0 = (tile % gxn) * TW, y0 = (tile / gxn) * TH;
    mbar_arrive_expect_tx(bar, expect);
    if (pend) tma_load_4d(base, maps + 128, x0 - A, y0 - 1, 0, (j_l - 1) & 1, bar);
    else tma_load_4d(base, maps, x0 - A, y0 - 1, 0, j_l - 1, bar);
    for (int u = 0; u < nfb; ++u)
      tma_load_4d(base + off_f + (size_t)u * fst * sizeof(T), maps, x0 - A, y0 - 1, 0, fbase + u - 1, bar);
    if (p > 0) tma_load_4d(base + off_b, maps + 256, x0, y0, 0, 0, bar);
    if (tma_nf > 0) tma_load_3d(base + off_d, maps + 384, x0, y0, 0, bar);
  };
  if (tid == 0) {
    for (int k = S; k < K && k < PF; ++k) prefetch(k);  // later tiles are prefetched by issue(k - PF)
    for (int k = 0; k < K && k < S; ++k) issue(k);
  }
  int done = 0;
  for (int k = 0; k < K; ++k) {
    const int tile = rank + k * nblk;
    const int st = (int)((q0 + (unsigned)k) % (unsigned)S);
    const unsigned par = ((q0 + (unsigned)k) / (unsigned)S) & 1u;
    char* base = sm + (size_t)st * stage_bytes;
    const int x0 = (tile % gxn) * TW, y0 = (tile / gxn) * TH;
    const int tw = min(TW, nx - x0), th = min(TH, ny - y0);  // the tile's extent in the grid (tw: a multiple of W)
    const int tv = tw / W;                                   // own vectors per row
    // the loops' extent: with a fixed shape always the whole box, also on a ragged tile at the grid's right or
    // bottom edge, whose points beyond the grid are the copy's zero fill (computed, never stored or summed)
    const int tvl = kFixed ? TW / W : tv, thl = kFixed ? TH : th;
    const bool edge = bc != 0 && (x0 == 0 || y0 == 0 || x0 + tw == nx || y0 + th == ny);
    // Edge tile of a periodic or reflected grid: the halo points outside the grid that the stencil reads
    // (the row above / below the tile, the column left / right of it; no corners), point e of
    // ns * L in species-major order.  Their values are those at the mapped index: inside this box
    // (reflection: one or two points inside the edge) or elsewhere in the grid (periodic wrap).
    const int ntop = y0 == 0 ? tw : 0, nbot = y0 + th == ny ? tw : 0;
    const int nlft = x0 == 0 ? th : 0, nrgt = x0 + tw == nx ? th : 0;
    const int L = edge ? ntop + nbot + nlft + nrgt : 0;
    // point e: species, box row, box column (points), and the mapped point's row-major offset in a plane and
    // box coordinates
    auto halo_point = [&](int e, int& sp, int& hy, int& hx, size_t& r, int& mbx, int& mby) {
      sp = e / L;
      int q = e - sp * L;
      if (q < ntop) {
        hy = 0, hx = W + q;
      } else if ((q -= ntop) < nbot) {
        hy = th + 1, hx = W + q;
      } else if ((q -= nbot) < nlft) {
        hy = 1 + q, hx = W - 1;
      } else {
        q -= nlft;
        hy = 1 + q, hx = W + tw;
      }
      const int mx = (int)bc_index(bc, x0 - W + hx, nx), my = (int)bc_index(bc, y0 - 1 + hy, ny);
      r = (size_t)sp * npts + (uint32_t)my * nx + (uint32_t)mx;
      mbx = mx - (x0 - W), mby = my - (y0 - 1);
    };
    auto in_box = [&](int mbx, int mby) { return mbx >= 0 && mbx < tw + 2 * W && mby >= 0 && mby < th + 2; };
    T* side = (T*)(sm_side) + tid * 4;  // this thread's landing slots: x_j (or v_j), then the window
    if (edge && tid < ns * L) {
      // the first point of this thread lying outside the box: its sources copied into the landing slots
      // now, so that the global-memory latency overlaps the wait for the tile and its finalisation
      int sp, hy, hx, mbx, mby;
      size_t r;
      halo_point(tid, sp, hy, hx, r, mbx, mby);
      if (!in_box(mbx, mby)) {
        cp_async_elem(side, (pend ? raw + (size_t)((j_l - 1) & 1) * ldv : V + (size_t)(j_l - 1) * ldv) + r);
        const T* f0 = V + (size_t)(fbase - 1) * ldv + r;
        for (int u = 0; u < fnw; ++u) cp_async_elem(side + 1 + u, f0 + (size_t)u * ldv);
      }
    }
    const bool ok = mbar_wait(bars + st, par, timeout_ns);
    KIOPS_TICK(14);
    T* sb = (T*)base;
    const T* fb = (const T*)(base + off_f);
    const T* bb = (const T*)(base + off_b);
    const T* db = (const T*)(base + off_d);
    // v_j = (x_j - sum h v) / s over the tile and its halo, in place in the source box: box rows 0..th+1,
    // vectors 0..tv+1 of each row (box vector c covers the points x0 - W + c W ...)
    if (ok) {
      const int rv = tvl + 2, tot = ns * (thl + 2) * rv;
      TileWalk wk(tid, rv, thl + 2);
      for (int e = tid; e < tot; e += kThreads, wk.next()) {
        const int sp = wk.s, hy = wk.y, cv = wk.x;
        const int bi = sp * bplane + hy * BW + cv * W;
        const int gy = y0 - 1 + hy, gxv = x0 - W + cv * W;
        const bool own = hy >= 1 && hy <= th && cv >= 1 && cv <= tv;  // in the grid: the tile's actual extent
        Vec16<T> v = ld16(sb + bi);
        if (pend) {
          Vec16<T> g0 = ld16(fb + bi), g1, g2;
          if (fnw > 1) g1 = ld16(fb + fst + bi);
          if (fnw > 2) g2 = ld16(fb + 2 * fst + bi);
#pragma unroll
          for (int u = 0; u < W; ++u) {
            T x = fma(-fh0, g0.e[u], v.e[u]);
            if (fnw > 1) x = fma(-fh1, g1.e[u], x);
            if (fnw > 2) x = fma(-fh2, g2.e[u], x);
            v.e[u] = x * frs;
          }
        }
        st16(sb + bi, v);
        if (pend && own) stg16(vj + (size_t)sp * npts + (uint32_t)gy * nx + (uint32_t)gxv, v);
      }
    }
    if (edge) {  // uniform over the block
      // the halo points outside the grid, finalised, over the values the loop above derived from the
      // copy's zero fill: from this box where the mapped point lies in it (finalised above), else from the
      // landing slots (a thread's first point) or global memory
      cp_async_wait_all();
      __syncthreads();
      if (ok) {
        const T* src = pend ? raw + (size_t)((j_l - 1) & 1) * ldv : V + (size_t)(j_l - 1) * ldv;
        const T* f0 = V + (size_t)(fbase - 1) * ldv;  // the finalisation window, consecutive columns
        for (int e = tid; e < ns * L; e += kThreads) {
          int sp, hy, hx, mbx, mby;
          size_t r;
          halo_point(e, sp, hy, hx, r, mbx, mby);
          T x;
          if (in_box(mbx, mby)) {
            x = sb[sp * bplane + mby * BW + mbx];
          } else {
            const bool landed = e == tid;
            x = landed ? side[0] : src[r];
            if (pend) {
              x = fma(-fh0, landed ? side[1] : f0[r], x);
              if (fnw > 1) x = fma(-fh1, landed ? side[2] : f0[r + ldv], x);
              if (fnw > 2) x = fma(-fh2, landed ? side[3] : f0[r + 2 * ldv], x);
              x = x * frs;
            }
          }
          sb[sp * bplane + hy * BW + hx] = x;
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      // a copy that never completed: raise the abort flag (the step's barrier then stops every block)
      if (tid == 0 && a.abort_flag) atomicExch(a.abort_flag, ST_ETIMEOUT);
      break;
    }
    done = k + 1;
    KIOPS_TICK(12);
    // A~ v_j on the tile's own points and the step's dots, every operand from the stage
    {
      const int tot = ns * thl * tvl;
      TileWalk wk(tid, tvl, thl);
      for (int e = tid; e < tot; e += kThreads, wk.next()) {
        const int sp = wk.s, ly = wk.y, cv = wk.x;
        if (kFixed && (ly >= th || cv >= tv)) continue;  // beyond the grid (ragged tile)
        const int bi = sp * bplane + (ly + 1) * BW + W + cv * W;
        const int pi = ly * TW + cv * W;
        const int fo = sp ? fo_s[1] : fo_s[0], ft = sp ? ft_s[1] : ft_s[0];
        const T c1 = sp ? cfr[1][1] : cfr[0][1], c2 = sp ? cfr[1][2] : cfr[0][2];
        const T c3 = sp ? cfr[1][3] : cfr[0][3], c4 = sp ? cfr[1][4] : cfr[0][4];
        const Aff4<T> af = tma_aff<T>(a, sp);  // centre and coupling constants (one shared-memory read)
        // each operand vector is read right before its terms are added (short live ranges); per element the
        // terms are added in the order of fused_st2d_tiles (a plane that is the entry itself has weight 1 and
        // no constant, so that fma(1, d, c) = c + d)
        const Vec16<T> ctr = ld16(sb + bi);
        Vec16<T> out;
        {
          Vec16<T> dow;
          if (fo >= 0) dow = ld16(db + fo * oplane + pi);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = (fo >= 0 ? fma(af.wo, dow.e[u], af.cc) : af.cc) * ctr.e[u];
        }
        {
          const T wl = sb[bi - 1], er = sb[bi + W];
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(c1, u == 0 ? wl : ctr.e[u == 0 ? 0 : u - 1], out.e[u]);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(c2, u == W - 1 ? er : ctr.e[u == W - 1 ? 0 : u + 1], out.e[u]);
        }
        {
          const Vec16<T> up = ld16(sb + bi - BW);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(c3, up.e[u], out.e[u]);
        }
        {
          const Vec16<T> dn = ld16(sb + bi + BW);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(c4, dn.e[u], out.e[u]);
        }
        if (ft >= 0) {
          const Vec16<T> oth = ld16(sb + bi + (1 - 2 * sp) * bplane), dth = ld16(db + ft * oplane + pi);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(fma(af.wt, dth.e[u], af.ct), oth.e[u], out.e[u]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < p) {
            const Vec16<T> bv = ld16(bb + (t * ns + sp) * oplane + pi);
#pragma unroll
            for (int u = 0; u < W; ++u) out.e[u] = fma(ntr[t], bv.e[u], out.e[u]);
          }
        if (CP < 0 || CP > 4)
          for (int t = 4; t < p; ++t) {
            const Vec16<T> bv = ld16(bb + (t * ns + sp) * oplane + pi);
#pragma unroll
            for (int u = 0; u < W; ++u) out.e[u] = fma(ntp[t], bv.e[u], out.e[u]);
          }
        stg16(xo + (size_t)sp * npts + (uint32_t)(y0 + ly) * nx + (uint32_t)(x0 + cv * W), out);
        {  // the step's dots
          Vec16<T> g;
          if (i0_l != j_l) g = ld16(fb + wslot0 * fst + bi);
          T v0[W];
#pragma unroll
          for (int u = 0; u < W; ++u) v0[u] = (i0_l == j_l) ? ctr.e[u] : g.e[u];
          acc.template add_item<W>(0, v0, out.e);
          acc.template add_item<W>(kChunk, ctr.e, v0);
        }
        if (nwin_l > 1) {
          Vec16<T> g;
          if (i0_l + 1 != j_l) g = ld16(fb + wslot1 * fst + bi);
          T v1[W];
#pragma unroll
          for (int u = 0; u < W; ++u) v1[u] = (i0_l + 1 == j_l) ? ctr.e[u] : g.e[u];
          acc.template add_item<W>(1, v1, out.e);
          acc.template add_item<W>(kChunk + 1, ctr.e, v1);
        }
        if (nwin_l > 2) {  // i0 + 2 == j
          acc.template add_item<W>(2, ctr.e, out.e);
          acc.template add_item<W>(kChunk + 2, ctr.e, ctr.e);
        }
        acc.template add_item<W>(2 * kChunk, out.e, out.e);
      }
    }
    KIOPS_TICK(13);
    fence_proxy_async_smem();  // this stage's shared-memory accesses come before the next copies into it
    __syncthreads();
    KIOPS_TICK(15);
    if (tid == 0 && k + S < K) issue(k + S);
  }
  // copies issued but not consumed (only after a copy timed out): wait for them, bounded, before the
  // stages are reused
  for (int k = done; k < K && k < done + S; ++k) {
    const int st = (int)((q0 + (unsigned)k) % (unsigned)S);
    mbar_wait(bars + st, ((q0 + (unsigned)k) / (unsigned)S) & 1u, timeout_ns);
  }
  __syncthreads();
  if (tid == 0) c.tma_seq = q0 + (unsigned)K;
}

// TMA: the kernel instantiation that contains the bulk-tensor-copy path (kept out of the other
// instantiations, whose register allocation it would otherwise share).
template <typename T, int TMA>
__device__ void fused_st2d_phase(const SolveArgs& a, Ctl& c, int rank, int nblk, int j, int i0, int nwin, bool lead,
                                 T* V, size_t ldv, double* smem, DotAcc<T>& acc, bool prof_on) {
  const OpDesc& op = a.op;
  const uint32_t nx = (uint32_t)op.nx, ny = (uint32_t)op.ny, npts = nx * ny;
  const int ns = op.nspecies;
  const int64_t N = a.N;
  const int p = a.p;
  const int tid = threadIdx.x;
  T* raw = (T*)a.raw;
  const bool pend = c.fin_pending != 0;
  const T* src = pend ? raw + (size_t)((j - 1) & 1) * ldv : V + (size_t)(j - 1) * ldv;  // v_j before finalising
  const bool staged = pend && a.stage_on && c.pre_j == j;  // raw x_j already in shared memory
  T* vj = V + (size_t)(j - 1) * ldv;
  T* xo = raw + (size_t)(j & 1) * ldv;  // raw x_{j+1}
  const int fnw = pend ? c.fin_nwin : 0;
  const T fh0 = fnw > 0 ? T(c.fin_h[0]) : T(0), fh1 = fnw > 1 ? T(c.fin_h[1]) : T(0),
          fh2 = fnw > 2 ? T(c.fin_h[2]) : T(0);
  const T frs = pend ? T(c.fin_rs) : T(1);
  const T* f0 = V + (size_t)((pend ? c.fin_i0 : 1) - 1) * ldv;
  const T* f1 = V + (size_t)((pend ? c.fin_i0 : 1) + (fnw > 1 ? 1 : 0) - 1) * ldv;
  const T* f2 = V + (size_t)((pend ? c.fin_i0 : 1) + (fnw > 2 ? 2 : 0) - 1) * ldv;
  const T* w0 = V + (size_t)(i0 - 1) * ldv;  // dot window of step j (v_j itself comes from shared memory)
  const T* w1 = V + (size_t)(i0 + (nwin > 1 ? 1 : 0) - 1) * ldv;
  const T* w2 = V + (size_t)(i0 + (nwin > 2 ? 2 : 0) - 1) * ldv;
  // shared-memory ring: v_k's finalised tile (with halo) sits in slot (k-1) % ring_n; entries below
  // max(ring_lo, j - ring_n + 1) are stale
  const int nr = a.ring_n;
  const int ring_valid_from = nr > 0 ? max(c.ring_lo, j - nr + 1) : (1 << 30);
  const int ntiles = a.tile_gx * a.tile_gy;
  if (TMA != 0 && ntiles > nblk && a.tma_on) {
    if constexpr (TMA == kTmaFixed)  // 32 x 16 tiles, two species, p = 3
      fused_st2d_tma<T, 32, 16, 2, 3>(a, c, rank, nblk, j, i0, nwin, V, ldv, smem, acc, prof_on);
    else if constexpr (TMA != 0)
      fused_st2d_tma<T>(a, c, rank, nblk, j, i0, nwin, V, ldv, smem, acc, prof_on);
  } else if (ntiles > nblk) {
    fused_st2d_tiles<T>(a, c, rank, nblk, j, i0, nwin, V, ldv, smem, acc, prof_on);
  } else {
    // one tile per block, with the shared-memory extras
    if (rank < a.tile_gx * a.tile_gy) {
      const int bx = rank % a.tile_gx, by = rank / a.tile_gx;
      const int x0 = bx * a.tile_w, y0 = by * a.tile_h;
      const int tw = min(a.tile_w, (int)nx - x0), th = min(a.tile_h, (int)ny - y0);
      if (tw > 0 && th > 0) {
        const int hw = tw + 2, hh = th + 2, plane = hw * hh;
        T* ring = (T*)smem;
        const size_t rstride = (size_t)ns * plane;
        T* st = nr > 0 ? ring + (size_t)((j - 1) % nr) * rstride : ring;
        const T* stage = (const T*)(smem + a.sm_stage);
        T* cache = (T*)(smem + a.sm_cache);
        const bool cfill = a.cache_on && !c.cache_ok;
        const int E = ns * tw * th;
        // halo point e -> 2 r + (1 if the point is this block's own), ~0u outside a Dirichlet grid
        unsigned* tbl = (unsigned*)(smem + a.sm_tbl);
        const bool tok = a.stage_on && c.tbl_ok;
        auto rslot = [&](int k) -> const T* { return ring + (size_t)((k - 1) % nr) * rstride; };
        const bool rf0 = pend && fnw > 0 && c.fin_i0 >= ring_valid_from;
        const bool rf1 = pend && fnw > 1 && c.fin_i0 + 1 >= ring_valid_from;
        const bool rf2 = pend && fnw > 2 && c.fin_i0 + 2 >= ring_valid_from;
        const T* g0 = rf0 ? rslot(c.fin_i0) : nullptr;
        const T* g1 = rf1 ? rslot(c.fin_i0 + 1) : nullptr;
        const T* g2 = rf2 ? rslot(c.fin_i0 + 2) : nullptr;
        // finalisation over tile + halo; TOK: the index table is filled (no index arithmetic)
        const bool wtbl = a.stage_on;  // (the argument block is in shared memory)
        const int bc = op.bc;
        auto finalize = [&](auto tok_tag) {
          constexpr bool TOK = decltype(tok_tag)::value;
          TileWalk wk(tid, hw, hh);
          for (int e = tid; e < ns * plane; e += kThreads, wk.next()) {
            unsigned code;
            if constexpr (TOK) {
              code = tbl[e];
            } else {
              const int sp = wk.s, hy = wk.y, hx = wk.x;
              int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
              gx = (int)bc_index(bc, gx, nx);
              gy = (int)bc_index(bc, gy, ny);
              const bool inside = gx >= 0 && gy >= 0;
              const unsigned own = (hx >= 1 && hx <= tw && hy >= 1 && hy <= th) ? 1u : 0u;
              code = inside ? 2u * ((unsigned)sp * npts + (unsigned)gy * nx + (unsigned)gx) + own : ~0u;
              if (wtbl) tbl[e] = code;
            }
            T v = T(0);
            if (code != ~0u) {
              const size_t r = code >> 1;
              v = staged ? stage[e] : src[r];
              if (pend) {
                v = fma(-fh0, rf0 ? g0[e] : f0[r], v);
                if (fnw > 1) v = fma(-fh1, rf1 ? g1[e] : f1[r], v);
                if (fnw > 2) v = fma(-fh2, rf2 ? g2[e] : f2[r], v);
                v = v * frs;
                if (code & 1u) vj[r] = v;
              }
            }
            st[e] = v;
          }
        };
        if (tok) finalize(std::true_type{});
        else finalize(std::false_type{});
        if (cfill) {  // B columns and coupling fields of the tile's own points (each thread its own e)
          TileWalk wk(tid, tw, th);
          for (int e = tid; e < E; e += kThreads, wk.next()) {
            const int sp = wk.s, ly = wk.y, lx = wk.x;
            const uint32_t pt = (uint32_t)(y0 + ly) * nx + (uint32_t)(x0 + lx);
            const size_t r = (size_t)sp * npts + pt;
            for (int t = 0; t < p; ++t) cache[(size_t)t * E + e] = bcol<T>(a, t, r);
            for (int q = 0; q < ns; ++q)  // the point's own coupling entry is kept merged with the centre
              if (op.diag[sp][q])
                cache[(size_t)(p + q) * E + e] = q == sp ? coef_ptr<T>(op, sp)[0] + diag_val<T>(a, sp, q, pt)
                                                         : diag_val<T>(a, sp, q, pt);
          }
        }
        __syncthreads();
        KIOPS_TICK(12);
        const bool rw0 = i0 != j && i0 >= ring_valid_from, rw1 = nwin > 1 && i0 + 1 != j && i0 + 1 >= ring_valid_from;
        const T* q0 = rw0 ? rslot(i0) : nullptr;
        const T* q1 = rw1 ? rslot(i0 + 1) : nullptr;
        // A~ v_j on the own points and the step's dots; CACHE: B and coupling values from shared memory
        auto compute = [&](auto cache_tag) {
          constexpr bool CACHE = decltype(cache_tag)::value;
          // FP32 basis: the products of up to kGroup of this thread's points are summed by FMAs in part[]
          // and added to the float-float accumulators by one TwoSum (DotAcc::add_item's bound, per group)
          constexpr bool kPart = sizeof(T) == 4;
          constexpr int kGroup = 4;
          T part[2 * kChunk + 1];
#pragma unroll
          for (int k = 0; k <= 2 * kChunk; ++k) part[k] = T(0);
          int npart = 0;
          auto dot = [&](int k, T x, T y) {
            if constexpr (kPart) part[k] = fma(x, y, part[k]);
            else acc.add(k, x, y);
          };
          auto flush = [&]() {
#pragma unroll
            for (int k = 0; k <= 2 * kChunk; ++k) {
              acc.add_sum(k, part[k]);
              part[k] = T(0);
            }
            npart = 0;
          };
          TileWalk wk(tid, tw, th);
          for (int e = tid; e < E; e += kThreads, wk.next()) {
            const int sp = wk.s, ly = wk.y, lx = wk.x;
            const uint32_t pt = (uint32_t)(y0 + ly) * nx + (uint32_t)(x0 + lx);
            const size_t r = (size_t)sp * npts + pt;
            const int h = sp * plane + (ly + 1) * hw + (lx + 1);
            const T* cf = coef_ptr<T>(op, sp);
            const T* nt = ntail_ptr<T>(c);
            const T ctr = st[h];
            T xv;
            if constexpr (CACHE) {
              // centre: (c_0 + own coupling entry) v with the sum read from the cache, then the neighbours,
              // the other species' coupling and the B block, all from shared memory
              T cc = cf[0];
              if (op.diag[sp][sp]) cc = cache[(size_t)(p + sp) * E + e];
              xv = cc * ctr;
              xv = fma(cf[1], st[h - 1], xv);
              xv = fma(cf[2], st[h + 1], xv);
              xv = fma(cf[3], st[h - hw], xv);
              xv = fma(cf[4], st[h + hw], xv);
              for (int q = 0; q < ns; ++q)
                if (q != sp && op.diag[sp][q]) xv = fma(cache[(size_t)(p + q) * E + e], st[q * plane + (ly + 1) * hw + (lx + 1)], xv);
              for (int t = 0; t < p; ++t) xv = fma(nt[t], cache[(size_t)t * E + e], xv);
            } else {
              // the same arithmetic from global memory, every coupling and B value loaded before its use so
              // that the loads overlap
              const int qo = 1 - sp;
              const bool has_own = op.diag[sp][sp] != nullptr, has_oth = ns == 2 && op.diag[sp][qo] != nullptr;
              const T d_own = has_own ? diag_val<T>(a, sp, sp, pt) : T(0);
              const T d_oth = has_oth ? diag_val<T>(a, sp, qo, pt) : T(0);
              const T cc = has_own ? cf[0] + d_own : cf[0];
              xv = cc * ctr;
              xv = fma(cf[1], st[h - 1], xv);
              xv = fma(cf[2], st[h + 1], xv);
              xv = fma(cf[3], st[h - hw], xv);
              xv = fma(cf[4], st[h + hw], xv);
              if (has_oth) xv = fma(d_oth, st[qo * plane + (ly + 1) * hw + (lx + 1)], xv);
              xv = add_btail<T>(a, nt, p, r, xv);
            }
            xo[r] = xv;
            const T v0 = (i0 == j) ? ctr : (rw0 ? q0[h] : w0[r]);
            dot(0, v0, xv);
            dot(kChunk, ctr, v0);
            if (nwin > 1) {
              const T v1 = (i0 + 1 == j) ? ctr : (rw1 ? q1[h] : w1[r]);
              dot(1, v1, xv);
              dot(kChunk + 1, ctr, v1);
            }
            if (nwin > 2) {  // i0 + 2 == j
              dot(2, ctr, xv);
              dot(kChunk + 2, ctr, ctr);
            }
            dot(2 * kChunk, xv, xv);
            if constexpr (kPart)
              if (++npart == kGroup) flush();
          }
          if constexpr (kPart)
            if (npart > 0) flush();
        };
        if (a.cache_on) compute(std::true_type{});
        else compute(std::false_type{});
      }
    }
  }
  if (lead && tid < p) {  // tail rows: finalised tail of v_j (c.tail) and the shift K of Theorem 1
    const int64_t rr = N + tid;
    if (pend) vj[rr] = (T)c.tail[tid];
    const T xv = tid + 1 < p ? (T)c.tail[tid + 1] : T(0);
    xo[rr] = xv;
    const T vjt = (T)c.tail[tid];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      if (u < nwin) {
        const T vi = (i0 + u == j) ? vjt : V[(size_t)(i0 + u - 1) * ldv + rr];
        acc.add(u, vi, xv);
        acc.add(kChunk + u, vjt, vi);
      }
    }
    acc.add(2 * kChunk, xv, xv);
  }
}

// Fused step for 3D 7-point stencils with an FP32 basis on grids with more tiles than blocks, operands staged
// by bulk tensor copies: the 3D counterpart of fused_st2d_tma.  Block `rank` takes tiles rank, rank + nblk, ...;
// thread 0 issues each tile's copies into one of tma_stages shared-memory stages, tma_stages tiles ahead.
// Per tile (tile_w x tile_h x tile_d points): halo'd boxes (one-point halo in y and z, 16-byte aligned start in
// x) of raw x_j (or v_j itself on the first step of a substep) and of the window vectors of its finalisation;
// an own-point box of the reaction field.  The B columns (first four) of each thread's products item are
// copied by 16-byte cp.async into per-thread slots before the tile's wait, so that their latency overlaps the
// wait and the finalisation; further columns are read from global memory in the products.  v_j is finalised over the box in shared memory (lagged
// normalisation: no separate normalise pass and no second grid barrier per step), its own points stored;
// then x_{j+1} = A~ v_j on the own points, stored raw, and the step's dots (each item's products as one sum,
// DotAcc::add_item).  Points outside the grid arrive as
// zeros (the Dirichlet value); for periodic or reflected boundaries the halo points the stencil reads there
// (one face layer per side, no edges or corners) are filled after the finalisation from the box, where the
// mapped point lies in it, else from global memory, finalised.
// CTW, CTH, CTD > 0 fix the tile shape at compile time (a kernel instantiation of its own): loop bounds and
// shared-memory offsets are constants, and a ragged tile at the grid's far faces runs the whole box with the
// points beyond the grid left out of the stores and the dots.  0: taken from the arguments.
template <typename T, int CTW = 0, int CTH = 0, int CTD = 0>
__device__ void fused_st3d_tma(const SolveArgs& a, Ctl& c, int rank, int nblk, int j, int i0, int nwin, bool lead,
                               T* V, size_t ldv, double* smem, DotAcc<T>& acc, bool prof_on) {
  constexpr int W = Vec16<T>::W;
  const OpDesc& op = a.op;
  const int nx = (int)op.nx, ny = (int)op.ny, nz = (int)op.nz;
  const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
  const int64_t N = a.N;
  const int p = a.p;
  const int tid = threadIdx.x;
  const int bc = op.bc;
  T* raw = (T*)a.raw;
  const T* bf = (const T*)a.bf;  // B columns in the basis precision, column t at t * ldv
  const bool pend = c.fin_pending != 0;
  T* vj = V + (size_t)(j - 1) * ldv;
  T* xo = raw + (size_t)(j & 1) * ldv;  // raw x_{j+1}
  const int fnw = pend ? c.fin_nwin : 0;
  const T fh0 = fnw > 0 ? T(c.fin_h[0]) : T(0), fh1 = fnw > 1 ? T(c.fin_h[1]) : T(0),
          fh2 = fnw > 2 ? T(c.fin_h[2]) : T(0);
  const T frs = pend ? T(c.fin_rs) : T(1);
  const int fbase = pend ? c.fin_i0 : i0;
  const int nfb = pend ? fnw : nwin - 1;
  const int wslot0 = i0 - fbase, wslot1 = i0 + 1 - fbase;  // window entries i0, i0 + 1 (when below j)
  T cf[7], ntr[4];
  {
    const T* cp = coef_ptr<T>(op, 0);
#pragma unroll
    for (int k = 0; k < 7; ++k) cf[k] = cp[k];
    const T* nt = ntail_ptr<T>(c);
#pragma unroll
    for (int t = 0; t < 4; ++t) ntr[t] = t < p ? nt[t] : T(0);
  }
  const T* ntp = ntail_ptr<T>(c);
  constexpr bool kFixed = CTW > 0 && CTH > 0 && CTD > 0;
  const int S = a.tma_stages, A = W;
  const int TW = kFixed ? CTW : a.tile_w, TH = kFixed ? CTH : a.tile_h, TD = kFixed ? CTD : a.tile_d;
  const int BW = kFixed ? CTW + 2 * W : a.tma_bw, BH = kFixed ? CTH + 2 : a.tma_bh;
  const int bplane = BW * BH;
  // elements between window boxes (box bytes rounded up to 128)
  const int fst = kFixed ? (bplane * (CTD + 2) * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T)
                         : a.tma_box_bytes / (int)sizeof(T);
  const int gxn = a.tile_gx, gyn = a.tile_gy, ntiles = a.tile_gx * a.tile_gy * a.tile_gz;
  const int K = rank < ntiles ? (ntiles - rank + nblk - 1) / nblk : 0;
  const int nwin_l = nwin, i0_l = i0, j_l = j;
  char* sm = (char*)smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
  uint64_t* bars = (uint64_t*)(sm + a.tma_bar_off);
  T* bslot = (T*)(sm + a.tma_side_off) + (size_t)tid * 16;  // four 16-byte B vectors of this thread's item
  const char* maps = (const char*)a.tmaps;  // 128 bytes each: basis, raw ring, (unused), reaction field
  const bool hasf = a.tma_nf > 0;
  const int off_f = a.tma_off_f, off_d = a.tma_off_d;
  const int stage_bytes = a.tma_stage_bytes;
  const long long timeout_ns = a.timeout_ns;
  const int BD = kFixed ? CTD + 2 : a.tma_bd;
  const unsigned expect = (unsigned)(bplane * BD * (int)sizeof(T) * (1 + nfb)) +
                          (hasf ? (unsigned)(TW * TH * TD * (int)sizeof(T)) : 0u);
  if (tid == 0 && !c.tma_init) {
    for (int s = 0; s < S; ++s) mbar_init(bars + s, 1);
    mbar_init_fence();
    c.tma_init = 1;
  }
  // raw x_j and v_j - 1 were written by every block before the barrier that opened this step
  fence_proxy_async_all();
  __syncthreads();
  const unsigned q0 = c.tma_seq;
  auto origin = [&](int tile, int& x0, int& y0, int& z0) {
    const int tx = tile % gxn, r = tile / gxn;
    x0 = tx * TW;
    y0 = (r % gyn) * TH;
    z0 = (r / gyn) * TD;
  };
  auto issue = [&](int k) {  // thread 0: the copies of this block's k-th tile of the step
    const int tile = rank + k * nblk;
    const int st = (int)((q0 + (unsigned)k) % (unsigned)S);
    char* base = sm + (size_t)st * stage_bytes;
    uint64_t* bar = bars + st;
    int x0, y0, z0;
    origin(tile, x0, y0, z0);
    mbar_arrive_expect_tx(bar, expect);
    if (pend) tma_load_4d(base, maps + 128, x0 - A, y0 - 1, z0 - 1, (j_l - 1) & 1, bar);
    else tma_load_4d(base, maps, x0 - A, y0 - 1, z0 - 1, j_l - 1, bar);
    for (int u = 0; u < nfb; ++u)
      tma_load_4d(base + off_f + (size_t)u * fst * sizeof(T), maps, x0 - A, y0 - 1, z0 - 1, fbase + u - 1, bar);
    if (hasf) tma_load_3d(base + off_d, maps + 384, x0, y0, z0, bar);
  };
  if (tid == 0)
    for (int k = 0; k < K && k < S; ++k) issue(k);
  int done = 0;
  for (int k = 0; k < K; ++k) {
    const int tile = rank + k * nblk;
    const int st = (int)((q0 + (unsigned)k) % (unsigned)S);
    const unsigned par = ((q0 + (unsigned)k) / (unsigned)S) & 1u;
    char* base = sm + (size_t)st * stage_bytes;
    int x0, y0, z0;
    origin(tile, x0, y0, z0);
    const int tw = min(TW, nx - x0), th = min(TH, ny - y0), td = min(TD, nz - z0);  // tw: a multiple of W
    const int tv = tw / W;
    // the loops' extent: with a fixed shape the whole box, also on a ragged tile (beyond the grid: the copy's
    // zero fill, computed, never stored or summed)
    const int tvl = kFixed ? TW / W : tv, thl = kFixed ? TH : th, tdl = kFixed ? TD : td;
    const bool edge = bc != 0 && (x0 == 0 || y0 == 0 || z0 == 0 || x0 + tw == nx || y0 + th == ny || z0 + td == nz);
    // this thread's first products item: its B vectors into the slots now (consumed after the finalisation)
    const int pitems = tdl * thl * tvl;
    const int plz = tid / (tvl * thl), prem = tid - plz * (tvl * thl), ply = prem / tvl, pcv = prem - ply * tvl;
    if (tid < pitems && plz < td && ply < th && pcv < tv) {
      const size_t r = (size_t)(z0 + plz) * nxy + (uint32_t)(y0 + ply) * nx + (uint32_t)(x0 + pcv * W);
      for (int t = 0; t < p && t < 4; ++t) cp_async_16(bslot + 4 * t, bf + (size_t)t * ldv + r);
    }
    const bool ok = mbar_wait(bars + st, par, timeout_ns);
    KIOPS_TICK(14);
    T* sb = (T*)base;
    const T* fb = (const T*)(base + off_f);
    const T* db = (const T*)(base + off_d);
    // v_j over the box: planes 0..td+1, rows 0..th+1, vectors 0..tv+1 (box vector c covers x0 - W + c W ...)
    if (ok) {
      const int rv = tvl + 2, tot = (tdl + 2) * (thl + 2) * rv;
      TileWalk wk(tid, rv, thl + 2);
      for (int e = tid; e < tot; e += kThreads, wk.next()) {
        const int hz = wk.s, hy = wk.y, cv = wk.x;
        const int bi = hz * bplane + hy * BW + cv * W;
        Vec16<T> v = ld16(sb + bi);
        if (pend) {
          Vec16<T> g0 = ld16(fb + bi), g1, g2;
          if (fnw > 1) g1 = ld16(fb + fst + bi);
          if (fnw > 2) g2 = ld16(fb + 2 * fst + bi);
#pragma unroll
          for (int u = 0; u < W; ++u) {
            T x = fma(-fh0, g0.e[u], v.e[u]);
            if (fnw > 1) x = fma(-fh1, g1.e[u], x);
            if (fnw > 2) x = fma(-fh2, g2.e[u], x);
            v.e[u] = x * frs;
          }
        }
        st16(sb + bi, v);
        const bool own = hz >= 1 && hz <= td && hy >= 1 && hy <= th && cv >= 1 && cv <= tv;
        if (pend && own)
          stg16(vj + (size_t)(z0 - 1 + hz) * nxy + (uint32_t)(y0 - 1 + hy) * nx + (uint32_t)(x0 - W + cv * W), v);
      }
    }
    if (edge) {  // uniform over the block
      // halo points outside the grid that the stencil reads: one layer per face of the tile
      __syncthreads();
      if (ok) {
        const int nxl = x0 == 0 ? th * td : 0, nxh = x0 + tw == nx ? th * td : 0;
        const int nyl = y0 == 0 ? tw * td : 0, nyh = y0 + th == ny ? tw * td : 0;
        const int nzl = z0 == 0 ? tw * th : 0, nzh = z0 + td == nz ? tw * th : 0;
        const int L = nxl + nxh + nyl + nyh + nzl + nzh;
        const T* src = pend ? raw + (size_t)((j_l - 1) & 1) * ldv : V + (size_t)(j_l - 1) * ldv;
        const T* f0 = V + (size_t)(fbase - 1) * ldv;  // the finalisation window, consecutive columns
        for (int e = tid; e < L; e += kThreads) {
          int q = e, hx, hy, hz;  // box coordinates (points)
          if (q < nxl + nxh) {  // x faces: (ly, lz) over th x td
            const bool hi = q >= nxl;
            if (hi) q -= nxl;
            hy = 1 + q % th, hz = 1 + q / th, hx = hi ? W + tw : W - 1;
          } else if ((q -= nxl + nxh) < nyl + nyh) {  // y faces: (lx, lz) over tw x td
            const bool hi = q >= nyl;
            if (hi) q -= nyl;
            hx = W + q % tw, hz = 1 + q / tw, hy = hi ? th + 1 : 0;
          } else {  // z faces: (lx, ly) over tw x th
            q -= nyl + nyh;
            const bool hi = q >= nzl;
            if (hi) q -= nzl;
            hx = W + q % tw, hy = 1 + q / tw, hz = hi ? td + 1 : 0;
          }
          const int mx = (int)bc_index(bc, x0 - W + hx, nx), my = (int)bc_index(bc, y0 - 1 + hy, ny),
                    mz = (int)bc_index(bc, z0 - 1 + hz, nz);
          const int mbx = mx - (x0 - W), mby = my - (y0 - 1), mbz = mz - (z0 - 1);
          T x;
          if (mx < 0 || my < 0 || mz < 0) {
            x = T(0);  // no mapped point (a reflected axis of one point)
          } else if (mbx >= 0 && mbx < tw + 2 * W && mby >= 0 && mby < th + 2 && mbz >= 0 && mbz < td + 2) {
            x = sb[mbz * bplane + mby * BW + mbx];  // inside the box (reflection): finalised above
          } else {
            const size_t r = (size_t)mz * nxy + (uint32_t)my * nx + (uint32_t)mx;
            x = src[r];
            if (pend) {
              x = fma(-fh0, f0[r], x);
              if (fnw > 1) x = fma(-fh1, f0[r + ldv], x);
              if (fnw > 2) x = fma(-fh2, f0[r + 2 * ldv], x);
              x = x * frs;
            }
          }
          sb[hz * bplane + hy * BW + hx] = x;
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      // a copy that never completed: raise the abort flag (the step's barrier then stops every block)
      if (tid == 0 && a.abort_flag) atomicExch(a.abort_flag, ST_ETIMEOUT);
      break;
    }
    done = k + 1;
    KIOPS_TICK(12);
    cp_async_wait_all();  // this thread's B slots
    // A~ v_j on the tile's own points and the step's dots
    {
      const int tot = tdl * thl * tvl;
      TileWalk wk(tid, tvl, thl);
      for (int e = tid; e < tot; e += kThreads, wk.next()) {
        const int lz = wk.s, ly = wk.y, cv = wk.x;
        if (kFixed && (lz >= td || ly >= th || cv >= tv)) continue;  // beyond the grid (ragged tile)
        const int bi = (lz + 1) * bplane + (ly + 1) * BW + W + cv * W;
        const size_t r = (size_t)(z0 + lz) * nxy + (uint32_t)(y0 + ly) * nx + (uint32_t)(x0 + cv * W);
        const Vec16<T> ctr = ld16(sb + bi);
        Vec16<T> out;
#pragma unroll
        for (int u = 0; u < W; ++u) out.e[u] = cf[0] * ctr.e[u];
        {
          const T wl = sb[bi - 1], er = sb[bi + W];
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(cf[1], u == 0 ? wl : ctr.e[u == 0 ? 0 : u - 1], out.e[u]);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(cf[2], u == W - 1 ? er : ctr.e[u == W - 1 ? 0 : u + 1], out.e[u]);
        }
        {
          const Vec16<T> ym = ld16(sb + bi - BW);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(cf[3], ym.e[u], out.e[u]);
        }
        {
          const Vec16<T> yp = ld16(sb + bi + BW);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(cf[4], yp.e[u], out.e[u]);
        }
        {
          const Vec16<T> zm = ld16(sb + bi - bplane);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(cf[5], zm.e[u], out.e[u]);
        }
        {
          const Vec16<T> zp = ld16(sb + bi + bplane);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(cf[6], zp.e[u], out.e[u]);
        }
        if (hasf) {
          const Vec16<T> dv = ld16(db + (lz * TH + ly) * TW + cv * W);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(dv.e[u], ctr.e[u], out.e[u]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < p) {
            const Vec16<T> bv = e == tid ? ld16(bslot + 4 * t) : ld16(bf + (size_t)t * ldv + r);
#pragma unroll
            for (int u = 0; u < W; ++u) out.e[u] = fma(ntr[t], bv.e[u], out.e[u]);
          }
        for (int t = 4; t < p; ++t) {
          const Vec16<T> bv = ld16(bf + (size_t)t * ldv + r);
#pragma unroll
          for (int u = 0; u < W; ++u) out.e[u] = fma(ntp[t], bv.e[u], out.e[u]);
        }
        stg16(xo + r, out);
        {  // the step's dots
          Vec16<T> g;
          if (i0_l != j_l) g = ld16(fb + wslot0 * fst + bi);
          T v0[W];
#pragma unroll
          for (int u = 0; u < W; ++u) v0[u] = (i0_l == j_l) ? ctr.e[u] : g.e[u];
          acc.template add_item<W>(0, v0, out.e);
          acc.template add_item<W>(kChunk, ctr.e, v0);
        }
        if (nwin_l > 1) {
          Vec16<T> g;
          if (i0_l + 1 != j_l) g = ld16(fb + wslot1 * fst + bi);
          T v1[W];
#pragma unroll
          for (int u = 0; u < W; ++u) v1[u] = (i0_l + 1 == j_l) ? ctr.e[u] : g.e[u];
          acc.template add_item<W>(1, v1, out.e);
          acc.template add_item<W>(kChunk + 1, ctr.e, v1);
        }
        if (nwin_l > 2) {  // i0 + 2 == j
          acc.template add_item<W>(2, ctr.e, out.e);
          acc.template add_item<W>(kChunk + 2, ctr.e, ctr.e);
        }
        acc.template add_item<W>(2 * kChunk, out.e, out.e);
      }
    }
    KIOPS_TICK(13);
    fence_proxy_async_smem();  // this stage's shared-memory accesses come before the next copies into it
    __syncthreads();
    KIOPS_TICK(15);
    if (tid == 0 && k + S < K) issue(k + S);
  }
  // copies issued but not consumed (only after a copy timed out): wait for them, bounded
  cp_async_wait_all();
  for (int k = done; k < K && k < done + S; ++k) {
    const int st = (int)((q0 + (unsigned)k) % (unsigned)S);
    mbar_wait(bars + st, ((q0 + (unsigned)k) / (unsigned)S) & 1u, timeout_ns);
  }
  __syncthreads();
  if (tid == 0) c.tma_seq = q0 + (unsigned)K;
  if (lead && tid < p) {  // tail rows: finalised tail of v_j (c.tail) and the shift K of Theorem 1
    const int64_t rr = N + tid;
    if (pend) vj[rr] = (T)c.tail[tid];
    const T xv = tid + 1 < p ? (T)c.tail[tid + 1] : T(0);
    xo[rr] = xv;
    const T vjt = (T)c.tail[tid];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      if (u < nwin) {
        const T vi = (i0 + u == j) ? vjt : V[(size_t)(i0 + u - 1) * ldv + rr];
        acc.add(u, vi, xv);
        acc.add(kChunk + u, vjt, vi);
      }
    }
    acc.add(2 * kChunk, xv, xv);
  }
}

// Fused path: issue the asynchronous copies of raw x_jn (written by every block before the barrier that
// was passed) over this block's tile + halo into the stage, from the halo index table.  Threads below
// `first` issue none (thread 0 computes the step's coefficients meanwhile); the copies are waited for
// before the block barrier that opens the next step.
template <typename T>
__device__ void fused_prefetch(const SolveArgs& a, int rank, int jn, double* smem, int first) {
  const OpDesc& op = a.op;
  if (rank >= a.tile_gx * a.tile_gy || (int)threadIdx.x < first) return;
  const int x0 = (rank % a.tile_gx) * a.tile_w, y0 = (rank / a.tile_gx) * a.tile_h;
  const int tw = min(a.tile_w, (int)op.nx - x0), th = min(a.tile_h, (int)op.ny - y0);
  if (tw <= 0 || th <= 0) return;
  const int nel = op.nspecies * (tw + 2) * (th + 2);
  const T* src = (const T*)a.raw + (size_t)((jn - 1) & 1) * (size_t)a.ldv;
  T* stage = (T*)(smem + a.sm_stage);
  const unsigned* tbl = (const unsigned*)(smem + a.sm_tbl);
  for (int e = threadIdx.x - first; e < nel; e += kThreads - first) {
    const unsigned code = tbl[e];
    if (code != ~0u) cp_async_elem(stage + e, src + (code >> 1));
  }
}

// ------------------------------------------------------------------------------------------------
// The solver kernel.
// ------------------------------------------------------------------------------------------------
template <typename T, int KIND, class Team, int TMA = 0>
__device__ void solve_body(const SolveArgs& a, Team& team, Ctl& c, double* smem_dyn);

// Tensor maps of the TMA path, passed by value as a grid-constant kernel parameter (128 bytes each, 64-byte
// aligned): basis, raw ring, B columns, coupling fields.
struct TmaMaps {
  alignas(64) unsigned char m[4][128];
};

template <typename T, int KIND, bool GRID, int TMA = 0>
__global__ void __launch_bounds__(kThreads, kMinBlocks) kiops_solve_kernel(const SolveArgs* __restrict__ all,
                                                                           const __grid_constant__ TmaMaps tmaps) {
  extern __shared__ double smem_dyn[];
  __shared__ Ctl c;
  // The argument block is copied to shared memory: gpu-scope acquires at every barrier invalidate L1,
  // and reading it from global memory would put chains of L2 round trips in every phase.
  __shared__ __align__(16) SolveArgs sa;
  {
    const SolveArgs* src = GRID ? all : all + blockIdx.x;
    const int words = (int)(sizeof(SolveArgs) / sizeof(int));
    for (int i = threadIdx.x; i < words; i += kThreads) ((int*)&sa)[i] = ((const int*)src)[i];
    __syncthreads();
    if (threadIdx.x == 0) sa.tmaps = &tmaps;  // generic address of the parameter (the bulk copies read it)
    __syncthreads();
  }
  if (GRID) {
    GridTeam team{(int)blockIdx.x, (int)gridDim.x, sa.bar, sa.abort_flag, sa.timeout_ns, 0u};
    solve_body<T, KIND, GridTeam, TMA>(sa, team, c, smem_dyn);
  } else {
    CtaTeam team;
    solve_body<T, KIND, CtaTeam>(sa, team, c, smem_dyn);
  }
}

// Builds exp(tau H~) for the current j; leaves F(:,1) in a.fvec[0..j) and F(j, j+1) in a.fvec[m_max+1].
// With a.expm_only, exponentiates a.expm_in (n x n) into a.expm_out instead.
template <class Team>
__device__ __noinline__ bool expm_phase(const SolveArgs& a, Team& team, Ctl& c, int& parity, double* smem_dyn,
                                        bool aug = true, double scale = 0.0) {
  // aug: exp(tau H~) of size j+1 (eqs 37-38), F(:,1) and F(j, j+1) into fvec.  !aug: exp(scale H_j) of
  // size j (Algorithm 3), its first column into fvec.
  const bool prof_on = a.prof != nullptr && team.rank == 0;
  const int n = a.expm_only ? a.expm_n : (aug ? c.j + 1 : c.j);
  const size_t ldm = (size_t)(a.m_max + 1) * (a.m_max + 1);
  // the fused path's shared-memory ring, stage and cache live in this region: wait for this thread's
  // copies in flight and mark them all stale
  cp_async_wait_all();
  if (threadIdx.x == 0) {
    c.ring_lo = 1 << 30;
    c.pre_j = 0;
    c.cache_ok = 0;
    c.tbl_ok = 0;
  }
  double* sA = smem_dyn;
  double* sB = smem_dyn + kTile * kMaxN;
  // ||tau H~||_1 from the running column sums (every block holds the same values): a block-wide max,
  // exact in any order
  {
    double mx = 0.0;
    if (!a.expm_only)
      for (int k = 1 + threadIdx.x; k <= c.j; k += kThreads) {
        const double col = c.colabs[k] + (k < c.j ? c.sub[k] : 0.0);
        mx = col > mx ? col : mx;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0) c.wred[threadIdx.x >> 5][0] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double nrm = 0.0;
      if (!a.expm_only) {
        nrm = aug ? 1.0 : 0.0;  // column j+1 of H~ is e_1
        for (int w = 0; w < kWarps; ++w) nrm = c.wred[w][0] > nrm ? c.wred[w][0] : nrm;
        nrm *= aug ? c.tau : scale;
      }
      c.red[0] = nrm;
      if (aug && !a.expm_only) c.hnorm = nrm;
    }
    __syncthreads();
  }
  if (a.expm_only) {
    // column sums of |a| by one warp per column group, same order in every block
    if (threadIdx.x == 0) {
      double best = 0.0;
      for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(a.expm_in[(size_t)i * n + k]);
        best = s > best ? s : best;
      }
      c.red[0] = best;
    }
    __syncthreads();
  }
  // degree choice: squarings s_i and products of every tabulated degree in parallel, then the cheapest
  // (first on ties)
  if (threadIdx.x < a.tt.count) {
    const int i = threadIdx.x;
    const double nrm = c.red[0];
    int s = 0;
    if (nrm > a.tt.theta[i]) s = ceil_log2(nrm / a.tt.theta[i]);
    if (s < 0) s = 0;
    c.wred[0][i] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best_i = 0, best_cost = 1 << 30, best_s = 0;
    for (int i = 0; i < a.tt.count; ++i) {
      const int s = (int)c.wred[0][i];
      const int cost = a.tt.r[i] - 1 + a.tt.q[i] - 1 + s;
      if (cost < best_cost) { best_cost = cost; best_i = i; best_s = s; }
    }
    c.deg_i = best_i;
    c.s_sq = best_s;
    c.n_exp = n;
    c.xscale = ldexp(a.expm_only ? 1.0 : (aug ? c.tau : scale), -best_s);
  }
  __syncthreads();
  const int r = a.tt.r[c.deg_i], q = a.tt.q[c.deg_i], deg = a.tt.deg[c.deg_i];
  double* P = a.mats;                        // P_t at P + (t-1)*ldm, t = 1..r
  double* T0 = a.mats + (size_t)r * ldm;     // Horner / squaring ping-pong
  double* T1 = T0 + ldm;
  // X = xscale * H~ (band entries of H only; H~(1, j+1) = 1; last row 0), or xscale * input
  for (int64_t e = (int64_t)team.rank * kThreads + threadIdx.x; e < (int64_t)n * n; e += (int64_t)team.size * kThreads) {
    const int i = (int)(e / n), k = (int)(e - (int64_t)i * n);  // 0-based
    double v = 0.0;
    if (a.expm_only) {
      v = a.expm_in[e];
    } else if (aug && k == n - 1) {
      v = (i == 0) ? 1.0 : 0.0;
    } else if (!aug || i < n - 1) {
      // H(i+1, k+1) is stored if it is in the window of column k+1 or is the sub-diagonal entry
      const int col = k + 1, row = i + 1;
      const int lo = col - a.m_o + 1 < 1 ? 1 : col - a.m_o + 1;
      if ((row >= lo && row <= col) || row == col + 1) v = a.H[(size_t)(row - 1) * (a.m_max + 2) + (col - 1)];
    }
    P[e] = c.xscale * v;
  }
  if (!team.sync(&c.sync_ok)) return false;
  MmEpi none{0, nullptr, ldm};
  const Band bX = a.expm_only ? Band{n - 1, n - 1} : Band{min(1, n - 1), min(a.m_o - 1, n - 1)};
  Band bP = bX;  // band of X^t
  for (int t = 2; t <= r; ++t) {  // powers X^2..X^r
    mm_team(P + (size_t)(t - 2) * ldm, bP, P, bX, P + (size_t)(t - 1) * ldm, n, team.rank, team.size, c, none, sA, sB);
    bP = band_product(bP, bX, n);
    if (!team.sync(&c.sync_ok)) return false;
  }
  const Band bXr = bP;
  // band of sum_{t<r} c_t X^t (the Horner chunks)
  Band bT{0, 0};
  for (int t = 1; t < r; ++t) bT = Band{min(n - 1, bX.lo * t), min(n - 1, bX.up * t)};
  if (a.expm_only) bT = bX;
  KIOPS_TICK(6);
  // Horner in X^r: T = B_{q-1}; T = T X^r + B_i, B_i = sum_{t<r} coef(i r + t) X^t, coef(k) = 1/k!
  auto coef = [&](int k) -> double { return k > deg ? 0.0 : a.tt.invfact[k]; };
  if (threadIdx.x < r) c.hc[threadIdx.x] = coef((q - 1) * r + threadIdx.x);
  __syncthreads();
  for (int64_t e = (int64_t)team.rank * kThreads + threadIdx.x; e < (int64_t)n * n; e += (int64_t)team.size * kThreads) {
    const int i = (int)(e / n), k = (int)(e - (int64_t)i * n);
    double v = (i == k) ? c.hc[0] : 0.0;
    for (int t = 1; t < r; ++t) v = fma(c.hc[t], P[(size_t)(t - 1) * ldm + e], v);
    T0[e] = v;
  }
  if (!team.sync(&c.sync_ok)) return false;
  double* Tc = T0;
  double* Tn = T1;
  for (int i = q - 2; i >= 0; --i) {
    if (threadIdx.x < r) c.hc[threadIdx.x] = coef(i * r + threadIdx.x);
    __syncthreads();
    MmEpi epi{r, P, ldm};
    mm_team(Tc, bT, P + (size_t)(r - 1) * ldm, bXr, Tn, n, team.rank, team.size, c, epi, sA, sB);
    bT = band_product(bT, bXr, n);
    if (!team.sync(&c.sync_ok)) return false;
    double* t = Tc; Tc = Tn; Tn = t;
  }
  KIOPS_TICK(7);
  // squarings: all but the last in full
  const int ssq = c.s_sq;
  for (int k = 0; k + 1 < ssq || (a.expm_only && k < ssq); ++k) {
    mm_team(Tc, bT, Tc, bT, Tn, n, team.rank, team.size, c, none, sA, sB);
    bT = band_product(bT, bT, n);
    if (!team.sync(&c.sync_ok)) return false;
    double* t = Tc; Tc = Tn; Tn = t;
  }
  if (a.expm_only) {
    for (int64_t e = (int64_t)team.rank * kThreads + threadIdx.x; e < (int64_t)n * n; e += (int64_t)team.size * kThreads)
      a.expm_out[e] = Tc[e];
    return team.sync(&c.sync_ok);
  }
  // last squaring (or none): only F(:,1) and F(j, j+1) are needed
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int jj = c.j;  // 1-based j: F(j, j+1) is (jj-1, jj) 0-based
  const int nrows = aug ? n : n - 1;  // F(j, j+1) only for H~
  for (int row = team.rank * kWarps + warp; row <= nrows; row += team.size * kWarps) {
    // rows 0..n-1: F(row, 0); row n: F(jj-1, jj)
    const int ri = row < n ? row : jj - 1;
    const int ck = row < n ? 0 : jj;
    double s = 0.0;
    if (ssq > 0) {
      for (int l = lane; l < n; l += 32) s = fma(Tc[(size_t)ri * n + l], Tc[(size_t)l * n + ck], s);
      s = warp_sum(s);
    } else {
      s = Tc[(size_t)ri * n + ck];
    }
    if (lane == 0) a.fvec[row < n ? row : a.m_max + 1] = s;
  }
  const bool ok = team.sync(&c.sync_ok);
  KIOPS_TICK(8);
  return ok;
}

// out[r] = beta * sum_k V(r, k) y_k for this rank's rows (Algorithm 3, eq 33).  FP32 basis: y is split into
// float hi + lo, v*yhi is formed exactly (TwoProduct) and the sum is accumulated with TwoSum.
template <typename T>
__device__ void combine_rows(Ctl& c, const T* V, size_t ldv, int j, const double* y, double beta, double* out,
                             int64_t r0, int64_t r1) {
  const int tid = threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    for (int k = tid; k < j; k += kThreads) {
      const float hi = (float)y[k];
      c.yhi[k] = hi;
      c.ylo[k] = (float)(y[k] - (double)hi);
    }
    __syncthreads();
    for (int64_t r = r0 + tid; r < r1; r += kThreads) {
      DotAcc<float> s2;
      s2.hi[0] = 0.0f;
      s2.lo[0] = 0.0f;
      for (int k = 0; k < j; ++k) {
        const float v = (float)V[(size_t)k * ldv + r];
        s2.add(0, v, c.yhi[k]);
        s2.lo[0] = __fmaf_rn(v, c.ylo[k], s2.lo[0]);
      }
      out[r] = beta * ((double)s2.hi[0] + (double)s2.lo[0]);
    }
  } else {
    for (int64_t r = r0 + tid; r < r1; r += kThreads) {
      double s = 0.0;
      for (int k = 0; k < j; ++k) s = fma((double)V[(size_t)k * ldv + r], y[k], s);
      out[r] = beta * s;
    }
  }
}

template <typename T, int KIND, class Team, int TMA>
__device__ void solve_body(const SolveArgs& a, Team& team, Ctl& c, double* smem_dyn) {
  const int tid = threadIdx.x;
  const int64_t N = a.N;
  const int p = a.p;
  // contiguous row range of this rank
  const int64_t chunk = (N + team.size - 1) / team.size;
  const int64_t r0 = (int64_t)team.rank * chunk;
  const int64_t r1 = r0 + chunk < N ? r0 + chunk : N;
  const bool lead = team.rank == 0;
  int parity = 0;
  T* V = (T*)a.V;
  const size_t ldv = (size_t)a.ldv;
  const int ldh = a.m_max + 2;
  const bool prof_on = a.prof != nullptr && lead;
  // lagged normalisation: 2D grids (tiles), 3D grids with an FP32 basis staged in 3D tiles (TMA kernels)
  const bool fused = (KIND == OP_ST2D || (KIND == OP_ST3D && TMA != 0 && sizeof(T) == 4)) && a.fused != 0;

  if (tid == 0) {
    c.status = ST_OK;
    c.done = 0;
    c.substeps = c.rejected = c.matvecs = c.iters = c.expm_calls = 0;
    c.eps_last = 0.0;
    for (int k = 0; k < 16; ++k) c.prof[k] = 0;
    c.prof_last = clock64();
    c.ell = 0;
    c.ring_lo = 1 << 30;
    c.pre_j = 0;
    c.cache_ok = 0;
    c.tbl_ok = 0;
    c.tma_seq = 0;
    c.tma_init = 0;
  }
  __syncthreads();

  if (a.expm_only) {
    expm_phase<Team>(a, team, c, parity, smem_dyn);
    return;
  }

  // ---- setup (section 3.7): ||B||_1 = max_k sum_i |b_k,i|; w = b_0 (Algorithm 1)
  {
    double acc[kRegK];
    for (int base = 1; base <= p; base += kRegK) {
      const int cnt = p - base + 1 < kRegK ? p - base + 1 : kRegK;
#pragma unroll
      for (int k = 0; k < kRegK; ++k) acc[k] = 0.0;
      for (int64_t r = r0 + tid; r < r1; r += kThreads)
#pragma unroll
        for (int k = 0; k < kRegK; ++k)
          if (k < cnt) acc[k] += fabs(__ldg(a.b[base + k] + r));
      block_reduce(c, acc, cnt, base - 1);
    }
    if (a.w != a.b[0])
      for (int64_t r = r0 + tid; r < r1; r += kThreads) a.w[r] = __ldg(a.b[0] + r);
    if constexpr (sizeof(T) == 4) {  // FP32 basis: the matvec's B block and coupling fields in FP32
      for (int t = 0; t < p; ++t)
        for (int64_t r = r0 + tid; r < r1; r += kThreads) a.bf[(size_t)t * a.ldv + r] = (float)__ldg(a.b[p - t] + r);
      if (KIND != OP_CSR) {
        const int ns = KIND == OP_ST3D ? 1 : a.op.nspecies;
        const int64_t npts = a.op.nx * a.op.ny * (KIND == OP_ST3D ? a.op.nz : 1);
        const int64_t pchunk = (npts + team.size - 1) / team.size;
        const int64_t q0 = (int64_t)team.rank * pchunk, q1 = q0 + pchunk < npts ? q0 + pchunk : npts;
        for (int sp = 0; sp < ns; ++sp)
          for (int q = 0; q < ns; ++q)
            if (a.op.diag[sp][q])
              for (int64_t pt = q0 + tid; pt < q1; pt += kThreads)
                a.df[(size_t)(sp * ns + q) * npts + pt] = (float)__ldg(a.op.diag[sp][q] + pt);
      }
    }
    if (TMA != 0 && KIND == OP_ST2D && a.tma_on) {  // TMA path: B columns (FP64 basis) and coupling fields as staged
      if constexpr (sizeof(T) == 8) {
        double* tb = (double*)a.tma_b;
        for (int t = 0; t < p; ++t)
          for (int64_t r = r0 + tid; r < r1; r += kThreads) tb[(size_t)t * a.ldv + r] = __ldg(a.b[p - t] + r);
      }
      const int ns = a.op.nspecies;
      const int64_t npts = a.op.nx * a.op.ny;
      const int64_t pchunk = (npts + team.size - 1) / team.size;
      const int64_t q0 = (int64_t)team.rank * pchunk, q1 = q0 + pchunk < npts ? q0 + pchunk : npts;
      T* tf = (T*)a.tma_f;
      if (a.op.nfields > 0) {  // shared coupling fields: the planes are the fields
        for (int f = 0; f < a.op.nfields; ++f)
          for (int64_t pt = q0 + tid; pt < q1; pt += kThreads) tf[(size_t)f * npts + pt] = (T)__ldg(a.op.field[f] + pt);
      } else {
        for (int sp = 0; sp < ns; ++sp)
          for (int q = 0; q < ns; ++q)
            if (a.tma_fidx[sp][q] >= 0)
              for (int64_t pt = q0 + tid; pt < q1; pt += kThreads)
                tf[(size_t)a.tma_fidx[sp][q] * npts + pt] = (T)__ldg(a.op.diag[sp][q] + pt);
      }
    }
    if (p > 0) {
      if (!finish_reduce<Team>(team, c, a.partials, parity, p)) goto stop;
    } else {
      if (!team.sync(&c.sync_ok)) goto stop;
    }
    if (tid == 0) {
      double nb = 0.0;
      for (int k = 0; k < p; ++k) nb = c.red[k] > nb ? c.red[k] : nb;
      c.nu = 1.0;
      c.mu = 1.0;
      // section 3.7 scaling, FP64 basis only: with an FP32 basis the tail entries (~||B||_1) would dwarf
      // the state entries (~||b_0||_2) in every basis vector and cost about three digits of the result
      if (p >= 1 && a.normalize && nb > 0.0 && sizeof(T) == 8) {
        const int e = ceil_log2(nb);
        c.nu = ldexp(1.0, -e);
        c.mu = ldexp(1.0, e);
      }
      // Algorithm 1: first tau and m
      int m = a.m_init < a.m_max ? a.m_init : a.m_max;
      c.m = m > a.m_min ? m : a.m_min;
      c.tau = a.T_end;
      c.t_now = 0.0;
      c.j = 0;
    }
    __syncthreads();
  }

  KIOPS_TICK(0);
  while (c.t_now < a.T_end) {  // Algorithm 1
    if (c.iters >= a.max_iters || c.substeps >= a.max_substeps) {
      if (tid == 0) c.status = ST_ENOTCONV;
      __syncthreads();
      break;
    }
    if (c.j == 0) {
      // ---- new substep: tail (corrigendum, eq 47, times mu), beta = ||[w; tail]||, V_1
      if (tid == 0) {
        if (c.tau > a.T_end - c.t_now) c.tau = a.T_end - c.t_now;
        for (int t = 0; t < p; ++t) {
          const int e = p - 1 - t;
          double v = 1.0;
          for (int i = 1; i <= e; ++i) v *= c.t_now / (double)i;
          c.tail[t] = c.mu * v;
        }
        c.have_prev = 0;
        c.kappa = 2.0;
        c.qp1_est = 0.0;
        c.fin_pending = 0;
        c.ring_lo = 1 << 30;
        c.pre_j = 0;
      }
      __syncthreads();
      double acc[kRegK];
#pragma unroll
      for (int k = 0; k < kRegK; ++k) acc[k] = 0.0;
      for (int64_t r = r0 + tid; r < r1; r += kThreads) {
        const double x = a.w[r];
        acc[0] = fma(x, x, acc[0]);
      }
      if (lead && tid == 0)
        for (int t = 0; t < p; ++t) acc[0] = fma(c.tail[t], c.tail[t], acc[0]);
      block_reduce(c, acc, 1, 0);
      if (!finish_reduce<Team>(team, c, a.partials, parity, 1)) goto stop;
      if (tid == 0) c.beta = sqrt(c.red[0]);
      __syncthreads();
      if (c.beta == 0.0) {  // v = 0 maps to 0
        for (int64_t r = r0 + tid; r < r1; r += kThreads) a.w[r] = 0.0;
        break;
      }
      {
        const double ib = 1.0 / c.beta;  // Algorithm 1
        for (int64_t r = r0 + tid; r < r1; r += kThreads) V[r] = (T)(a.w[r] * ib);
        if (lead && tid < p) V[N + tid] = (T)(c.tail[tid] * ib);
      }
      if (!team.sync(&c.sync_ok)) goto stop;
      KIOPS_TICK(1);
    }

    // ---- Algorithm 2: IOP steps while j < m
    if (tid == 0) c.breakdown = 0;
    __syncthreads();
    while (c.j < c.m) {
      const int j = c.j + 1;  // step j builds v_{j+1} (slot j) from v_j (slot j-1)
      const int i0 = j - a.m_o + 1 < 1 ? 1 : j - a.m_o + 1;
      const int nwin = j - i0 + 1;
      const T* vj = V + (size_t)(j - 1) * ldv;
      T* x = V + (size_t)j * ldv;
      if (tid < p) {
        if (fused && c.fin_pending) {
          // finalise the pending tail with the arithmetic of the normalise pass; the raw tail of x_j is
          // K v_{j-1} and the window's tails are kept per block, so no global value is needed
          T xv = tid + 1 < p ? T(c.vtail[(j - 1) % kGramRing][tid + 1]) : T(0);
          for (int u = 0; u < c.fin_nwin; ++u)
            xv = fma(-T(c.fin_h[u]), T(c.vtail[(c.fin_i0 + u) % kGramRing][tid]), xv);
          xv = xv * T(c.fin_rs);
          c.tail[tid] = (double)xv;
        } else {
          c.tail[tid] = (double)vj[N + tid];
        }
        c.vtail[j % kGramRing][tid] = c.tail[tid];
        c.ntail[tid] = c.nu * c.tail[tid];
        c.ntail_f[tid] = (float)c.ntail[tid];
      }
      if (fused) cp_async_wait_all();  // the stage prefetched during the last step
      __syncthreads();
      // pass 0 computes x = A~ v_j, stores it raw, and reduces <v_i, x>, <x, x>, <v_j, v_i> for the
      // first kChunk window entries; later passes reread x for further window entries (m_o > kChunk).
      const int Ktot = 2 * nwin + 1;
      T* xraw = fused ? (T*)a.raw + (size_t)(j & 1) * ldv : x;  // where x_{j+1} lives before normalisation
      if (fused) {
        DotAcc<T> dacc;
        dacc.zero();
        if constexpr (KIND == OP_ST3D) {
          if constexpr (TMA == kTmaFixed && sizeof(T) == 4)  // 32 x 8 x 4 tiles
            fused_st3d_tma<T, 32, 8, 4>(a, c, team.rank, team.size, j, i0, nwin, lead, V, ldv, smem_dyn, dacc, prof_on);
          else if constexpr (TMA != 0 && sizeof(T) == 4)
            fused_st3d_tma<T>(a, c, team.rank, team.size, j, i0, nwin, lead, V, ldv, smem_dyn, dacc, prof_on);
        } else {
          fused_st2d_phase<T, TMA>(a, c, team.rank, team.size, j, i0, nwin, lead, V, ldv, smem_dyn, dacc, prof_on);
        }
        __syncthreads();
        if (tid == 0) {
          c.ring_lo = (c.ring_lo <= j - 1) ? c.ring_lo : j;  // v_j is now in the ring
          c.cache_ok = a.cache_on;
          c.tbl_ok = a.stage_on;
        }
        KIOPS_TICK(13);
        block_reduce_dots<T>(c, dacc, 2 * kChunk + 1, nwin);  // compact layout straight into blk
      } else if (nwin <= kChunk) {
        // single pass: R rows per thread in flight (four for FP32 3D stencils, else two), every load issued
        // before the stores; the four-row case adds each dot's R products as one item (DotAcc::add_item),
        // the two-row case takes the rows last to first.  (The two-row case keeps its own straight-line
        // code: written as the R-row loop it ran 2.6 % slower on 160^3 FP64.)
        constexpr int R = (KIND == OP_ST3D && sizeof(T) == 4) ? 4 : 2;
        DotAcc<T> dacc;
        dacc.zero();
        const T* __restrict__ vjr = vj;
        T* __restrict__ xo = x;
        const T* __restrict__ w0 = V + (size_t)(i0 - 1) * ldv;
        const T* __restrict__ w1 = V + (size_t)(i0 + (nwin > 1 ? 1 : 0) - 1) * ldv;
        const T* __restrict__ w2 = V + (size_t)(i0 + (nwin > 2 ? 2 : 0) - 1) * ldv;
        // 3D stencils: the rows' grid coordinates carried from pass to pass (no division per row)
        const uint32_t cnx = (uint32_t)a.op.nx, cny = (uint32_t)a.op.ny, cnxy = cnx * cny;
        Coord3 ca{0u, 0u, 0u}, s1{0u, 0u, 0u}, sR{0u, 0u, 0u};
        if constexpr (KIND == OP_ST3D) {
          ca.set((uint32_t)(r0 + tid), cnx, cnxy);
          s1.set((uint32_t)kThreads, cnx, cnxy);
          sR.set((uint32_t)(R * kThreads), cnx, cnxy);
        }
        if constexpr (R == 4) {
          for (int64_t rb = r0 + tid; rb < r1; rb += R * kThreads) {
            T xr[R];
            bool has[R];
#pragma unroll
            for (int q = 0; q < R; ++q) has[q] = rb + (int64_t)q * kThreads < r1;  // has[0] holds
            if constexpr (KIND == OP_ST3D) {
              Coord3 cq = ca;
#pragma unroll
              for (int q = 0; q < R; ++q) {
                const uint32_t r = (uint32_t)(rb + (int64_t)q * kThreads);
                xr[q] = has[q] ? apply_row_3d<T>(a, vjr, r, cq.ix, cq.iy, cq.iz) : T(0);
                if (q + 1 < R) cq.add(s1, cnx, cny);
              }
              ca.add(sR, cnx, cny);
            } else {
#pragma unroll
              for (int q = 0; q < R; ++q)
                xr[q] = has[q] ? apply_row_fast<T, KIND>(a, vjr, (uint32_t)(rb + (int64_t)q * kThreads)) : T(0);
            }
            {  // B block (weights from shared memory): every load before the first product, same order
              constexpr int kB = 4;
              T bq[R][kB];
#pragma unroll
              for (int t = 0; t < kB; ++t)
#pragma unroll
                for (int q = 0; q < R; ++q)
                  bq[q][t] = (t < p && has[q]) ? bcol<T>(a, t, (size_t)(rb + (int64_t)q * kThreads)) : T(0);
#pragma unroll
              for (int t = 0; t < kB; ++t)
                if (t < p) {
                  const T wt = ntail_ptr<T>(c)[t];
#pragma unroll
                  for (int q = 0; q < R; ++q)
                    if (has[q]) xr[q] = fma(wt, bq[q][t], xr[q]);
                }
              for (int t = kB; t < p; ++t) {
                const T wt = ntail_ptr<T>(c)[t];
#pragma unroll
                for (int q = 0; q < R; ++q)
                  if (has[q]) xr[q] = fma(wt, bcol<T>(a, t, (size_t)(rb + (int64_t)q * kThreads)), xr[q]);
              }
            }
            T vq[R], w0q[R], w1q[R], w2q[R];  // each vector across the rows, then the next vector
#pragma unroll
            for (int q = 0; q < R; ++q) vq[q] = has[q] ? vjr[rb + (int64_t)q * kThreads] : T(0);
#pragma unroll
            for (int q = 0; q < R; ++q) w0q[q] = has[q] ? w0[rb + (int64_t)q * kThreads] : T(0);
#pragma unroll
            for (int q = 0; q < R; ++q) w1q[q] = (nwin > 1 && has[q]) ? w1[rb + (int64_t)q * kThreads] : T(0);
#pragma unroll
            for (int q = 0; q < R; ++q) w2q[q] = (nwin > 2 && has[q]) ? w2[rb + (int64_t)q * kThreads] : T(0);
#pragma unroll
            for (int q = 0; q < R; ++q)
              if (has[q]) xo[rb + (int64_t)q * kThreads] = xr[q];
            // the pass's R rows as one item of the dot accumulators (rows beyond r1 hold zeros)
            dacc.template add_item<R>(0, w0q, xr);
            dacc.template add_item<R>(kChunk, vq, w0q);
            if (nwin > 1) {
              dacc.template add_item<R>(1, w1q, xr);
              dacc.template add_item<R>(kChunk + 1, vq, w1q);
            }
            if (nwin > 2) {
              dacc.template add_item<R>(2, w2q, xr);
              dacc.template add_item<R>(kChunk + 2, vq, w2q);
            }
            dacc.template add_item<R>(2 * kChunk, xr, xr);
          }
        } else {
          for (int64_t rA = r0 + tid; rA < r1; rA += 2 * kThreads) {
            const int64_t rB = rA + kThreads;
            const bool hasB = rB < r1;
            T xa, xb;
            if constexpr (KIND == OP_ST3D) {
              Coord3 cb = ca;
              cb.add(s1, cnx, cny);
              xa = apply_row_3d<T>(a, vjr, (uint32_t)rA, ca.ix, ca.iy, ca.iz);
              xb = hasB ? apply_row_3d<T>(a, vjr, (uint32_t)rB, cb.ix, cb.iy, cb.iz) : T(0);
              ca.add(sR, cnx, cny);
            } else {
              xa = apply_row_fast<T, KIND>(a, vjr, (uint32_t)rA);
              xb = hasB ? apply_row_fast<T, KIND>(a, vjr, (uint32_t)rB) : T(0);
            }
            {  // B block (weights from shared memory): every load before the first product, same order
              constexpr int kB = 4;
              T ba[kB], bb[kB];
#pragma unroll
              for (int t = 0; t < kB; ++t) {
                ba[t] = t < p ? bcol<T>(a, t, (size_t)rA) : T(0);
                bb[t] = (t < p && hasB) ? bcol<T>(a, t, (size_t)rB) : T(0);
              }
#pragma unroll
              for (int t = 0; t < kB; ++t)
                if (t < p) {
                  const T wt = ntail_ptr<T>(c)[t];
                  xa = fma(wt, ba[t], xa);
                  if (hasB) xb = fma(wt, bb[t], xb);
                }
              for (int t = kB; t < p; ++t) {
                const T wt = ntail_ptr<T>(c)[t];
                xa = fma(wt, bcol<T>(a, t, (size_t)rA), xa);
                if (hasB) xb = fma(wt, bcol<T>(a, t, (size_t)rB), xb);
              }
            }
            const T vja = vjr[rA], vjb = hasB ? vjr[rB] : T(0);
            const T wa0 = w0[rA], wb0 = hasB ? w0[rB] : T(0);
            const T wa1 = nwin > 1 ? w1[rA] : T(0), wb1 = (nwin > 1 && hasB) ? w1[rB] : T(0);
            const T wa2 = nwin > 2 ? w2[rA] : T(0), wb2 = (nwin > 2 && hasB) ? w2[rB] : T(0);
            xo[rA] = xa;
            if (hasB) xo[rB] = xb;
            dacc.add(0, wb0, xb);
            dacc.add(0, wa0, xa);
            dacc.add(kChunk, vjb, wb0);
            dacc.add(kChunk, vja, wa0);
            if (nwin > 1) {
              dacc.add(1, wb1, xb);
              dacc.add(1, wa1, xa);
              dacc.add(kChunk + 1, vjb, wb1);
              dacc.add(kChunk + 1, vja, wa1);
            }
            if (nwin > 2) {
              dacc.add(2, wb2, xb);
              dacc.add(2, wa2, xa);
              dacc.add(kChunk + 2, vjb, wb2);
              dacc.add(kChunk + 2, vja, wa2);
            }
            dacc.add(2 * kChunk, xb, xb);
            dacc.add(2 * kChunk, xa, xa);
          }
        }
        if (lead && tid < p) {  // tail rows N..N+p-1: the shift K of Theorem 1
          const int64_t rr = N + tid;
          const T xv = tid + 1 < p ? (T)c.tail[tid + 1] : T(0);
          x[rr] = xv;
          const T vjt = vj[rr];
#pragma unroll
          for (int u = 0; u < kChunk; ++u) {  // static indices keep the accumulators in registers
            if (u < nwin) {
              const T vi = V[(size_t)(i0 + u - 1) * ldv + rr];
              dacc.add(u, vi, xv);
              dacc.add(kChunk + u, vjt, vi);
            }
          }
          dacc.add(2 * kChunk, xv, xv);
        }
        block_reduce_dots<T>(c, dacc, 2 * kChunk + 1, nwin);  // compact layout straight into blk
      }
      for (int cb = 0; cb < nwin && nwin > kChunk && !fused; cb += kChunk) {
        const int cnt = nwin - cb < kChunk ? nwin - cb : kChunk;
        double acc[kRegK];
#pragma unroll
        for (int k = 0; k < kRegK; ++k) acc[k] = 0.0;
        const T* vw[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) vw[u] = V + (size_t)(i0 + cb + (u < cnt ? u : 0) - 1) * ldv;
        for (int64_t r = r0 + tid; r < r1 + (lead ? p : 0); r += kThreads) {
          // rows r1..r1+p-1 of the lead rank stand for the tail rows N..N+p-1
          const bool tailrow = r >= r1;
          const int64_t rr = tailrow ? N + (r - r1) : r;
          T xv;
          if (cb == 0) {
            if (!tailrow) {
              T s = apply_row<T, KIND>(a.op, vj, rr);
              for (int t = 0; t < p; ++t) s += ntail_ptr<T>(c)[t] * bcol<T>(a, t, (size_t)rr);
              xv = s;
            } else {
              const int t = (int)(rr - N);
              xv = t + 1 < p ? (T)c.tail[t + 1] : T(0);
            }
            x[rr] = xv;
          } else {
            xv = x[rr];
          }
          const double xd = (double)xv;
          const double vjd = (double)vj[rr];
#pragma unroll
          for (int u = 0; u < kChunk; ++u) {
            if (u < cnt) {
              const double vi = (double)vw[u][rr];
              acc[u] = fma(vi, xd, acc[u]);
              acc[kChunk + u] = fma(vjd, vi, acc[kChunk + u]);
            }
          }
          if (cb == 0) acc[2 * kChunk] = fma(xd, xd, acc[2 * kChunk]);
        }
        // scatter into the global layout: d at [cb + u], |x|^2 at [nwin], g at [nwin + 1 + cb + u]
        block_reduce(c, acc, 2 * kChunk + 1, 0);
        if (tid == 0) {  // stage this pass in red (free until the all-reduce below)
          for (int u = 0; u < cnt; ++u) {
            c.red[cb + u] = c.blk[u];
            c.red[nwin + 1 + cb + u] = c.blk[kChunk + u];
          }
          if (cb == 0) c.red[nwin] = c.blk[2 * kChunk];
        }
        __syncthreads();
      }
      if (nwin > kChunk && !fused) {  // the multi-pass form staged its sums in red
        for (int k = tid; k < Ktot; k += kThreads) c.blk[k] = c.red[k];
        __syncthreads();
      }
      KIOPS_TICK(2);
      {
        // fused path: x_{j+1} is complete once the barrier is passed; stage its tile for step j + 1
        auto prefetch = [&]() {
          if (fused && a.stage_on && c.tbl_ok && j < c.m) {
            fused_prefetch<T>(a, team.rank, j + 1, smem_dyn, 32);
            if (tid == 0) c.pre_j = j + 1;
          }
        };
        if (!finish_reduce_hook<Team>(team, c, a.partials, parity, Ktot, prof_on, prefetch)) goto stop;
      }
      KIOPS_TICK(3);
      // ---- MGS coefficients from CGS dots and the Gram entries (Algorithm 2):
      // h_i = <v_i, x> - sum_{k<i} h_k <v_i, v_k>;  ||x - sum h_i v_i||^2 expanded over the window
      if (tid == 0) {
        const double nx2 = c.red[nwin];
        auto G = [&](int i, int k) -> double {  // <v_i, v_k>, i, k in the window, 1-based
          if (i < k) { int t = i; i = k; k = t; }
          if (i == j) return c.red[nwin + 1 + (k - i0)];
          if (a.m_o <= kGramRing) return c.gram[i % kGramRing][i - k];
          return a.gram[(size_t)(i - 1) * a.m_o + (i - k)];
        };
        double s2;
        if (nwin == 2 && a.m_o <= kGramRing) {
          // straight-line form of the general expressions below (window {j-1, j})
          const double d0 = c.red[0], d1 = c.red[1];
          const double g10 = c.red[3], g11 = c.red[4], g00 = c.gram[(j - 1) % kGramRing][0];
          const double h0 = d0;
          const double h1 = fma(-h0, g10, d1);
          c.hcoef[0] = h0;
          c.hcoef[1] = h1;
          const double q0 = fma(h0, g00, -2.0 * d0), q1 = fma(h1, g11, -2.0 * d1);
          s2 = fma(h0, q0, fma(h1, q1, fma(2.0 * h0 * h1, g10, nx2)));
        } else {
          for (int u = 0; u < nwin; ++u) {
            const int i = i0 + u;
            double h = c.red[u];
            for (int v = 0; v < u; ++v) h -= c.hcoef[v] * G(i, i0 + v);
            c.hcoef[u] = h;
          }
          s2 = nx2;
          for (int u = 0; u < nwin; ++u) s2 -= 2.0 * c.hcoef[u] * c.red[u];
          for (int u = 0; u < nwin; ++u)
            for (int v = 0; v < nwin; ++v) s2 += c.hcoef[u] * c.hcoef[v] * G(i0 + u, i0 + v);
        }
        c.recompute = !(s2 > 1e-6 * nx2);
        c.s2 = s2;
        c.nx2_pre = nx2;  // ||A~ v_j||^2 for the breakdown test
        c.i0 = i0;
        c.nwin = nwin;
        // common case finished here (one FP64 rsqrt gives both s and 1/s): no breakdown is possible
        // when s^2 > 1e-6 ||x_pre||^2 > breakdown_tol^2 ||x_pre||^2
        if (!c.recompute) {
          const double rs = rsqrt(s2);
          c.rs = rs;
          c.s = s2 * rs;
          c.sub[j] = c.s;
          if (lead) a.H[(size_t)j * ldh + (j - 1)] = c.s;
          double ca = 0.0;
          for (int u = 0; u < nwin; ++u) ca += fabs(c.hcoef[u]);
          c.colabs[j] = ca;
          if (lead)
            for (int u = 0; u < nwin; ++u) a.H[(size_t)(i0 + u - 1) * ldh + (j - 1)] = c.hcoef[u];
          c.matvecs += 1;
          c.j = j;
          if (fused) {  // v_{j+1} is finalised by the next step's tiles (lagged normalisation)
            for (int u = 0; u < nwin; ++u) c.fin_h[u] = c.hcoef[u];
            c.fin_rs = rs;
            c.fin_i0 = i0;
            c.fin_nwin = nwin;
            c.fin_pending = 1;
          }
        }
        // record Gram row j: <v_j, v_{j-o}> for o = 0..nwin-1
        if (a.m_o <= kGramRing) {
          for (int u = 0; u < nwin; ++u) c.gram[j % kGramRing][j - (i0 + u)] = c.red[nwin + 1 + u];
        } else if (lead) {
          for (int u = 0; u < nwin; ++u) a.gram[(size_t)(j - 1) * a.m_o + (j - (i0 + u))] = c.red[nwin + 1 + u];
        }
      }
      __syncthreads();
      const double nx2_pre = c.nx2_pre;
      if (c.recompute) {
        // explicit norm of x - sum h_i v_i (cancellation guard)
        double acc[kRegK];
#pragma unroll
        for (int k = 0; k < kRegK; ++k) acc[k] = 0.0;
        for (int64_t r = r0 + tid; r < r1 + (lead ? p : 0); r += kThreads) {
          const int64_t rr = r >= r1 ? N + (r - r1) : r;
          T xv = xraw[rr];
          for (int u = 0; u < c.nwin; ++u) xv -= T(c.hcoef[u]) * V[(size_t)(c.i0 + u - 1) * ldv + rr];
          const double xd = (double)xv;
          acc[0] = fma(xd, xd, acc[0]);
        }
        block_reduce(c, acc, 1, 0);
        if (!finish_reduce<Team>(team, c, a.partials, parity, 1)) goto stop;
        if (tid == 0) {
          c.s = sqrt(c.red[0]);
          c.matvecs += 1;
          double ca = 0.0;
          for (int u = 0; u < c.nwin; ++u) ca += fabs(c.hcoef[u]);
          c.colabs[j] = ca;
          if (lead)
            for (int u = 0; u < c.nwin; ++u) a.H[(size_t)(c.i0 + u - 1) * ldh + (j - 1)] = c.hcoef[u];
          c.j = j;
          if (c.s * c.s <= a.bd_tol * a.bd_tol * nx2_pre) {  // happy breakdown (Algorithm 2)
            c.breakdown = 1;
            c.sub[j] = 0.0;
          } else {
            c.sub[j] = c.s;
            c.rs = 1.0 / c.s;
            if (lead) a.H[(size_t)j * ldh + (j - 1)] = c.s;
            if (fused) {  // lagged normalisation, as in the common case
              for (int u = 0; u < c.nwin; ++u) c.fin_h[u] = c.hcoef[u];
              c.fin_rs = c.rs;
              c.fin_i0 = c.i0;
              c.fin_nwin = c.nwin;
              c.fin_pending = 1;
            }
          }
        }
        __syncthreads();
      }
      KIOPS_TICK(4);
      if (c.breakdown) break;
      if (fused) continue;  // v_{j+1} is finalised by the next step's tiles (or stays pending)
      // ---- v_{j+1} = (1/s) (x - sum_i h_i v_i) in MGS order (Algorithm 2)
      if (nwin <= kChunk) {
        const T h0 = T(c.hcoef[0]), h1 = nwin > 1 ? T(c.hcoef[1]) : T(0), h2 = nwin > 2 ? T(c.hcoef[2]) : T(0);
        const T rsT = T(c.rs);
        T* __restrict__ xo = x;
        const T* __restrict__ w0 = V + (size_t)(i0 - 1) * ldv;
        const T* __restrict__ w1 = V + (size_t)(i0 + (nwin > 1 ? 1 : 0) - 1) * ldv;
        const T* __restrict__ w2 = V + (size_t)(i0 + (nwin > 2 ? 2 : 0) - 1) * ldv;
        // kNormU rows per pass, their loads issued before the first store
        constexpr int kNormU = 4;
        const int64_t rend = r1 + (lead ? p : 0);
        for (int64_t rb = r0 + tid; rb < rend; rb += kNormU * kThreads) {
          int64_t rr[kNormU];
          T xv[kNormU], a0[kNormU], a1[kNormU], a2[kNormU];
#pragma unroll
          for (int u = 0; u < kNormU; ++u) {
            const int64_t r = rb + (int64_t)u * kThreads;
            rr[u] = -1;
            xv[u] = a0[u] = a1[u] = a2[u] = T(0);
            if (r < rend) {
              rr[u] = r >= r1 ? N + (r - r1) : r;
              xv[u] = xo[rr[u]];
              a0[u] = w0[rr[u]];
              if (nwin > 1) a1[u] = w1[rr[u]];
              if (nwin > 2) a2[u] = w2[rr[u]];
            }
          }
#pragma unroll
          for (int u = 0; u < kNormU; ++u)
            if (rr[u] >= 0) {
              T v = fma(-h0, a0[u], xv[u]);
              if (nwin > 1) v = fma(-h1, a1[u], v);
              if (nwin > 2) v = fma(-h2, a2[u], v);
              xo[rr[u]] = v * rsT;
            }
        }
      } else {
        for (int64_t r = r0 + tid; r < r1 + (lead ? p : 0); r += kThreads) {
          const int64_t rr = r >= r1 ? N + (r - r1) : r;
          T xv = x[rr];
          for (int u = 0; u < c.nwin; ++u) xv -= T(c.hcoef[u]) * V[(size_t)(c.i0 + u - 1) * ldv + rr];
          x[rr] = xv * T(c.rs);
        }
      }
      if (!team.sync(&c.sync_ok)) goto stop;
      KIOPS_TICK(5);
    }

    // ---- Algorithm 1: F = exp(tau H~)
    if (!expm_phase<Team>(a, team, c, parity, smem_dyn)) goto stop;

    // ---- estimate (eq 36), omega (eq 39), Algorithm 4 (sections 3.6.1, 3.6.2)
    if (tid == 0) {
      const double delta = 1.4, gamma = 0.9, gamma_max = 0.6;
      const int j = c.j;
      c.expm_calls += 1;
      double eps = 0.0, omega = 0.0;
      if (!c.breakdown) {
        eps = c.beta * c.sub[j] * fabs(a.fvec[a.m_max + 1]);
        omega = a.T_end * eps / (c.tau * a.tol);
      }
      c.eps_last = eps;
      const int accepted = omega <= delta;
      const double t_next = accepted ? c.t_now + c.tau : c.t_now;
      const double remaining = a.T_end - t_next;
      if (!accepted && c.have_prev) {
        if (j != c.prev_j && c.tau == c.prev_tau) {
          const double k = pow(omega / c.prev_omega, 1.0 / (double)(c.prev_j - j));  // eq 45
          c.kappa = (isfinite(k) && k > 1.0) ? k : 2.0;
        } else if (j == c.prev_j && c.tau != c.prev_tau) {
          const double e = log(eps / c.prev_eps) / log(c.tau / c.prev_tau);  // eq 43 (order q + 1)
          c.qp1_est = (isfinite(e) && e > 0.0) ? e : 0.0;
        }
      }
      const double qp1 = c.qp1_est > 0.0 ? c.qp1_est : (double)j / 4.0;
      double tau_new;
      int m_new;
      if (c.breakdown) {
        tau_new = c.tau < remaining ? c.tau : remaining;
        m_new = c.m;
      } else if (j == a.m_max) {
        if (omega > delta) {
          m_new = j;
          tau_new = c.tau * pow(gamma_max / omega, 1.0 / qp1);
          if (tau_new < c.tau / 5.0) tau_new = c.tau / 5.0;
          if (tau_new > remaining) tau_new = remaining;
        } else {
          m_new = c.m;
          tau_new = c.tau * pow(gamma / omega, 1.0 / qp1);
          if (!(tau_new <= 5.0 * c.tau)) tau_new = 5.0 * c.tau;
          if (tau_new < c.tau / 5.0) tau_new = c.tau / 5.0;
          if (tau_new > remaining) tau_new = remaining;
        }
      } else {
        tau_new = c.tau;
        double mn = (double)c.m + log(omega / gamma) / log(c.kappa);  // eq 46
        const double lo = floor(0.75 * (double)c.m), hi = ceil(4.0 * (double)c.m / 3.0);
        if (!(mn >= lo)) mn = lo;
        if (mn > hi) mn = hi;
        mn = ceil(mn);
        if (mn < a.m_min) mn = a.m_min;
        if (mn > a.m_max) mn = a.m_max;
        m_new = (int)mn;
      }
      // cost model (section 3.2, eqs 40-42) for scenario A (keep m, tau from eq 44) and B (keep tau, m
      // from eq 46); with a.scenario = 1 the cheaper one replaces the change of m above (ties keep B).
      // Evaluated only when it decides or is recorded (its pow / log chain is serial FP64 latency).
      double cost_a = 0.0, cost_b = 0.0;
      if (!c.breakdown && (a.scenario == 1 || (lead && a.trace))) {
        double tau_a = c.tau * pow((accepted ? gamma : gamma_max) / omega, 1.0 / qp1);
        if (accepted && !(tau_a <= 5.0 * c.tau)) tau_a = 5.0 * c.tau;
        if (!(tau_a >= c.tau / 5.0)) tau_a = c.tau / 5.0;
        if (tau_a > remaining) tau_a = remaining;
        double mb = (double)c.m + log(omega / gamma) / log(c.kappa);
        const double lo = floor(0.75 * (double)c.m), hi = ceil(4.0 * (double)c.m / 3.0);
        if (!(mb >= lo)) mb = lo;
        if (mb > hi) mb = hi;
        mb = ceil(mb);
        if (mb < a.m_min) mb = a.m_min;
        if (mb > a.m_max) mb = a.m_max;
        cost_a = scenario_cost(remaining, tau_a, (double)c.m, (double)N, (double)p, a.nz_op,
                               pade_mults(c.hnorm * (tau_a / c.tau)));
        cost_b = scenario_cost(remaining, c.tau, mb, (double)N, (double)p, a.nz_op, pade_mults(c.hnorm));
        if (a.scenario == 1 && j < a.m_max && cost_a < cost_b) {
          tau_new = tau_a;
          m_new = c.m;
        }
      }
      if (lead && a.trace && *a.trace_len < a.trace_cap) {
        TraceRec& tr = a.trace[*a.trace_len];
        tr.substep = c.substeps; tr.j = j; tr.accepted = accepted; tr.breakdown = c.breakdown; tr.m_new = m_new;
        tr.tau = c.tau; tr.t_now = c.t_now; tr.eps = eps; tr.omega = omega; tr.tau_new = tau_new;
        tr.cost_a = cost_a; tr.cost_b = cost_b;
        tr.hnorm = c.hnorm;
        *a.trace_len += 1;
      }
      c.iters += 1;
      c.accepted = accepted;
      c.t_sub = c.t_now;
      c.tau_sub = c.tau;
      if (accepted) {
        if (c.tau >= a.T_end - c.t_now || t_next >= a.T_end) c.t_now = a.T_end;
        else c.t_now = t_next;
        c.substeps += 1;
      } else {
        c.rejected += 1;
        c.have_prev = 1; c.prev_j = j; c.prev_tau = c.tau; c.prev_omega = omega; c.prev_eps = eps;
      }
      c.hc[0] = c.beta;  // beta of this substep for the update
      // a non-finite estimate, or a rejection that changes neither m nor tau, would repeat forever
      if (!isfinite(omega) || (!accepted && m_new <= j && !(tau_new < c.tau))) {
        c.status = ST_ENOTCONV;
        c.done = 1;
      }
      c.tau = tau_new;
      c.m = m_new;
    }
    __syncthreads();
    KIOPS_TICK(9);
    if (c.done) break;
    if (c.accepted) {
      // ---- Algorithm 3: w = beta V(1:N, 1:j) F(1:j, 1), after the Task I outputs inside the substep
      const int j = c.j;
      for (int k = tid; k < j; k += kThreads) c.hcoef[k] = a.fvec[k];
      __syncthreads();
      const double beta = c.beta;
      if (a.n_times > 0) {  // Task I: outputs T(k) < T_now + tau (Algorithm 3)
        while (c.ell < a.n_times - 1 && fabs(a.times[c.ell]) < fabs(c.t_sub + c.tau_sub)) {
          if (!expm_phase<Team>(a, team, c, parity, smem_dyn, false, a.times[c.ell] - c.t_sub)) goto stop;
          for (int k = tid; k < j; k += kThreads) c.yint[k] = a.fvec[k];
          __syncthreads();
          combine_rows<T>(c, V, ldv, j, c.yint, beta, a.wout[c.ell], r0, r1);
          __syncthreads();
          if (tid == 0) c.ell += 1;
          __syncthreads();
        }
      }
      combine_rows<T>(c, V, ldv, j, c.hcoef, beta, a.w, r0, r1);
      if (tid == 0) c.j = 0;
      __syncthreads();
      KIOPS_TICK(10);
    }
  }
  if (a.n_times > 0 && c.status == ST_OK) {  // Task I: w(:, l) *= (1/T(l))^p (Algorithm 1)
    for (int l = 0; l < a.n_times; ++l) {
      double sc = 1.0;
      for (int k = 0; k < p; ++k) sc *= 1.0 / a.times[l];
      for (int64_t r = r0 + tid; r < r1; r += kThreads) a.wout[l][r] *= sc;
    }
  }
stop:
  cp_async_wait_all();  // no copy of the fused path outlives the block
  __syncthreads();
  if (lead && tid == 0) {
    int st = c.status;
    if (a.abort_flag && ld_volatile_int(a.abort_flag)) st = ld_volatile_int(a.abort_flag);
    a.stats[0] = c.substeps; a.stats[1] = c.rejected; a.stats[2] = c.matvecs; a.stats[3] = c.iters;
    a.stats[4] = c.expm_calls; a.stats[5] = c.m; a.stats[6] = st;
    a.stats_d[0] = c.eps_last;
    if (a.prof)
      for (int k = 0; k < 16; ++k) a.prof[k] = c.prof[k];
  }
}

// Single-block solve with the argument block passed by value (no staging buffer): the allocation-free
// entry point uses it.
template <int KIND>
__global__ void __launch_bounds__(kThreads, kMinBlocks) kiops_solve_kernel_byval(const __grid_constant__ SolveArgs args) {
  extern __shared__ double smem_dyn[];
  __shared__ Ctl c;
  __shared__ __align__(16) SolveArgs sa;
  const int words = (int)(sizeof(SolveArgs) / sizeof(int));
  for (int i = threadIdx.x; i < words; i += kThreads) ((int*)&sa)[i] = ((const int*)&args)[i];
  __syncthreads();
  CtaTeam team;
  solve_body<double, KIND, CtaTeam>(sa, team, c, smem_dyn);
}

// ------------------------------------------------------------------------------------------------
// Team engine for batches: one cooperative launch is split into teams of `team_blocks` blocks.  Team t
// runs the instances plan_idx[plan_ptr[t] .. plan_ptr[t+1]) one after another, each with the grid-team
// code above restricted to the team (its own barrier counter, partial sums and workspace).  The host plans
// the lists (largest estimated work first, each to the least-loaded team).
// ------------------------------------------------------------------------------------------------
template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads, kMinBlocks) kiops_team_kernel(const SolveArgs* __restrict__ all,
                                                             const int* __restrict__ plan_ptr,
                                                             const int* __restrict__ plan_idx, int team_blocks,
                                                             int n_teams, unsigned int* team_ctr, int* abort_flag,
                                                             long long timeout_ns) {
  extern __shared__ double smem_dyn[];
  __shared__ Ctl c;
  __shared__ __align__(16) SolveArgs sa;
  const int t = blockIdx.x / team_blocks;
  if (t >= n_teams) return;  // blocks left over when the grid is not a multiple of the team size
  GridTeam team{(int)(blockIdx.x % team_blocks), team_blocks, team_ctr + (size_t)t * 64, abort_flag, timeout_ns, 0u};
  const int words = (int)(sizeof(SolveArgs) / sizeof(int));
  for (int q = plan_ptr[t]; q < plan_ptr[t + 1]; ++q) {
    const SolveArgs* src = all + plan_idx[q];
    for (int i = threadIdx.x; i < words; i += kThreads) ((int*)&sa)[i] = ((const int*)src)[i];
    __syncthreads();
    solve_body<T, KIND, GridTeam>(sa, team, c, smem_dyn);
    // every block of the team leaves the instance before its workspace is reused
    if (!team.sync(&c.sync_ok)) break;
  }
}

// ------------------------------------------------------------------------------------------------
// Serving: a persistent kernel whose teams take requests from queues as they arrive (continuous
// batching).  Queue words and request slots live in mapped host memory: the host writes a slot and then
// advances the class's tail with release semantics; a team leader claims index `head` with a CAS when
// head < tail (acquire), copies the slot, runs the solve, and publishes the request's ticket in the
// slot's completion word (system-scope release).  Teams of class c have team_blocks[c] blocks.  Every
// wait is bounded: an idle team leaves after idle_ns without work (the host relaunches the kernel), the
// barriers keep their own deadline.
// ------------------------------------------------------------------------------------------------
constexpr int kServerClasses = 2;

struct ServerDev {
  int n_classes;
  int team_blocks[kServerClasses], teams[kServerClasses], first_block[kServerClasses];
  int slots_per_class;
  const unsigned int* tail[kServerClasses];  // mapped host memory
  unsigned int* head[kServerClasses];        // device memory
  const int* stop;                           // mapped host memory
  const SolveArgs* slots[kServerClasses];    // mapped host memory
  unsigned long long* done[kServerClasses];  // mapped host memory
  unsigned int* team_ctr;                    // 64 words per team (device)
  double* team_partials;                     // 2 * kMaxRed * team_blocks per team (device)
  size_t team_partials_stride;               // doubles per team
  int* team_claim;                           // one word per team, 64 apart (device)
  int* abort_flag;
  long long timeout_ns, idle_ns;
};

__device__ __forceinline__ unsigned int ld_acquire_sys(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_sys_int(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int Unused>
__global__ void __launch_bounds__(kThreads, kMinBlocks) kiops_server_kernel(const __grid_constant__ ServerDev sd) {
  extern __shared__ double smem_dyn[];
  __shared__ Ctl c;
  __shared__ __align__(16) SolveArgs sa;
  int cls = -1;
  for (int k = 0; k < sd.n_classes; ++k)
    if ((int)blockIdx.x >= sd.first_block[k] && (int)blockIdx.x < sd.first_block[k] + sd.teams[k] * sd.team_blocks[k])
      cls = k;
  if (cls < 0) return;
  const int local = (int)blockIdx.x - sd.first_block[cls];
  const int K = sd.team_blocks[cls];
  int team_id = local / K;
  for (int k = 0; k < cls; ++k) team_id += sd.teams[k];
  GridTeam team{local % K, K, sd.team_ctr + (size_t)team_id * 64, sd.abort_flag, sd.timeout_ns, 0u};
  const int words = (int)(sizeof(SolveArgs) / sizeof(int));
  while (true) {
    if (team.rank == 0 && threadIdx.x == 0) {
      int claimed = -1;
      const long long t0 = global_ns();
      while (true) {
        if (ld_volatile_int(sd.abort_flag)) break;  // a wait gave up: claim nothing more in this launch
        const unsigned int h = *(volatile unsigned int*)sd.head[cls];
        const unsigned int tl = ld_acquire_sys(sd.tail[cls]);
        if ((int)(tl - h) > 0) {
          if (atomicCAS(sd.head[cls], h, h + 1) == h) { claimed = (int)h; break; }
          continue;
        }
        if (ld_acquire_sys_int(sd.stop)) break;
        if (global_ns() - t0 > sd.idle_ns) break;
        __nanosleep(1000);
      }
      sd.team_claim[(size_t)team_id * 64] = claimed;
    }
    if (!team.sync(&c.sync_ok)) return;
    const int claimed = *(volatile int*)(sd.team_claim + (size_t)team_id * 64);
    if (claimed < 0) return;
    const SolveArgs* src = sd.slots[cls] + (claimed % sd.slots_per_class);
    for (int i = threadIdx.x; i < words; i += kThreads) ((int*)&sa)[i] = ((const volatile int*)src)[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      sa.partials = sd.team_partials + (size_t)team_id * sd.team_partials_stride;
      sa.abort_flag = sd.abort_flag;
    }
    __syncthreads();
    const int kind = sa.op.kind;
    if (sa.prec == 0) {
      if (kind == OP_CSR) solve_body<double, OP_CSR, GridTeam>(sa, team, c, smem_dyn);
      else if (kind == OP_ST2D) solve_body<double, OP_ST2D, GridTeam>(sa, team, c, smem_dyn);
      else solve_body<double, OP_ST3D, GridTeam>(sa, team, c, smem_dyn);
    } else {
      if (kind == OP_CSR) solve_body<float, OP_CSR, GridTeam>(sa, team, c, smem_dyn);
      else if (kind == OP_ST2D) solve_body<float, OP_ST2D, GridTeam>(sa, team, c, smem_dyn);
      else solve_body<float, OP_ST3D, GridTeam>(sa, team, c, smem_dyn);
    }
    if (!team.sync(&c.sync_ok)) return;
    if (team.rank == 0 && threadIdx.x == 0) {
      __threadfence_system();
      st_release_sys_u64(sd.done[cls] + (claimed % sd.slots_per_class), sa.ticket);
    }
  }
}

}  // namespace KIOPS_DEV_NS
