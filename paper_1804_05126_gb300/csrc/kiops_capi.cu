// Host side of the C ABI declared in include/kiops.h: contexts, operators, workspace, launches.
//
// A solve is one launch: the grid engine is a cooperative launch of as many blocks as are co-resident
// (the whole GPU works on one solve), the CTA engine launches one block per request of a batch.  The
// host only validates arguments, lays out the workspace, uploads the argument block and reads back the
// statistics; every step of Algorithm 1 runs in the kernel of kiops_device.cuh.
#include <cuda.h>  // tensor-map types (the encoder is reached through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>  // header-only NVTX: ranges cost nothing unless a profiler is attached

#include "kiops.h"
#include "kiops_device.cuh"
#include "kiops_kernels.h"

using namespace kiops_dev;

struct KiopsServer;  // serving state (kiops_server_start)
struct kiops_ctx;

extern "C" {
static kiops_status batch_teams(kiops_ctx* ctx, int count, const kiops_request* reqs, kiops_stats* stats);
}

struct kiops_ctx {
  kiops_config cfg;
  cudaStream_t stream = nullptr;
  int sms = 0;
  std::string err;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  void* host_pinned = nullptr;  // argument block + stats + trace staging
  size_t host_pinned_bytes = 0;
  double* stage_dev = nullptr;  // device staging of host-buffer solves
  size_t stage_bytes = 0;
  TaylorTable tt{};
  bool busy = false;
  KiopsServer* server = nullptr;
  double* integ = nullptr;      // integrator workspace (kiops_integrate)
  size_t integ_bytes = 0;
};

struct kiops_op {
  kiops_ctx* ctx;
  OpDesc d;
  double nz = 0.0;         // stored nonzeros (the cost model's nz(A))
  double* owned = nullptr; // entries of a block given by shared coupling fields (written at creation)
};

namespace {

kiops_status fail(kiops_ctx* ctx, kiops_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return s;
}

#define KCHECK(ctx, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(ctx, KIOPS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Host-side NVTX range around an entry point (visible in nsys / ncu timelines).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Truncation tail sum_{k > d} theta^k / k! (terms through exp/lgamma; every term positive).
double taylor_tail(double theta, int d) {
  double s = 0.0;
  for (int k = d + 1; k < d + 200; ++k) {
    double t = std::exp(k * std::log(theta) - std::lgamma((double)k + 1.0));
    s += t;
    if (t < 1e-40 * s) break;
  }
  return s;
}

// Paterson-Stockmeyer degrees deg = r q - 1 for costs r + q - 2 = 3..10 matrix products; theta is the
// largest ||X||_1 with a truncation tail below 2^-53 (bisection).
void build_taylor_table(TaylorTable& tt) {
  tt.count = 0;
  for (int cost = 3; cost <= 10 && tt.count < kMaxDeg; ++cost) {
    int r = (cost + 2) / 2, q = (cost + 2) - r;
    int d = r * q - 1;
    double lo = 1e-8, hi = 64.0;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (taylor_tail(mid, d) <= std::ldexp(1.0, -53)) lo = mid; else hi = mid;
    }
    tt.deg[tt.count] = d;
    tt.r[tt.count] = r;
    tt.q[tt.count] = q;
    tt.theta[tt.count] = lo;
    tt.count++;
  }
  for (int k = 0; k < 64; ++k) {  // 1/k! by repeated division, the order the device used to take
    double v = 1.0;
    for (int i = 2; i <= k; ++i) v /= (double)i;
    tt.invfact[k] = v;
  }
}

int max_r(const TaylorTable& tt) {
  int r = 1;
  for (int i = 0; i < tt.count; ++i) r = std::max(r, tt.r[i]);
  return r;
}

void* pick_kernel(bool fp32, int kind) { return fp32 ? kiops_k::solve_kernel_f32(kind) : kiops_k::solve_kernel_f64(kind); }

void* pick_team_kernel(bool fp32, int kind) {
  return fp32 ? kiops_k::team_kernel_f32(kind) : kiops_k::team_kernel_f64(kind);
}

constexpr size_t kDynSmem = 2 * kTile * kMaxN * sizeof(double);
constexpr int kMaxTilesPerBlock = 64;  // fused 2D path: larger grids take the separate normalise pass

// Per-solve device layout (each region 256-byte aligned).
struct Layout {
  size_t V, H, gram, mats, fvec, partials, bar, stats, trace_len, prof, args, trace, raw, bf, df, total;
};

Layout layout(int64_t N, int p, int m_max, int m_o, bool fp32, int grid_blocks, int r_max, int64_t trace_cap,
              int64_t* ldv_out, int64_t df_elems = 0) {
  Layout L{};
  const int64_t ldv = (int64_t)align_up((size_t)(N + p), 64);
  *ldv_out = ldv;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.V = take((size_t)(m_max + 1) * ldv * (fp32 ? 4 : 8));
  L.H = take((size_t)(m_max + 2) * (m_max + 2) * 8);
  L.gram = take((size_t)(m_max + 1) * std::max(m_o, 1) * 8);
  L.mats = take((size_t)(r_max + 2) * (m_max + 1) * (m_max + 1) * 8);
  L.fvec = take((size_t)(m_max + 2) * 8);
  L.partials = take((size_t)2 * std::max(grid_blocks, 1) * kMaxRed * 8);
  L.bar = take(256);
  L.stats = take(16 * 8);
  L.trace_len = take(8);
  L.prof = take(16 * 8);
  L.args = take(sizeof(SolveArgs));
  L.trace = take((size_t)std::max<int64_t>(trace_cap, 0) * sizeof(TraceRec));
  L.raw = take((size_t)2 * ldv * (fp32 ? 4 : 8));
  L.bf = take(fp32 ? (size_t)std::max(p, 1) * ldv * 4 : 0);
  L.df = take(fp32 ? (size_t)std::max<int64_t>(df_elems, 1) * 4 : 0);
  L.total = off;
  return L;
}

kiops_status ensure_workspace(kiops_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return KIOPS_OK;
  if (!ctx->ws_owned && ctx->ws)
    return fail(ctx, KIOPS_ENOMEM, "attached workspace has %zu bytes, the solve needs %zu", ctx->ws_bytes, bytes);
  if (ctx->ws_owned && ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  ctx->ws_owned = false;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(ctx, KIOPS_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  ctx->ws = p;
  ctx->ws_bytes = bytes;
  ctx->ws_owned = true;
  return KIOPS_OK;
}

kiops_status ensure_pinned(kiops_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->host_pinned_bytes) return KIOPS_OK;
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  ctx->host_pinned = nullptr;
  ctx->host_pinned_bytes = 0;
  KCHECK(ctx, cudaMallocHost(&ctx->host_pinned, bytes));
  ctx->host_pinned_bytes = bytes;
  return KIOPS_OK;
}

int grid_size(kiops_ctx* ctx, void* fn, int threads = kThreads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, kDynSmem) != cudaSuccess) return 0;
  int g = per_sm * ctx->sms;
  if (ctx->cfg.grid_blocks > 0) g = std::min(g, ctx->cfg.grid_blocks);
  return g;
}

kiops_status prepare_kernel(kiops_ctx* ctx, void* fn) {
  KCHECK(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem));
  return KIOPS_OK;
}

// 2D tiling of an nx x ny grid over at most `tiles` tiles for the lagged-normalisation path: smallest
// tile area whose halo'd tile (ns species, element size elem) fits the dynamic shared memory; ties go to
// the wider tile (coalesced rows).  Returns false if no tiling fits.
bool choose_tiles_k(int64_t nx, int64_t ny, int ns, int tiles, size_t elem, int& gx, int& gy, int& tw, int& th) {
  int64_t best = -1;
  for (int cx = 1; cx <= tiles && cx <= nx; ++cx) {
    const int cy = (int)std::min<int64_t>(tiles / cx, ny);
    if (cy < 1) continue;
    const int w = (int)((nx + cx - 1) / cx), h = (int)((ny + cy - 1) / cy);
    const size_t smem = (size_t)ns * (w + 2) * (h + 2) * elem;
    if (smem > kDynSmem) continue;
    const int64_t area = (int64_t)w * h;
    if (best < 0 || area < best || (area == best && w > tw)) {
      best = area;
      tw = w;
      th = h;
      gx = (int)((nx + w - 1) / w);
      gy = (int)((ny + h - 1) / h);
    }
  }
  return best > 0;
}

bool choose_tiles(int64_t nx, int64_t ny, int ns, int blocks, size_t elem, int& gx, int& gy, int& tw, int& th) {
  // the fewest tiles per block (k) for which a tile with its halo fits the tile buffer: k = 1 is one tile
  // per block; larger grids give each block k tiles in turn
  for (int k = 1; k <= kMaxTilesPerBlock; ++k)
    if (choose_tiles_k(nx, ny, ns, k * blocks, elem, gx, gy, tw, th)) return true;
  return false;
}

struct Prepared {
  SolveArgs args;
  Layout L;
  char* base;
  size_t dyn_smem = kDynSmem;  // dynamic shared memory of the launch
  size_t tma_b = 0, tma_f = 0;  // TMA path: workspace offsets of the staged copies of B (FP64) and the fields
  TmaMaps maps{};               // TMA path: tensor maps (a kernel parameter)
};

// ---- TMA path of the several-tiles 2D step (grid engine) --------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    cudaGetLastError();
  }
  return fn;
}

// Tile shape, stages and shared-memory layout of the TMA path, if it applies and keeps `blocks` blocks
// co-resident; the workspace grows by the tensor maps and the staged copies of B (FP64) and the fields.
// fn: the general instantiation; fn_fixed (or null): the one compiled for 32 x 16 tiles, two species and
// p = 3 (same stage layout).  On success *use_fixed tells which to launch.
bool setup_tma(kiops_ctx* ctx, void* fn, void* fn_fixed, int blocks, int threads, Prepared& P, bool* use_fixed) {
  SolveArgs& a = P.args;
  // automatic (tma = 1): FP32 basis only.  FP64 steps are bound by the FP64 pipe, and the staged path measured
  // slower there (2048^2 ADR 190 -> 202 us per step, 1024^2 Gray-Scott 8.9 -> 11.9 ms per solve)
  if (!a.fused || ctx->cfg.tma <= 0 || a.op.kind != OP_ST2D || (ctx->cfg.tma == 1 && !a.prec)) return false;
  if ((int64_t)a.tile_gx * a.tile_gy <= blocks) return false;  // one tile per block: the shared-memory extras
  const size_t es = a.prec ? 4 : 8;
  const int64_t nx = a.op.nx, ny = a.op.ny, npts = nx * ny;
  const int ns = a.op.nspecies, p = a.p;
  if ((nx * (int64_t)es) % 16 != 0 || (npts * (int64_t)es) % 16 != 0 || nx > (1 << 30) || ny > (1 << 30)) return false;
  if (!tensor_map_encoder()) return false;
  // staged planes and the constants that turn them into the block's entries (SolveArgs::tma_aff_*)
  int nf = 0, fidx[2][2] = {{-1, -1}, {-1, -1}};
  double aff[2][4] = {};
  for (int sp = 0; sp < ns; ++sp) {
    double* f = aff[sp];
    f[0] = a.op.coef[sp][0];
    f[1] = f[3] = 1.0;
  }
  if (a.op.nfields > 0) {  // shared coupling fields: one plane per field
    nf = a.op.nfields;
    for (int sp = 0; sp < ns; ++sp)
      for (int q = 0; q < ns; ++q) {
        const int k = a.op.dfield[sp][q];
        const double c0 = a.op.dconst[sp][q], w = a.op.dweight[sp][q];
        if (q == sp) {
          if (k >= 0) {
            fidx[sp][q] = k;
            aff[sp][1] = w;
          }
          aff[sp][0] += c0;  // the own entry's constant joins the centre coefficient
        } else if (k >= 0 || c0 != 0.0) {
          fidx[sp][q] = k >= 0 ? k : 0;  // a constant entry: any plane with weight 0
          aff[sp][2] = c0;
          aff[sp][3] = k >= 0 ? w : 0.0;
        }
      }
  } else {
    for (int sp = 0; sp < ns; ++sp)
      for (int q = 0; q < ns; ++q)
        if (a.op.diag[sp][q]) fidx[sp][q] = nf++;
  }
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->cfg.device) != cudaSuccess) return false;
  const int S = ctx->cfg.tma_stages >= 3 && ctx->cfg.tma_stages <= 6 ? ctx->cfg.tma_stages : 2;
  const int pad = (int)(16 / es);
  auto up = [](size_t x) { return (x + 127) & ~(size_t)127; };
  // candidates: the configured shape, then the automatic order (wide rows first)
  // automatic shapes, measured on 2048^2 Gray-Scott (FP32 basis): 32 x 16 best; every shape gives each thread
  // at least one 16-byte item of own points
  const int auto_shapes[][2] = {{32, 16}, {64, 8}, {128, 4}, {16, 32}, {64, 4}, {32, 8}};
  std::vector<std::pair<int, int>> cand;
  if (ctx->cfg.tile_w > 0 && ctx->cfg.tile_h > 0) cand.push_back({ctx->cfg.tile_w, ctx->cfg.tile_h});
  for (auto& sh : auto_shapes) cand.push_back({sh[0], sh[1]});
  for (auto [tw, th] : cand)
  for (int variant = 0; variant < 2; ++variant) {  // the fixed-shape kernel first, where it applies
    const bool fixed = variant == 0;
    if (fixed && !(fn_fixed && es == 4 && tw == 32 && th == 16 && ns == 2 && p == 3))
      continue;
    void* f = fixed ? fn_fixed : fn;
    const int Sv = S;
    if (tw < 4 || tw % 4 != 0 || th < 1 || tw > 248 || th > 254) continue;
    const int bw = tw + 2 * pad, bh = th + 2;
    const int64_t gx = (nx + tw - 1) / tw, gy = (ny + th - 1) / th;
    if (gx * gy <= blocks || gx * gy > INT32_MAX) continue;
    const size_t box = up((size_t)bw * bh * ns * es);
    const size_t off_f = box, off_b = off_f + (size_t)a.m_o * box;
    const size_t off_d = off_b + up((size_t)p * ns * tw * th * es);
    const size_t stage = up(off_d + up((size_t)nf * tw * th * es));
    const size_t bar_off = std::max((size_t)Sv * stage, up(kDynSmem));
    const size_t side_off = bar_off + 64;                       // after the stage barriers (<= 6)
    const size_t dyn = side_off + (size_t)threads * 4 * es + 128;  // landing slots, alignment slack
    if (dyn > (size_t)optin) continue;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) continue;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, dyn) != cudaSuccess) continue;
    if ((int64_t)per_sm * ctx->sms < blocks) continue;
    *use_fixed = fixed;
    a.tma_on = 1;
    a.tma_stages = Sv;
    // L2 prefetch ahead of the staged copies: off unless asked for (2048^2 Gray-Scott FP32: 117 us per step
    // without, 122 us with 2 tiles beyond the stages)
    a.tma_prefetch = ctx->cfg.tma_prefetch < 0 ? 0 : std::min(ctx->cfg.tma_prefetch, 64);
    a.tma_pad = pad;
    a.tma_bw = bw;
    a.tma_bh = bh;
    a.tma_nf = nf;
    for (int sp = 0; sp < 2; ++sp) {
      for (int q = 0; q < 2; ++q) a.tma_fidx[sp][q] = fidx[sp][q];
      for (int k = 0; k < 4; ++k) {
        a.tma_aff_d[sp][k] = aff[sp][k];
        a.tma_aff_f[sp][k] = (float)aff[sp][k];
      }
    }
    a.tma_stage_bytes = (int)stage;
    a.tma_box_bytes = (int)box;
    a.tma_off_f = (int)off_f;
    a.tma_off_b = (int)off_b;
    a.tma_off_d = (int)off_d;
    a.tma_bar_off = (int)bar_off;
    a.tma_side_off = (int)side_off;
    a.tile_w = tw;
    a.tile_h = th;
    a.tile_gx = (int)gx;
    a.tile_gy = (int)gy;
    P.dyn_smem = dyn;
    Layout& L = P.L;
    P.tma_b = align_up(L.total, 256);
    P.tma_f = align_up(P.tma_b + (a.prec ? 0 : (size_t)p * a.ldv * 8), 256);
    L.total = align_up(P.tma_f + (size_t)nf * npts * es, 256);
    return true;
  }
  cudaGetLastError();
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
  return false;
}

// 3D stencils with an FP32 basis: lagged normalisation on 3D tiles whose operands are staged by bulk tensor
// copies (fused_st3d_tma).  Stage: halo'd boxes of raw x_j and of the m_o window vectors, (tile_w + 8) x
// (tile_h + 2) x (tile_d + 2) points each, and the own-point box of the reaction field if the operator has one;
// the B columns go through per-thread slots (cp.async).  Candidate tiles give each thread one 16-byte item of own
// points; the first whose stages fit at the launch's block count is taken.  Needs more tiles than blocks and
// rows of a multiple of 16 bytes.
// fn_fixed (or null): the instantiation compiled for 32 x 8 x 4 tiles; *use_fixed tells which to launch.
bool setup_tma3d(kiops_ctx* ctx, void* fn, void* fn_fixed, int blocks, int threads, Prepared& P, bool* use_fixed) {
  SolveArgs& a = P.args;
  if (ctx->cfg.tma <= 0 || !ctx->cfg.fuse_stencil || a.op.kind != OP_ST3D || !a.prec || a.m_o > kChunk) return false;
  const int64_t nx = a.op.nx, ny = a.op.ny, nz = a.op.nz;
  if (nx % 4 != 0 || nx * ny * nz >= ((int64_t)1 << 31) || !tensor_map_encoder()) return false;
  const bool hasf = a.op.diag[0][0] != nullptr;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->cfg.device) != cudaSuccess) return false;
  const int S = ctx->cfg.tma_stages >= 3 && ctx->cfg.tma_stages <= 6 ? ctx->cfg.tma_stages : 2;
  auto up = [](size_t x) { return (x + 127) & ~(size_t)127; };
  const int shapes[][3] = {{32, 8, 4}, {64, 4, 4}, {16, 8, 8}, {32, 4, 8}};
  for (auto& sh : shapes)
  for (int variant = 0; variant < 2; ++variant) {  // the fixed-shape kernel first, where it applies
    const int tw = sh[0], th = sh[1], td = sh[2];
    const bool fixed = variant == 0;
    if (fixed && !(fn_fixed && tw == 32 && th == 8 && td == 4)) continue;
    void* f = fixed ? fn_fixed : fn;
    const int64_t gx = (nx + tw - 1) / tw, gy = (ny + th - 1) / th, gz = (nz + td - 1) / td;
    if (gx * gy * gz <= blocks || gx * gy * gz > INT32_MAX) continue;
    const int bw = tw + 8, bh = th + 2, bd = td + 2;
    const size_t box = up((size_t)bw * bh * bd * 4);
    const size_t off_f = box, off_d = off_f + (size_t)a.m_o * box;
    const size_t stage = up(off_d + (hasf ? (size_t)tw * th * td * 4 : 0));
    const size_t bar_off = std::max((size_t)S * stage, up(kDynSmem));
    const size_t side_off = bar_off + 64;                      // per-thread B slots: four 16-byte vectors
    const size_t dyn = side_off + (size_t)threads * 64 + 128;  // alignment slack
    if (dyn > (size_t)optin) continue;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) continue;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, dyn) != cudaSuccess) continue;
    if ((int64_t)per_sm * ctx->sms < blocks) continue;
    *use_fixed = fixed;
    a.fused = 1;
    a.tma_on = 1;
    a.tma_stages = S;
    a.tma_prefetch = 0;
    a.tma_pad = 4;
    a.tma_bw = bw;
    a.tma_bh = bh;
    a.tma_bd = bd;
    a.tma_nf = hasf ? 1 : 0;
    a.tma_stage_bytes = (int)stage;
    a.tma_box_bytes = (int)box;
    a.tma_off_f = (int)off_f;
    a.tma_off_b = (int)off_d;
    a.tma_off_d = (int)off_d;
    a.tma_bar_off = (int)bar_off;
    a.tma_side_off = (int)side_off;
    a.tile_w = tw;
    a.tile_h = th;
    a.tile_d = td;
    a.tile_gx = (int)gx;
    a.tile_gy = (int)gy;
    a.tile_gz = (int)gz;
    P.dyn_smem = dyn;
    return true;
  }
  cudaGetLastError();
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
  return false;
}

// The four tensor maps of the TMA path (basis, raw ring, B columns, coupling fields) for the bound
// workspace, into P.maps (passed to the kernel as a grid-constant parameter).
// Tensor maps of the 3D staged path (FP32 basis): the basis and the raw ring as 4D {nx, ny, nz, column} with
// halo'd boxes, the reaction field (its FP32 copy) as 3D with own-point boxes.
kiops_status encode_tma_maps_3d(kiops_ctx* ctx, Prepared& P) {
  SolveArgs& a = P.args;
  std::memset(&P.maps, 0, sizeof(P.maps));
  CUtensorMap* m = (CUtensorMap*)P.maps.m;
  auto enc = tensor_map_encoder();
  const cuuint64_t nx = (cuuint64_t)a.op.nx, ny = (cuuint64_t)a.op.ny, nz = (cuuint64_t)a.op.nz, es = 4;
  const cuuint32_t one[4] = {1, 1, 1, 1};
  auto check = [&](CUresult r, const char* what) -> kiops_status {
    if (r != CUDA_SUCCESS) return fail(ctx, KIOPS_ECUDA, "tensor map of the %s: error %d", what, (int)r);
    return KIOPS_OK;
  };
  const cuuint64_t st[3] = {nx * es, nx * ny * es, (cuuint64_t)a.ldv * es};
  const cuuint32_t box[4] = {(cuuint32_t)a.tma_bw, (cuuint32_t)a.tma_bh, (cuuint32_t)a.tma_bd, 1};
  const cuuint64_t dv[4] = {nx, ny, nz, (cuuint64_t)a.m_max + 1};
  kiops_status r = check(enc(&m[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.V, dv, st, box, one,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE), "basis");
  if (r) return r;
  const cuuint64_t dr[4] = {nx, ny, nz, 2};
  r = check(enc(&m[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.raw, dr, st, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE),
            "raw vectors");
  if (r) return r;
  if (a.tma_nf > 0) {
    const cuuint64_t sf[2] = {nx * es, nx * ny * es};
    const cuuint32_t bf[3] = {(cuuint32_t)a.tile_w, (cuuint32_t)a.tile_h, (cuuint32_t)a.tile_d};
    const cuuint64_t df[3] = {nx, ny, nz};
    r = check(enc(&m[3], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.df, df, sf, bf, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE),
              "reaction field");
    if (r) return r;
  }
  return KIOPS_OK;
}

kiops_status encode_tma_maps(kiops_ctx* ctx, Prepared& P) {
  SolveArgs& a = P.args;
  if (a.op.kind == OP_ST3D) return encode_tma_maps_3d(ctx, P);
  a.tma_b = a.prec ? (void*)a.bf : (void*)(P.base + P.tma_b);
  a.tma_f = P.base + P.tma_f;
  std::memset(&P.maps, 0, sizeof(P.maps));
  static_assert(sizeof(CUtensorMap) == 128 && sizeof(TmaMaps) == 512, "tensor map size");
  CUtensorMap* m = (CUtensorMap*)P.maps.m;
  auto enc = tensor_map_encoder();
  const CUtensorMapDataType dt = a.prec ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint64_t es = a.prec ? 4 : 8;
  const cuuint64_t nx = (cuuint64_t)a.op.nx, ny = (cuuint64_t)a.op.ny, ns = (cuuint64_t)a.op.nspecies;
  const cuuint32_t one[4] = {1, 1, 1, 1};
  auto check = [&](CUresult r, const char* what) -> kiops_status {
    if (r != CUDA_SUCCESS) return fail(ctx, KIOPS_ECUDA, "tensor map of the %s: error %d", what, (int)r);
    return KIOPS_OK;
  };
  {  // halo'd boxes of the basis and of the raw ring
    const cuuint64_t st[3] = {nx * es, nx * ny * es, (cuuint64_t)a.ldv * es};
    const cuuint32_t box[4] = {(cuuint32_t)a.tma_bw, (cuuint32_t)a.tma_bh, (cuuint32_t)ns, 1};
    const cuuint64_t dv[4] = {nx, ny, ns, (cuuint64_t)a.m_max + 1};
    kiops_status r = check(enc(&m[0], dt, 4, a.V, dv, st, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE), "basis");
    if (r) return r;
    const cuuint64_t dr[4] = {nx, ny, ns, 2};
    r = check(enc(&m[1], dt, 4, a.raw, dr, st, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE), "raw vectors");
    if (r) return r;
  }
  if (a.p > 0) {  // own-point box of the p B columns
    const cuuint64_t st[3] = {nx * es, nx * ny * es, (cuuint64_t)a.ldv * es};
    const cuuint32_t box[4] = {(cuuint32_t)a.tile_w, (cuuint32_t)a.tile_h, (cuuint32_t)ns, (cuuint32_t)a.p};
    const cuuint64_t d[4] = {nx, ny, ns, (cuuint64_t)a.p};
    kiops_status r = check(enc(&m[2], dt, 4, a.tma_b, d, st, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE), "B columns");
    if (r) return r;
  }
  if (a.tma_nf > 0) {  // own-point box of the coupling fields
    const cuuint64_t st[2] = {nx * es, nx * ny * es};
    const cuuint32_t box[3] = {(cuuint32_t)a.tile_w, (cuuint32_t)a.tile_h, (cuuint32_t)a.tma_nf};
    const cuuint64_t d[3] = {nx, ny, (cuuint64_t)a.tma_nf};
    kiops_status r = check(enc(&m[3], dt, 3, a.tma_f, d, st, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE), "coupling fields");
    if (r) return r;
  }
  return KIOPS_OK;
}

// Grid engine, tiled path: shared-memory extras of the fused phase, all placed over the exponential's
// region (which invalidates them).  Ring: finalised tiles of the last m_o + 1 basis vectors; stage: the
// next raw tile prefetched during the cross-block sum; cache: the tile's B columns and coupling fields.
// The first combination that still leaves `blocks` co-resident blocks is taken.
void enable_fused_smem(kiops_ctx* ctx, void* fn, int blocks, Prepared& P, int threads = kThreads) {
  SolveArgs& a = P.args;
  if (!a.fused) return;
  if ((int64_t)a.tile_gx * a.tile_gy > blocks) return;  // several tiles per block: none of the extras
  const size_t elem = a.prec ? 4 : 8;
  const int ns = a.op.nspecies;
  const size_t halo_pts = (size_t)ns * (a.tile_w + 2) * (a.tile_h + 2);
  const size_t tile = halo_pts * elem;
  const size_t cache = (size_t)(a.p + ns) * ns * a.tile_w * a.tile_h * elem;
  auto up = [](size_t x) { return (x + 127) & ~(size_t)127; };
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->cfg.device) != cudaSuccess) return;
  // automatic: preferred combinations (1 ring, 2 stage, 4 cache), measured on the 512^2 ADR (all three
  // best) and 1024^2 Gray-Scott FP32 (only the ring fits with two blocks per SM, and beats the stage)
  const int order[7] = {7, 3, 5, 1, 6, 2, 4};
  const int forced = ctx->cfg.fused_smem;
  for (int ci = 0; ci < (forced >= 0 ? 1 : 7); ++ci) {
    const int mask = forced >= 0 ? (forced & 7) : order[ci];
    if (mask == 0) break;
    const int cb[3] = {mask & 1, (mask >> 1) & 1, (mask >> 2) & 1};
    const int nr = cb[0] ? a.m_o + 1 : 0;
    const size_t ring_b = up((size_t)(nr > 0 ? nr : 1) * tile);
    const size_t stage_b = cb[1] ? up(tile) : 0;
    const size_t tbl_b = cb[1] ? up(halo_pts * 4) : 0;
    const size_t cache_b = cb[2] ? up(cache) : 0;
    const size_t dyn = std::max(kDynSmem, ring_b + stage_b + tbl_b + cache_b);
    if (dyn > (size_t)optin) continue;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) continue;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, dyn) != cudaSuccess) continue;
    if ((int64_t)per_sm * ctx->sms < blocks) continue;
    a.ring_n = nr;
    a.stage_on = cb[1];
    a.cache_on = cb[2];
    a.sm_stage = (int)(ring_b / 8);
    a.sm_tbl = (int)((ring_b + stage_b) / 8);
    a.sm_cache = (int)((ring_b + stage_b + tbl_b) / 8);
    P.dyn_smem = dyn;
    return;
  }
  cudaGetLastError();
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
}

// Validate one request and fill its argument block.
kiops_status prepare(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b, double tol,
                     int m_init, int m_o, kiops_precision prec, double* w, int grid_blocks, int64_t trace_cap,
                     Prepared& P) {
  if (!A || !b || !w) return fail(ctx, KIOPS_EINVAL, "NULL operator, b or w");
  if (A->ctx != ctx) return fail(ctx, KIOPS_EINVAL, "operator belongs to another context");
  if (p < 0 || p > KIOPS_MAX_P) return fail(ctx, KIOPS_EINVAL, "p = %d outside [0, %d]", p, KIOPS_MAX_P);
  if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(ctx, KIOPS_EINVAL, "tau must be finite and >= 0");
  if (!(tol > 0.0)) return fail(ctx, KIOPS_EINVAL, "tol must be > 0");
  if (m_init < 1) return fail(ctx, KIOPS_EINVAL, "m_init must be >= 1");
  if (m_o < 1) return fail(ctx, KIOPS_EINVAL, "m_o must be >= 1");
  if (prec != KIOPS_FP64 && prec != KIOPS_FP32_BASIS) return fail(ctx, KIOPS_EINVAL, "unknown precision");
  for (int k = 0; k <= p; ++k)
    if (!b[k]) return fail(ctx, KIOPS_EINVAL, "b[%d] is NULL", k);
  const int m_max = ctx->cfg.m_max;
  const int m_o_eff = std::min(m_o, m_max + 1);
  std::memset(&P.args, 0, sizeof(SolveArgs));
  SolveArgs& a = P.args;
  a.op = A->d;
  a.N = A->d.n;
  a.p = p;
  a.T_end = tau;
  a.tol = tol;
  a.m_init = m_init;
  a.m_min = ctx->cfg.m_min;
  a.m_max = m_max;
  a.m_o = m_o_eff;
  a.normalize = ctx->cfg.normalize_B;
  a.bd_tol = ctx->cfg.breakdown_tol;
  a.max_substeps = ctx->cfg.max_substeps;
  a.max_iters = ctx->cfg.max_iterations;
  for (int k = 0; k <= p; ++k) a.b[k] = b[k];
  a.w = w;
  a.timeout_ns = (long long)(ctx->cfg.timeout_s * 1e9);
  a.tt = ctx->tt;
  a.trace_cap = trace_cap;
  a.prec = prec == KIOPS_FP32_BASIS ? 1 : 0;
  a.scenario = ctx->cfg.scenario == 1 ? 1 : 0;
  a.nz_op = A->nz;
  int64_t ldv = 0;
  int64_t df_elems = 0;  // FP32 copies of the coupling fields: nspecies^2 fields of the grid's points
  if (A->d.kind == OP_ST2D) df_elems = (int64_t)A->d.nspecies * A->d.nspecies * A->d.nx * A->d.ny;
  if (A->d.kind == OP_ST3D) df_elems = A->d.nx * A->d.ny * A->d.nz;
  P.L = layout(a.N, p, m_max, m_o_eff, prec == KIOPS_FP32_BASIS, grid_blocks, max_r(ctx->tt), trace_cap, &ldv,
               df_elems);
  a.ldv = ldv;
  a.fused = 0;
  // (the tiled path codes a grid index r as 2 r + 1 in 32 bits)
  if (A->d.kind == OP_ST2D && m_o_eff <= kChunk && grid_blocks > 1 && ctx->cfg.fuse_stencil &&
      (int64_t)A->d.nspecies * A->d.nx * A->d.ny < ((int64_t)1 << 31)) {
    int gx = 0, gy = 0, tw = 0, th = 0;
    if (choose_tiles(A->d.nx, A->d.ny, A->d.nspecies, grid_blocks, prec == KIOPS_FP32_BASIS ? 4 : 8, gx, gy, tw, th)) {
      a.fused = 1;
      a.tile_gx = gx;
      a.tile_gy = gy;
      a.tile_w = tw;
      a.tile_h = th;
    }
  }
  return KIOPS_OK;
}

void bind(Prepared& P, char* base) {
  SolveArgs& a = P.args;
  const Layout& L = P.L;
  P.base = base;
  a.V = base + L.V;
  a.H = (double*)(base + L.H);
  a.gram = (double*)(base + L.gram);
  a.mats = (double*)(base + L.mats);
  a.fvec = (double*)(base + L.fvec);
  a.partials = (double*)(base + L.partials);
  a.bar = (unsigned int*)(base + L.bar);
  a.abort_flag = (int*)(base + L.bar + 64);
  a.stats = (int64_t*)(base + L.stats);
  a.stats_d = (double*)(base + L.stats + 10 * 8);
  a.trace_len = (int64_t*)(base + L.trace_len);
  a.trace = a.trace_cap > 0 ? (TraceRec*)(base + L.trace) : nullptr;
  a.prof = nullptr;
  a.raw = base + L.raw;
  a.bf = (float*)(base + L.bf);
  a.df = (float*)(base + L.df);
}

void fill_stats(kiops_stats* st, const int64_t* s, const double* sd, int engine, int blocks) {
  if (!st) return;
  std::memset(st->phase_cycles, 0, sizeof(st->phase_cycles));
  st->substeps = s[0];
  st->rejected = s[1];
  st->matvecs = s[2];
  st->iterations = s[3];
  st->expm_calls = s[4];
  st->m_last = (int)s[5];
  st->status = (int)s[6];
  st->engine = engine;
  st->grid_blocks = blocks;
  st->err_est = sd[0];
  st->tile_path = st->tile_w = st->tile_h = 0;
}

// One solve on the grid engine (or a single-block CTA launch).
kiops_status run_single(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b, double tol,
                        int m_init, int m_o, kiops_precision prec, double* w, kiops_stats* stats,
                        kiops_trace_rec* trace, int64_t trace_cap, int64_t* trace_len, const double* times = nullptr,
                        int n_times = 0, double* const* wout = nullptr) {
  NvtxRange nvtx_range("kiops solve");
  if (!ctx) return KIOPS_EINVAL;
  if (trace_len) *trace_len = 0;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (tau == 0.0 && A && b && w && b[0]) {  // w = b_0, no work (Algorithm 1)
    if (w != b[0]) KCHECK(ctx, cudaMemcpyAsync(w, b[0], (size_t)A->d.n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
    if (stats) stats->m_last = std::max(ctx->cfg.m_min, std::min(m_init, ctx->cfg.m_max));
    return KIOPS_OK;
  }
  const bool fp32 = prec == KIOPS_FP32_BASIS;
  int engine = ctx->cfg.engine == KIOPS_ENGINE_CTA ? KIOPS_ENGINE_CTA : KIOPS_ENGINE_GRID;
  if (!A) return fail(ctx, KIOPS_EINVAL, "NULL operator");
  if (engine == KIOPS_ENGINE_CTA) {  // one block: a batch of one request on a one-block team
    if (trace) return fail(ctx, KIOPS_EINVAL, "traces are recorded by the grid engine only");
    kiops_request r{A, tau, p, b, tol, m_init, m_o, prec, w};
    const int saved = ctx->cfg.batch_team_blocks;
    ctx->cfg.batch_team_blocks = 1;
    kiops_status st = batch_teams(ctx, 1, &r, stats);
    ctx->cfg.batch_team_blocks = saved;
    if (stats) stats->engine = KIOPS_ENGINE_CTA;
    return st;
  }
  void* fn = pick_kernel(fp32, A->d.kind);
  int threads = kThreads;
  // automatic block size (measured): latency-bound small problems gain from half the blocks to reduce over
  // and synchronise (400-point CSR: -5.5 %); from 512^2 on the two sizes are within 1 %
  const int bt = ctx->cfg.block_threads != 0 ? ctx->cfg.block_threads : (A->d.n <= 65536 ? 512 : 256);
  if (engine == KIOPS_ENGINE_GRID && !fp32 && bt == 512) {
    fn = kiops_k::solve_kernel_f64_wide(A->d.kind);
    threads = kiops_k::wide_threads();
  }
  kiops_status st = prepare_kernel(ctx, fn);
  if (st) return st;
  int blocks = engine == KIOPS_ENGINE_GRID ? grid_size(ctx, fn, threads) : 1;
  if (blocks < 1) return fail(ctx, KIOPS_ECUDA, "kernel does not fit on the device");
  // automatic (measured): FP64 problems of up to 2^19 unknowns keep their step's vectors in L2 and are
  // bound by the FP64 pipe, which 8 warps per SM keep as busy as 16; one 256-thread block per SM then
  // halves the blocks to reduce over and synchronise (512^2 ADR: 6.24 -> 5.91 ms).  Larger problems stream
  // from HBM and keep two blocks per SM (1024^2 ADR: 7.7 ms vs 9.4 ms with one).
  if (engine == KIOPS_ENGINE_GRID && !fp32 && ctx->cfg.block_threads == 0 && ctx->cfg.grid_blocks == 0 &&
      threads == kThreads && A->d.n > 65536 && A->d.n <= ((int64_t)1 << 19))
    blocks = std::min(blocks, ctx->sms);
  Prepared P;
  st = prepare(ctx, A, tau, p, b, tol, m_init, m_o, prec, w, blocks, trace ? trace_cap : 0, P);
  if (st) return st;
  if (n_times > 0) {  // Task I: the running state lives in the last output
    P.args.n_times = n_times;
    for (int l = 0; l < n_times; ++l) {
      P.args.times[l] = times[l];
      P.args.wout[l] = wout[l];
    }
  }
  void* fn_tma = (A->d.kind == OP_ST2D && threads == kThreads) ? kiops_k::solve_kernel_tma(fp32) : nullptr;
  // the instantiation compiled for 32 x 16 tiles, two species and p = 3 (FP32 basis)
  void* fn_fixed = fn_tma && fp32 && ctx->cfg.tma_fixed != 0 ? kiops_k::solve_kernel_tma_fixed() : nullptr;
  bool use_fixed = false;
  if (engine == KIOPS_ENGINE_GRID && fn_tma && prepare_kernel(ctx, fn_tma) == KIOPS_OK &&
      (!fn_fixed || prepare_kernel(ctx, fn_fixed) == KIOPS_OK) &&
      setup_tma(ctx, fn_tma, fn_fixed, blocks, threads, P, &use_fixed)) {
    fn = use_fixed ? fn_fixed : fn_tma;  // an instantiation with the bulk-tensor-copy path
  } else if (void* fn3 = (engine == KIOPS_ENGINE_GRID && A->d.kind == OP_ST3D && fp32 && threads == kThreads)
                             ? kiops_k::solve_kernel_tma3d() : nullptr;
             fn3 && prepare_kernel(ctx, fn3) == KIOPS_OK &&
             (ctx->cfg.tma_fixed == 0 || prepare_kernel(ctx, kiops_k::solve_kernel_tma3d_fixed()) == KIOPS_OK) &&
             setup_tma3d(ctx, fn3, ctx->cfg.tma_fixed != 0 ? kiops_k::solve_kernel_tma3d_fixed() : nullptr, blocks,
                         threads, P, &use_fixed)) {
    fn = use_fixed ? kiops_k::solve_kernel_tma3d_fixed() : fn3;  // 3D tiles staged by bulk tensor copies
  } else if (engine == KIOPS_ENGINE_GRID)
    enable_fused_smem(ctx, fn, blocks, P, threads);
  st = ensure_workspace(ctx, P.L.total);
  if (st) return st;
  bind(P, (char*)ctx->ws);
  if (ctx->cfg.profile) P.args.prof = (long long*)(P.base + P.L.prof);
  const size_t tr_bytes = (size_t)(trace ? trace_cap : 0) * sizeof(TraceRec);
  st = ensure_pinned(ctx, sizeof(SolveArgs) + 512 + tr_bytes);
  if (st) return st;
  char* hp = (char*)ctx->host_pinned;
  if (P.args.tma_on) {
    st = encode_tma_maps(ctx, P);
    if (st) return st;
  }
  std::memcpy(hp, &P.args, sizeof(SolveArgs));
  KCHECK(ctx, cudaMemsetAsync(P.base + P.L.bar, 0, 256 + 16 * 8 + 256, ctx->stream));
  KCHECK(ctx, cudaMemsetAsync(P.base + P.L.trace_len, 0, 8, ctx->stream));
  if (ctx->cfg.profile) KCHECK(ctx, cudaMemsetAsync(P.base + P.L.prof, 0, 16 * 8, ctx->stream));
  KCHECK(ctx, cudaMemcpyAsync(P.base + P.L.args, hp, sizeof(SolveArgs), cudaMemcpyHostToDevice, ctx->stream));
  const SolveArgs* dargs = (const SolveArgs*)(P.base + P.L.args);
  void* kargs[] = {(void*)&dargs, (void*)&P.maps};
  KCHECK(ctx, cudaLaunchCooperativeKernel(fn, blocks, threads, kargs, P.dyn_smem, ctx->stream));
  int64_t* hs = (int64_t*)(hp + sizeof(SolveArgs) + 0);
  KCHECK(ctx, cudaMemcpyAsync(hs, P.base + P.L.stats, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream));
  int64_t* htl = hs + 15;
  KCHECK(ctx, cudaMemcpyAsync(htl, P.base + P.L.trace_len, 8, cudaMemcpyDeviceToHost, ctx->stream));
  int64_t* hprof = hs + 16;
  if (ctx->cfg.profile)
    KCHECK(ctx, cudaMemcpyAsync(hprof, P.base + P.L.prof, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream));
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  if (trace && trace_cap > 0) {
    int64_t n = std::min(*htl, trace_cap);
    std::vector<TraceRec> tmp((size_t)n);
    if (n > 0)
      KCHECK(ctx, cudaMemcpy(tmp.data(), P.base + P.L.trace, (size_t)n * sizeof(TraceRec), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) {
      trace[i].substep = tmp[i].substep;
      trace[i].j = tmp[i].j;
      trace[i].accepted = tmp[i].accepted;
      trace[i].breakdown = tmp[i].breakdown;
      trace[i].m_new = tmp[i].m_new;
      trace[i].tau = tmp[i].tau;
      trace[i].t_now = tmp[i].t_now;
      trace[i].eps = tmp[i].eps;
      trace[i].omega = tmp[i].omega;
      trace[i].tau_new = tmp[i].tau_new;
      trace[i].cost_a = tmp[i].cost_a;
      trace[i].cost_b = tmp[i].cost_b;
      trace[i].hnorm = tmp[i].hnorm;
    }
    if (trace_len) *trace_len = n;
  }
  const double* hsd = (const double*)(hs + 10);
  fill_stats(stats, hs, hsd, engine, blocks);
  if (stats && ctx->cfg.profile) std::memcpy(stats->phase_cycles, hprof, 16 * 8);
  if (stats && P.args.fused && P.args.op.kind == OP_ST3D) {
    stats->tile_path = 4;  // 3D tiles staged by bulk tensor copies
    stats->tile_w = P.args.tile_w;
    stats->tile_h = P.args.tile_h;
  } else if (stats && P.args.fused && (int64_t)P.args.tile_gx * P.args.tile_gy > blocks) {
    stats->tile_path = !P.args.tma_on ? 1 : (fn == fn_tma ? 2 : 3);
    stats->tile_w = P.args.tile_w;
    stats->tile_h = P.args.tile_h;
  }
  const int dst = (int)hs[6];
  if (dst == ST_ETIMEOUT) return fail(ctx, KIOPS_ETIMEOUT, "a device-side wait exceeded %.3g s", ctx->cfg.timeout_s);
  if (dst == ST_ENOTCONV)
    return fail(ctx, KIOPS_ENOTCONV, "no convergence within max_substeps/max_iterations (%lld iterations)",
                (long long)hs[3]);
  if (dst != ST_OK) return fail(ctx, (kiops_status)dst, "device status %d", dst);
  return KIOPS_OK;
}

// Entry of a pointwise coupling block given by a shared field: out = fma(w, f, c), or c without a field.
__global__ void coupling_entry_kernel(const double* f, double w, double c, double* out, int64_t n) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    out[r] = f ? fma(w, __ldg(f + r), c) : c;
}

template <int KIND>
__global__ void op_apply_kernel(OpDesc op, const double* x, double* y) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < op.n; r += (int64_t)gridDim.x * blockDim.x)
    y[r] = apply_row<double, KIND>(op, x, r);
}

// One block of a two-block team passes the team barrier: the second arrival never comes, so the bounded
// wait gives up after timeout_ns, raises the abort flag with ST_ETIMEOUT and returns false.  out[0] = 1 if
// the barrier completed, out[1] = the abort flag.
__global__ void barrier_timeout_kernel(unsigned int* ctr, int* abort_flag, long long timeout_ns, int* out) {
  __shared__ int ok;
  GridTeam team{0, 2, ctr, abort_flag, timeout_ns, 0u};
  const bool passed = team.sync(&ok);
  if (threadIdx.x == 0) {
    out[0] = passed ? 1 : 0;
    out[1] = ld_volatile_int(abort_flag);
  }
}

}  // namespace

extern "C" {

kiops_status kiops_config_default(kiops_config* cfg) {
  if (!cfg) return KIOPS_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->m_min = 10;
  cfg->m_max = 128;
  cfg->normalize_B = 1;
  cfg->breakdown_tol = 1e-12;
  cfg->max_substeps = 1000000;
  cfg->max_iterations = 100000;
  cfg->timeout_s = 10.0;
  cfg->engine = KIOPS_ENGINE_AUTO;
  cfg->grid_blocks = 0;
  cfg->fuse_stencil = 1;
  cfg->batch_team_blocks = 0;
  cfg->fused_smem = -1;
  cfg->scenario = 0;
  cfg->block_threads = 0;
  cfg->tma = 1;
  cfg->tile_w = 0;
  cfg->tile_h = 0;
  cfg->tma_stages = 0;
  cfg->tma_prefetch = -1;
  cfg->tma_fixed = 1;
  return KIOPS_OK;
}

kiops_status kiops_constants(double out[6]) {
  if (!out) return KIOPS_EINVAL;
  out[0] = 1.4;  // delta, eq 39
  out[1] = 0.9;  // gamma, eq 44
  out[2] = 0.6;  // gamma_max, Algorithm 4
  out[3] = 2.0;  // kappa default, section 3.6.2
  out[4] = 5.0;  // tau clip factor, section 3.6.1
  out[5] = 2.0;  // m_o default, Algorithm 2
  return KIOPS_OK;
}

const char* kiops_status_string(kiops_status s) {
  switch (s) {
    case KIOPS_OK: return "ok";
    case KIOPS_EINVAL: return "invalid argument";
    case KIOPS_ENOMEM: return "out of memory";
    case KIOPS_ENOTCONV: return "not converged";
    case KIOPS_ETIMEOUT: return "device wait timed out";
    case KIOPS_ECUDA: return "CUDA error";
    case KIOPS_EBUSY: return "context busy";
  }
  return "unknown status";
}

kiops_status kiops_create(kiops_ctx** out, const kiops_config* cfg) {
  if (!out) return KIOPS_EINVAL;
  *out = nullptr;
  kiops_ctx* ctx = new (std::nothrow) kiops_ctx();
  if (!ctx) return KIOPS_ENOMEM;
  if (cfg) ctx->cfg = *cfg; else kiops_config_default(&ctx->cfg);
  const kiops_config& c = ctx->cfg;
  if (c.m_min < 1 || c.m_max < c.m_min || c.m_max > KIOPS_MAX_M || !(c.breakdown_tol >= 0) ||
      c.max_substeps < 1 || c.max_iterations < 1 || !(c.timeout_s > 0)) {
    delete ctx;
    return KIOPS_EINVAL;
  }
  if (cudaSetDevice(c.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess) {
    delete ctx;
    return KIOPS_ECUDA;
  }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c.device);
  if (!coop) {
    delete ctx;
    return KIOPS_ECUDA;
  }
  ctx->stream = (cudaStream_t)c.stream;
  build_taylor_table(ctx->tt);
  *out = ctx;
  return KIOPS_OK;
}

kiops_status kiops_server_stop(kiops_ctx* ctx);

kiops_status kiops_destroy(kiops_ctx* ctx) {
  if (!ctx) return KIOPS_EINVAL;
  if (ctx->server) kiops_server_stop(ctx);
  if (ctx->ws_owned && ctx->ws) cudaFree(ctx->ws);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  if (ctx->stage_dev) cudaFree(ctx->stage_dev);
  if (ctx->integ) cudaFree(ctx->integ);
  delete ctx;
  return KIOPS_OK;
}

const char* kiops_last_error(const kiops_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

kiops_status kiops_attach_workspace(kiops_ctx* ctx, void* dptr, size_t bytes) {
  if (!ctx) return KIOPS_EINVAL;
  if (ctx->ws_owned && ctx->ws) cudaFree(ctx->ws);
  ctx->ws = dptr;
  ctx->ws_bytes = dptr ? bytes : 0;
  ctx->ws_owned = false;
  return KIOPS_OK;
}

kiops_status kiops_workspace_size(kiops_ctx* ctx, const kiops_op* A, int p, int m_o, kiops_precision prec,
                                  size_t* bytes) {
  if (!ctx || !A || !bytes || p < 0 || p > KIOPS_MAX_P || m_o < 1) return KIOPS_EINVAL;
  const bool fp32 = prec == KIOPS_FP32_BASIS;
  void* fn = pick_kernel(fp32, A->d.kind);
  kiops_status st = prepare_kernel(ctx, fn);
  if (st) return st;
  int blocks = std::max(grid_size(ctx, fn), 1);
  int64_t ldv;
  Layout L = layout(A->d.n, p, ctx->cfg.m_max, std::min(m_o, ctx->cfg.m_max + 1), fp32, blocks, max_r(ctx->tt), 0, &ldv);
  *bytes = L.total;
  if (A->d.kind == OP_ST2D)  // the bulk-tensor-copy path's staged B columns (FP64) and coupling fields
    *bytes += align_up((size_t)p * ldv * 8, 256) +
              align_up((size_t)A->d.nspecies * A->d.nspecies * A->d.nx * A->d.ny * (fp32 ? 4 : 8), 256) + 512;
  return KIOPS_OK;
}

kiops_status kiops_op_csr(kiops_ctx* ctx, kiops_op** op, int64_t n, int64_t nnz, const int32_t* rowptr,
                          const int32_t* colind, const double* vals) {
  if (!ctx || !op) return KIOPS_EINVAL;
  *op = nullptr;
  if (n < 1 || nnz < 0 || n > INT32_MAX || !rowptr || (nnz > 0 && (!colind || !vals)))
    return fail(ctx, KIOPS_EINVAL, "invalid CSR description");
  kiops_op* o = new (std::nothrow) kiops_op();
  if (!o) return KIOPS_ENOMEM;
  o->ctx = ctx;
  std::memset(&o->d, 0, sizeof(o->d));
  o->d.kind = OP_CSR;
  o->d.n = n;
  o->d.rowptr = rowptr;
  o->d.colind = colind;
  o->d.vals = vals;
  o->nz = (double)nnz;
  *op = o;
  return KIOPS_OK;
}

kiops_status kiops_op_stencil2d(kiops_ctx* ctx, kiops_op** op, const kiops_stencil2d_desc* d) {
  if (!ctx || !op || !d) return KIOPS_EINVAL;
  *op = nullptr;
  if (d->nx < 1 || d->ny < 1 || (d->nspecies != 1 && d->nspecies != 2) || d->nx * d->ny * d->nspecies > INT32_MAX)
    return fail(ctx, KIOPS_EINVAL, "invalid 2D stencil description (sizes, species, or more than 2^31-1 unknowns)");
  if (d->bc < KIOPS_BC_DIRICHLET || d->bc > KIOPS_BC_NEUMANN || (d->bc == KIOPS_BC_NEUMANN && (d->nx < 2 || d->ny < 2)))
    return fail(ctx, KIOPS_EINVAL, "invalid boundary code %d (Neumann needs at least 2 points per dimension)", d->bc);
  kiops_op* o = new (std::nothrow) kiops_op();
  if (!o) return KIOPS_ENOMEM;
  o->ctx = ctx;
  std::memset(&o->d, 0, sizeof(o->d));
  o->d.kind = OP_ST2D;
  o->d.nx = d->nx;
  o->d.ny = d->ny;
  o->d.nz = 1;
  o->d.nspecies = d->nspecies;
  o->d.bc = d->bc;
  o->d.n = d->nx * d->ny * d->nspecies;
  for (int s = 0; s < 2; ++s) {
    for (int k = 0; k < 5; ++k) o->d.coef[s][k] = s < d->nspecies ? d->coef[s][k] : 0.0;
    for (int k = 0; k < 7; ++k) o->d.coef_f[s][k] = (float)o->d.coef[s][k];
    for (int r = 0; r < 2; ++r) o->d.diag[s][r] = (s < d->nspecies && r < d->nspecies) ? d->diag[s][r] : nullptr;
  }
  if (d->nfields != 0) {  // shared coupling fields: check, then write the block's entries once
    std::unique_ptr<kiops_op> guard(o);
    const int ns = d->nspecies, nf = d->nfields;
    if (nf < 0 || nf > 2) return fail(ctx, KIOPS_EINVAL, "nfields %d: shared coupling fields take 0, 1 or 2", nf);
    for (int f = 0; f < nf; ++f)
      if (!d->field[f]) return fail(ctx, KIOPS_EINVAL, "shared coupling field %d is NULL", f);
    int nent = 0;
    for (int s = 0; s < ns; ++s)
      for (int r = 0; r < ns; ++r) {
        if (d->diag[s][r]) return fail(ctx, KIOPS_EINVAL, "diag and shared coupling fields given together");
        if (d->dfield[s][r] < -1 || d->dfield[s][r] >= nf)
          return fail(ctx, KIOPS_EINVAL, "dfield[%d][%d] = %d outside -1..%d", s, r, d->dfield[s][r], nf - 1);
        if (d->dfield[s][r] >= 0 || d->dconst[s][r] != 0.0) ++nent;
      }
    const int64_t npts = d->nx * d->ny;
    if (nent > 0) {
      if (cudaMalloc(&o->owned, (size_t)nent * npts * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KIOPS_ENOMEM, "no device memory for the coupling block's entries (%d x %lld points)",
                    nent, (long long)npts);
      }
      struct Owned {  // frees the entries if a later step fails
        kiops_op* op;
        ~Owned() { if (op && op->owned) cudaFree(op->owned); }
      } owned_guard{o};
      int e = 0;
      const int blocks = (int)std::min<int64_t>((npts + 255) / 256, (int64_t)ctx->sms * 8);
      for (int s = 0; s < ns; ++s)
        for (int r = 0; r < ns; ++r) {
          const int k = d->dfield[s][r];
          if (k < 0 && d->dconst[s][r] == 0.0) continue;
          double* out = o->owned + (size_t)e++ * npts;
          coupling_entry_kernel<<<blocks, 256, 0, ctx->stream>>>(k >= 0 ? d->field[k] : nullptr, d->dweight[s][r],
                                                               d->dconst[s][r], out, npts);
          o->d.diag[s][r] = out;
        }
      KCHECK(ctx, cudaGetLastError());
      KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
      owned_guard.op = nullptr;
    }
    o->d.nfields = nf;
    for (int f = 0; f < 2; ++f) o->d.field[f] = f < nf ? d->field[f] : nullptr;
    for (int s = 0; s < 2; ++s)
      for (int r = 0; r < 2; ++r) {
        const bool in = s < ns && r < ns;
        o->d.dfield[s][r] = in ? d->dfield[s][r] : -1;
        o->d.dconst[s][r] = in ? d->dconst[s][r] : 0.0;
        o->d.dweight[s][r] = in ? d->dweight[s][r] : 0.0;
      }
    guard.release();
  }
  o->nz = 5.0 * (double)o->d.n;
  for (int s = 0; s < 2; ++s)
    for (int r = 0; r < 2; ++r)
      if (o->d.diag[s][r]) o->nz += (double)(d->nx * d->ny);
  *op = o;
  return KIOPS_OK;
}

kiops_status kiops_op_stencil3d(kiops_ctx* ctx, kiops_op** op, const kiops_stencil3d_desc* d) {
  if (!ctx || !op || !d) return KIOPS_EINVAL;
  *op = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx * d->ny * d->nz > INT32_MAX)
    return fail(ctx, KIOPS_EINVAL, "invalid 3D stencil description (sizes or more than 2^31-1 unknowns)");
  if (d->bc < KIOPS_BC_DIRICHLET || d->bc > KIOPS_BC_NEUMANN ||
      (d->bc == KIOPS_BC_NEUMANN && (d->nx < 2 || d->ny < 2 || d->nz < 2)))
    return fail(ctx, KIOPS_EINVAL, "invalid boundary code %d (Neumann needs at least 2 points per dimension)", d->bc);
  kiops_op* o = new (std::nothrow) kiops_op();
  if (!o) return KIOPS_ENOMEM;
  o->ctx = ctx;
  std::memset(&o->d, 0, sizeof(o->d));
  o->d.kind = OP_ST3D;
  o->d.nx = d->nx;
  o->d.ny = d->ny;
  o->d.nz = d->nz;
  o->d.nspecies = 1;
  o->d.bc = d->bc;
  o->d.n = d->nx * d->ny * d->nz;
  for (int k = 0; k < 7; ++k) o->d.coef[0][k] = d->coef[k];
  for (int k = 0; k < 7; ++k) o->d.coef_f[0][k] = (float)d->coef[k];
  o->d.diag[0][0] = d->diag;
  o->nz = (double)o->d.n * (d->diag ? 8.0 : 7.0);
  *op = o;
  return KIOPS_OK;
}

kiops_status kiops_op_destroy(kiops_op* op) {
  if (!op) return KIOPS_EINVAL;
  if (op->owned) cudaFree(op->owned);
  delete op;
  return KIOPS_OK;
}

int64_t kiops_op_size(const kiops_op* op) { return op ? op->d.n : -1; }

kiops_status kiops_op_apply(kiops_ctx* ctx, const kiops_op* A, const double* x, double* y) {
  if (!ctx || !A || !x || !y) return KIOPS_EINVAL;
  const int blocks = (int)std::min<int64_t>((A->d.n + 255) / 256, (int64_t)ctx->sms * 8);
  if (A->d.kind == OP_CSR) op_apply_kernel<OP_CSR><<<blocks, 256, 0, ctx->stream>>>(A->d, x, y);
  else if (A->d.kind == OP_ST2D) op_apply_kernel<OP_ST2D><<<blocks, 256, 0, ctx->stream>>>(A->d, x, y);
  else op_apply_kernel<OP_ST3D><<<blocks, 256, 0, ctx->stream>>>(A->d, x, y);
  KCHECK(ctx, cudaGetLastError());
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  return KIOPS_OK;
}

kiops_status kiops_solve(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b, double tol,
                         int m_init, int m_o, kiops_precision prec, double* w, kiops_stats* stats) {
  return run_single(ctx, A, tau, p, b, tol, m_init, m_o, prec, w, stats, nullptr, 0, nullptr);
}

kiops_status kiops_solve_traced(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b,
                                double tol, int m_init, int m_o, kiops_precision prec, double* w,
                                kiops_stats* stats, kiops_trace_rec* trace, int64_t trace_cap,
                                int64_t* trace_len) {
  if (!trace || trace_cap < 1) return fail(ctx, KIOPS_EINVAL, "trace buffer required");
  return run_single(ctx, A, tau, p, b, tol, m_init, m_o, prec, w, stats, trace, trace_cap, trace_len);
}

kiops_status kiops_solve_task1(kiops_ctx* ctx, const kiops_op* A, const double* T, int n_times, int p,
                               const double* const* b, double tol, int m_init, int m_o, kiops_precision prec,
                               double* const* w, kiops_stats* stats) {
  if (!ctx) return KIOPS_EINVAL;
  if (!T || !w || n_times < 1 || n_times > KIOPS_MAX_TIMES)
    return fail(ctx, KIOPS_EINVAL, "Task I needs 1..%d output times and as many outputs", KIOPS_MAX_TIMES);
  for (int l = 0; l < n_times; ++l) {
    if (!w[l]) return fail(ctx, KIOPS_EINVAL, "w[%d] is NULL", l);
    if (!(T[l] > 0.0) || !std::isfinite(T[l]) || (l > 0 && !(T[l] > T[l - 1])))
      return fail(ctx, KIOPS_EINVAL, "output times must be positive and increasing");
  }
  return run_single(ctx, A, T[n_times - 1], p, b, tol, m_init, m_o, prec, w[n_times - 1], stats, nullptr, 0, nullptr,
                    T, n_times, w);
}

kiops_status kiops_solve_host(kiops_ctx* ctx, const kiops_op* A, double tau, int p, const double* const* b_host,
                              double tol, int m_init, int m_o, kiops_precision prec, double* w_host,
                              kiops_stats* stats) {
  if (!ctx || !A || !b_host || !w_host || p < 0 || p > KIOPS_MAX_P) return KIOPS_EINVAL;
  for (int k = 0; k <= p; ++k)
    if (!b_host[k]) return fail(ctx, KIOPS_EINVAL, "b_host[%d] is NULL", k);
  const size_t n = (size_t)A->d.n;
  const size_t need = (size_t)(p + 2) * n * sizeof(double);
  if (need > ctx->stage_bytes) {
    if (ctx->stage_dev) cudaFree(ctx->stage_dev);
    ctx->stage_dev = nullptr;
    ctx->stage_bytes = 0;
    KCHECK(ctx, cudaMalloc(&ctx->stage_dev, need));
    ctx->stage_bytes = need;
  }
  const double* bd[KIOPS_MAX_P + 1];
  for (int k = 0; k <= p; ++k) {
    double* dst = ctx->stage_dev + (size_t)k * n;
    KCHECK(ctx, cudaMemcpyAsync(dst, b_host[k], n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    bd[k] = dst;
  }
  double* wd = ctx->stage_dev + (size_t)(p + 1) * n;
  kiops_status st = run_single(ctx, A, tau, p, bd, tol, m_init, m_o, prec, wd, stats, nullptr, 0, nullptr);
  if (st != KIOPS_OK) return st;
  KCHECK(ctx, cudaMemcpyAsync(w_host, wd, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  return KIOPS_OK;
}

// Work estimate of one request for the batch plan: N times a step count from a Gershgorin bound of
// ||tau A|| (Krylov dimensions grow like its square root; beyond m_max the solve substeps).
static double estimate_work(const kiops_ctx* ctx, const kiops_request& r) {
  const OpDesc& d = r.A->d;
  double nrm = 0.0;
  if (d.kind == OP_ST2D || d.kind == OP_ST3D) {
    const int nc = d.kind == OP_ST3D ? 7 : 5;
    for (int sp = 0; sp < (d.kind == OP_ST3D ? 1 : d.nspecies); ++sp) {
      double rs = 0.0;
      for (int k = 0; k < nc; ++k) rs += std::fabs(d.coef[sp][k]);
      nrm = std::max(nrm, rs);
    }
  }
  const double nu = r.tau * nrm;
  double steps = d.kind == OP_CSR ? 30.0 : std::min((double)ctx->cfg.m_max, 10.0 + 2.0 * std::sqrt(nu));
  steps *= std::max(1.0, nu / 400.0);
  return (double)d.n * steps * (r.prec == KIOPS_FP32_BASIS ? 0.5 : 1.0);
}

// Team engine: requests grouped by (precision, operator kind); per group one cooperative launch of
// floor(G / K) teams of K blocks; requests sorted by estimated work and each given to the least-loaded
// team.  K = cfg.batch_team_blocks, or 0 = automatic (the heaviest request's share of the total work,
// rounded down to a power of two).
static kiops_status batch_teams(kiops_ctx* ctx, int count, const kiops_request* reqs, kiops_stats* stats) {
  NvtxRange nvtx_range("kiops batch");
  std::vector<int> order;
  for (int i = 0; i < count; ++i)
    if (reqs[i].tau > 0.0) order.push_back(i);
  for (int i = 0; i < count; ++i)
    if (reqs[i].tau == 0.0) {
      KCHECK(ctx, cudaMemcpyAsync(reqs[i].w, reqs[i].b[0], (size_t)reqs[i].A->d.n * 8, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
      if (stats) {
        std::memset(&stats[i], 0, sizeof(kiops_stats));
        stats[i].engine = KIOPS_ENGINE_CTA;
      }
    }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return reqs[x].prec * 4 + reqs[x].A->d.kind < reqs[y].prec * 4 + reqs[y].A->d.kind;
  });
  kiops_status worst = KIOPS_OK;
  size_t g0 = 0;
  while (g0 < order.size()) {
    size_t g1 = g0;
    const int key = reqs[order[g0]].prec * 4 + reqs[order[g0]].A->d.kind;
    while (g1 < order.size() && reqs[order[g1]].prec * 4 + reqs[order[g1]].A->d.kind == key) ++g1;
    const bool fp32 = reqs[order[g0]].prec == KIOPS_FP32_BASIS;
    void* fn = pick_team_kernel(fp32, reqs[order[g0]].A->d.kind);
    kiops_status st = prepare_kernel(ctx, fn);
    if (st) return st;
    const int G = grid_size(ctx, fn);
    if (G < 1) return fail(ctx, KIOPS_ECUDA, "team kernel does not fit on the device");
    const int n = (int)(g1 - g0);
    std::vector<double> work((size_t)n);
    double total = 0.0, heaviest = 0.0;
    for (int k = 0; k < n; ++k) {
      work[k] = estimate_work(ctx, reqs[order[g0 + k]]);
      total += work[k];
      heaviest = std::max(heaviest, work[k]);
    }
    int K = ctx->cfg.batch_team_blocks;
    if (K <= 0) {
      K = 1;
      while (2 * K <= G && (double)(2 * K) <= (double)G * heaviest / std::max(total, 1e-300)) K *= 2;
    }
    K = std::max(1, std::min(K, G));
    const int T = std::max(1, G / K);
    // LPT plan
    std::vector<int> byw((size_t)n);
    for (int k = 0; k < n; ++k) byw[k] = k;
    std::stable_sort(byw.begin(), byw.end(), [&](int x, int y) { return work[x] > work[y]; });
    std::vector<double> load((size_t)T, 0.0);
    std::vector<std::vector<int>> lists((size_t)T);
    for (int k : byw) {
      int best = 0;
      for (int t = 1; t < T; ++t)
        if (load[t] < load[best]) best = t;
      load[best] += work[k];
      lists[best].push_back(k);
    }
    // per-request argument blocks, per-team workspace sized for the team's own requests
    std::vector<Prepared> prep((size_t)n);
    std::vector<size_t> team_bytes((size_t)T, 0);
    for (int t = 0; t < T; ++t)
      for (int k : lists[t]) {
        const kiops_request& r = reqs[order[g0 + k]];
        st = prepare(ctx, r.A, r.tau, r.p, r.b, r.tol, r.m_init, r.m_o, r.prec, r.w, K, 0, prep[k]);
        if (st) return st;
        team_bytes[t] = std::max(team_bytes[t], prep[k].L.total);
      }
    size_t off = 0;
    std::vector<size_t> team_off((size_t)T);
    for (int t = 0; t < T; ++t) {
      team_off[t] = off;
      off = align_up(off + team_bytes[t], 256);
    }
    const size_t stats_off = off;
    off = align_up(off + (size_t)n * 16 * 8, 256);
    const size_t ctr_off = off;
    off = align_up(off + (size_t)T * 64 * 4 + 256, 256);
    const size_t args_off = off;
    off = align_up(off + (size_t)n * sizeof(SolveArgs), 256);
    const size_t plan_off = off;
    off = align_up(off + (size_t)(T + 1 + n) * 4, 256);
    st = ensure_workspace(ctx, off);
    if (st) return st;
    char* base = (char*)ctx->ws;
    std::vector<int> plan_ptr((size_t)T + 1, 0), plan_idx;
    for (int t = 0; t < T; ++t) {
      for (int k : lists[t]) {
        bind(prep[k], base + team_off[t]);
        prep[k].args.stats = (int64_t*)(base + stats_off + (size_t)k * 16 * 8);
        prep[k].args.stats_d = (double*)(prep[k].args.stats + 10);
        prep[k].args.abort_flag = (int*)(base + ctr_off + (size_t)T * 64 * 4);
        prep[k].args.timeout_ns = (long long)(ctx->cfg.timeout_s * 1e9);
        plan_idx.push_back(k);
      }
      plan_ptr[t + 1] = (int)plan_idx.size();
    }
    const size_t hbytes = (size_t)n * sizeof(SolveArgs) + (size_t)(T + 1 + n) * 4 + (size_t)n * 16 * 8 + 512;
    st = ensure_pinned(ctx, hbytes);
    if (st) return st;
    char* hp = (char*)ctx->host_pinned;
    for (int k = 0; k < n; ++k) std::memcpy(hp + (size_t)k * sizeof(SolveArgs), &prep[k].args, sizeof(SolveArgs));
    int* hplan = (int*)(hp + (size_t)n * sizeof(SolveArgs));
    std::memcpy(hplan, plan_ptr.data(), (size_t)(T + 1) * 4);
    std::memcpy(hplan + T + 1, plan_idx.data(), (size_t)n * 4);
    int64_t* hstats = (int64_t*)(hp + align_up((size_t)n * sizeof(SolveArgs) + (size_t)(T + 1 + n) * 4, 256));
    KCHECK(ctx, cudaMemsetAsync(base + ctr_off, 0, (size_t)T * 64 * 4 + 256, ctx->stream));
    KCHECK(ctx, cudaMemsetAsync(base + stats_off, 0, (size_t)n * 16 * 8, ctx->stream));
    KCHECK(ctx, cudaMemcpyAsync(base + args_off, hp, (size_t)n * sizeof(SolveArgs), cudaMemcpyHostToDevice, ctx->stream));
    KCHECK(ctx, cudaMemcpyAsync(base + plan_off, hplan, (size_t)(T + 1 + n) * 4, cudaMemcpyHostToDevice, ctx->stream));
    const SolveArgs* dargs = (const SolveArgs*)(base + args_off);
    const int* dptr = (const int*)(base + plan_off);
    const int* didx = dptr + T + 1;
    unsigned int* dctr = (unsigned int*)(base + ctr_off);
    int* dabort = (int*)(base + ctr_off + (size_t)T * 64 * 4);
    long long tns = (long long)(ctx->cfg.timeout_s * 1e9);
    int Kv = K, Tv = T;
    void* kargs[] = {(void*)&dargs, (void*)&dptr, (void*)&didx, (void*)&Kv, (void*)&Tv, (void*)&dctr, (void*)&dabort,
                     (void*)&tns};
    KCHECK(ctx, cudaLaunchCooperativeKernel(fn, T * K, kThreads, kargs, kDynSmem, ctx->stream));
    KCHECK(ctx, cudaMemcpyAsync(hstats, base + stats_off, (size_t)n * 16 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < n; ++k) {
      const int i = order[g0 + k];
      const int64_t* sv = hstats + (size_t)k * 16;
      fill_stats(stats ? &stats[i] : nullptr, sv, (const double*)(sv + 10), KIOPS_ENGINE_CTA, K);
      if (sv[6] != ST_OK && worst == KIOPS_OK) worst = (kiops_status)sv[6];
    }
    g0 = g1;
  }
  if (worst != KIOPS_OK) return fail(ctx, worst, "at least one batch request failed (status %d)", (int)worst);
  return KIOPS_OK;
}

kiops_status kiops_solve_batch(kiops_ctx* ctx, int count, const kiops_request* reqs, kiops_stats* stats) {
  if (!ctx || count < 0 || (count > 0 && !reqs)) return KIOPS_EINVAL;
  if (count == 0) return KIOPS_OK;
  for (int i = 0; i < count; ++i)
    if (!reqs[i].A || !reqs[i].b || !reqs[i].w) return fail(ctx, KIOPS_EINVAL, "request %d: NULL operator, b or w", i);
  return batch_teams(ctx, count, reqs, stats);
}

kiops_status kiops_set_batch_team_blocks(kiops_ctx* ctx, int team_blocks) {
  if (!ctx || team_blocks < 0) return KIOPS_EINVAL;
  ctx->cfg.batch_team_blocks = team_blocks;
  return KIOPS_OK;
}

kiops_status kiops_get_config(const kiops_ctx* ctx, kiops_config* cfg) {
  if (!ctx || !cfg) return KIOPS_EINVAL;
  *cfg = ctx->cfg;
  return KIOPS_OK;
}

kiops_status kiops_set_config(kiops_ctx* ctx, const kiops_config* cfg) {
  if (!ctx || !cfg) return KIOPS_EINVAL;
  if (ctx->server) return fail(ctx, KIOPS_EBUSY, "the configuration of a serving context is fixed");
  const kiops_config& c = *cfg;
  if (c.device != ctx->cfg.device || c.stream != ctx->cfg.stream)
    return fail(ctx, KIOPS_EINVAL, "the device and the stream of a context cannot change");
  if (c.m_min < 1 || c.m_max < c.m_min || c.m_max > KIOPS_MAX_M || !(c.breakdown_tol >= 0) || c.max_substeps < 1 ||
      c.max_iterations < 1 || !(c.timeout_s > 0) || c.tile_w < 0 || c.tile_h < 0 || c.tma < 0 || c.tma > 2)
    return fail(ctx, KIOPS_EINVAL, "invalid configuration");
  ctx->cfg = c;
  return KIOPS_OK;
}

kiops_status kiops_expm(kiops_ctx* ctx, int n, const double* a, double* f) {
  NvtxRange nvtx_range("kiops expm");
  if (!ctx || !a || !f || n < 1 || n > KIOPS_MAX_M + 1) return KIOPS_EINVAL;
  void* fn = pick_kernel(false, OP_CSR);
  kiops_status st = prepare_kernel(ctx, fn);
  if (st) return st;
  int blocks = grid_size(ctx, fn);
  if (blocks < 1) return fail(ctx, KIOPS_ECUDA, "kernel does not fit on the device");
  Prepared P;
  std::memset(&P.args, 0, sizeof(SolveArgs));
  SolveArgs& sa = P.args;
  sa.m_max = n - 1;
  sa.tt = ctx->tt;
  sa.expm_only = 1;
  sa.expm_n = n;
  sa.expm_in = a;
  sa.expm_out = f;
  sa.timeout_ns = (long long)(ctx->cfg.timeout_s * 1e9);
  int64_t ldv;
  P.L = layout(0, 0, n - 1, 1, false, blocks, max_r(ctx->tt), 0, &ldv);
  st = ensure_workspace(ctx, P.L.total);
  if (st) return st;
  bind(P, (char*)ctx->ws);
  st = ensure_pinned(ctx, sizeof(SolveArgs) + 256);
  if (st) return st;
  std::memcpy(ctx->host_pinned, &P.args, sizeof(SolveArgs));
  KCHECK(ctx, cudaMemsetAsync(P.base + P.L.bar, 0, 256 + 16 * 8 + 256, ctx->stream));
  KCHECK(ctx, cudaMemcpyAsync(P.base + P.L.args, ctx->host_pinned, sizeof(SolveArgs), cudaMemcpyHostToDevice, ctx->stream));
  const SolveArgs* dargs = (const SolveArgs*)(P.base + P.L.args);
  void* kargs[] = {(void*)&dargs, (void*)&P.maps};
  KCHECK(ctx, cudaLaunchCooperativeKernel(fn, blocks, kThreads, kargs, kDynSmem, ctx->stream));
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  int flag = 0;
  KCHECK(ctx, cudaMemcpy(&flag, P.base + P.L.bar + 64, 4, cudaMemcpyDeviceToHost));
  if (flag) return fail(ctx, KIOPS_ETIMEOUT, "a device-side wait exceeded the limit");
  return KIOPS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Allocation-free solve: the workspace is a file-scope device array.  In host code the array's name
// is only a host-side stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernel.
// ------------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[KIOPS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

}  // namespace

extern "C" kiops_status kiops_solve_noalloc(kiops_ctx* ctx, const kiops_op* A, double tau, int p,
                                            const double* const* b, double tol, int m_init, int m_o, double* w,
                                            kiops_stats* stats) {
  NvtxRange nvtx_range("kiops solve (no allocation)");
  if (!ctx) return KIOPS_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const int dev = ctx->cfg.device;
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(ctx, KIOPS_EINVAL, "device ordinal %d not supported", dev);
  KCHECK(ctx, cudaSetDevice(dev));
  if (!g_noalloc_addr[dev]) {  // set-up, once per device (make the first call before any stream capture)
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(ctx, KIOPS_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_addr[dev] = ptr;
  }
  if (tau == 0.0 && A && b && w && b[0]) {
    if (w != b[0]) KCHECK(ctx, cudaMemcpyAsync(w, b[0], (size_t)A->d.n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
    if (stats) stats->m_last = std::max(ctx->cfg.m_min, std::min(m_init, ctx->cfg.m_max));
    return KIOPS_OK;
  }
  Prepared P;
  kiops_status st = prepare(ctx, A, tau, p, b, tol, m_init, m_o, KIOPS_FP64, w, 1, 0, P);
  if (st) return st;
  if (P.L.total > (size_t)KIOPS_NOALLOC_SCRATCH_BYTES)
    return fail(ctx, KIOPS_EINVAL,
                "kiops_solve_noalloc: this solve needs %zu bytes of workspace but the fixed scratch holds %u "
                "(N + p = %lld, m_max = %d); use kiops_solve or a smaller m_max",
                P.L.total, (unsigned)KIOPS_NOALLOC_SCRATCH_BYTES, (long long)(A->d.n + p), ctx->cfg.m_max);
  bind(P, (char*)g_noalloc_addr[dev]);
  // the array keeps the previous call's contents: clear the barrier word, abort flag, stats, trace count
  KCHECK(ctx, cudaMemsetAsync(P.base + P.L.bar, 0, 256 + 16 * 8 + 256, ctx->stream));
  void* fn = kiops_k::noalloc_kernel(A->d.kind);
  KCHECK(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem));
  void* kargs[] = {(void*)&P.args};
  KCHECK(ctx, cudaLaunchKernel(fn, 1, kThreads, kargs, kDynSmem, ctx->stream));
  int64_t hs[16];
  KCHECK(ctx, cudaMemcpyAsync(hs, P.base + P.L.stats, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  fill_stats(stats, hs, (const double*)(hs + 10), KIOPS_ENGINE_CTA, 1);
  const int dst = (int)hs[6];
  if (dst == ST_ENOTCONV)
    return fail(ctx, KIOPS_ENOTCONV, "no convergence within max_substeps/max_iterations (%lld iterations)",
                (long long)hs[3]);
  if (dst != ST_OK) return fail(ctx, (kiops_status)dst, "device status %d", dst);
  return KIOPS_OK;
}

// ------------------------------------------------------------------------------------------------
// Serving (continuous batching): one persistent server kernel per context, request queues in mapped
// host memory, per-request workspace from an arena of the HBM budget (first-fit free list).
// ------------------------------------------------------------------------------------------------
namespace {

struct Arena {
  size_t bytes = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  void init(size_t n) {
    bytes = n;
    free_.clear();
    if (n) free_[0] = n;
  }
  bool alloc(size_t n, size_t& off) {
    n = align_up(n, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= n) {
        off = it->first;
        const size_t rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t n) {
    n = align_up(n, 256);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct MappedQueues {  // lives in mapped pinned host memory
  unsigned int tail[kServerClasses][16];
  int stop[16];
};

struct InFlight {
  int cls = 0, slot = -1;
  unsigned int index = 0;  // queue index of the request in its class (claimed once head has passed it)
  size_t off = 0, bytes = 0;
  int64_t* stats_dev = nullptr;
};

struct Pending {
  uint64_t ticket;
  int cls;
  Prepared P;
};

struct SoloReq {  // a request that runs alone on the whole GPU (server_config.solo_min_unknowns)
  uint64_t ticket;
  kiops_request r;
  std::vector<const double*> b;  // copy of the caller's b[0..p]
};

}  // namespace

struct KiopsServer {
  kiops_server_config cfg{};
  cudaStream_t kstream = nullptr, cstream = nullptr;
  cudaEvent_t kdone = nullptr;
  bool launched = false;
  bool exit_checked = false;  // the exited launch's abort word has been read
  // mapped host memory
  MappedQueues* q = nullptr;
  SolveArgs* slots_h[kServerClasses] = {};
  unsigned long long* done_h[kServerClasses] = {};
  void* mapped_base = nullptr;
  // device memory
  void* dev_base = nullptr;
  ServerDev sd{};
  char* arena_base = nullptr;
  Arena arena;
  std::vector<char> slot_busy[kServerClasses];
  unsigned int next_index[kServerClasses] = {};
  uint64_t next_ticket = 1;
  std::deque<Pending> pending;
  std::deque<SoloReq> solo;  // waiting to run alone; while any waits, nothing is admitted and the kernel drains
  std::unordered_map<uint64_t, InFlight> inflight;
  std::unordered_map<uint64_t, std::vector<int64_t>> finished;  // ticket -> 16 stats words
  int grid = 0;
};

namespace {

kiops_status server_launch(kiops_ctx* ctx, KiopsServer* S) {
  void* fn = kiops_k::server_kernel();
  KCHECK(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem));
  // a new launch starts every team's barrier epochs at zero: clear the team counters, the claim words and
  // the abort word that follows them (raised by a wait of the previous launch that gave up)
  const int n_teams = S->sd.teams[0] + S->sd.teams[1];
  KCHECK(ctx, cudaMemsetAsync(S->sd.team_ctr, 0, (size_t)n_teams * 64 * 4 * 2 + 256, S->kstream));
  void* kargs[] = {(void*)&S->sd};
  KCHECK(ctx, cudaLaunchCooperativeKernel(fn, S->grid, kThreads, kargs, kDynSmem, S->kstream));
  KCHECK(ctx, cudaEventRecord(S->kdone, S->kstream));
  S->launched = true;
  S->exit_checked = false;
  return KIOPS_OK;
}

// Once per exited launch: if a device-side wait gave up (abort word raised), the teams left without
// finishing the requests they had claimed.  Those tickets finish here with the abort status and give back
// their slot and workspace; requests still queued (not claimed) run on the next launch.
kiops_status server_check_exit(kiops_ctx* ctx, KiopsServer* S) {
  if (!S->launched || S->exit_checked) return KIOPS_OK;
  const cudaError_t e = cudaEventQuery(S->kdone);
  if (e == cudaErrorNotReady) return KIOPS_OK;
  if (e != cudaSuccess) return fail(ctx, KIOPS_ECUDA, "server kernel: %s", cudaGetErrorString(e));
  S->exit_checked = true;
  int ab = 0;
  unsigned int heads[kServerClasses] = {};
  KCHECK(ctx, cudaMemcpyAsync(&ab, S->sd.abort_flag, sizeof(int), cudaMemcpyDeviceToHost, S->cstream));
  for (int c = 0; c < kServerClasses; ++c)
    KCHECK(ctx, cudaMemcpyAsync(heads + c, S->sd.head[c], sizeof(unsigned int), cudaMemcpyDeviceToHost, S->cstream));
  KCHECK(ctx, cudaStreamSynchronize(S->cstream));
  if (ab == 0) return KIOPS_OK;
  std::vector<uint64_t> lost;
  for (auto& kv : S->inflight) {
    const InFlight& f = kv.second;
    const bool claimed = (int)(heads[f.cls] - f.index) > 0;
    const bool done = *(volatile unsigned long long*)(S->done_h[f.cls] + f.slot) == kv.first;
    if (claimed && !done) lost.push_back(kv.first);
  }
  for (uint64_t t : lost) {
    const InFlight f = S->inflight[t];
    std::vector<int64_t> st(16, 0);
    st[6] = ab;
    S->finished[t] = st;
    S->arena.release(f.off, f.bytes);
    S->slot_busy[f.cls][f.slot] = 0;
    S->inflight.erase(t);
  }
  return KIOPS_OK;
}

bool server_kernel_running(KiopsServer* S) { return S->launched && cudaEventQuery(S->kdone) == cudaErrorNotReady; }

// Admit pending requests (budget and slot permitting), collect completions, relaunch an exited kernel.
// Finished requests (completion word = ticket): stats back, slot and workspace free.
kiops_status server_collect(kiops_ctx* ctx, KiopsServer* S) {
  std::vector<uint64_t> done_now;
  for (auto& kv : S->inflight) {
    const InFlight& f = kv.second;
    const unsigned long long v = *(volatile unsigned long long*)(S->done_h[f.cls] + f.slot);
    if (v == kv.first) done_now.push_back(kv.first);
  }
  for (uint64_t t : done_now) {
    InFlight f = S->inflight[t];
    std::vector<int64_t> st(16);
    KCHECK(ctx, cudaMemcpyAsync(st.data(), f.stats_dev, 16 * 8, cudaMemcpyDeviceToHost, S->cstream));
    KCHECK(ctx, cudaStreamSynchronize(S->cstream));
    S->finished[t] = st;
    S->arena.release(f.off, f.bytes);
    S->slot_busy[f.cls][f.slot] = 0;
    S->inflight.erase(t);
  }
  return KIOPS_OK;
}

// Requests that run alone: with the server kernel gone (it drains its queues and exits once the stop word is
// up) and nothing in flight, run the oldest on the whole GPU with the grid engine, synchronously.
kiops_status server_run_solo(kiops_ctx* ctx, KiopsServer* S) {
  __atomic_store_n(&S->q->stop[0], 1, __ATOMIC_RELEASE);  // the kernel exits when its queues are empty
  while (!S->solo.empty() && S->inflight.empty() && !server_kernel_running(S)) {
    kiops_status xs = server_check_exit(ctx, S);
    if (xs) return xs;
    SoloReq q = S->solo.front();
    S->solo.pop_front();
    kiops_stats st{};
    const kiops_status rc = run_single(ctx, q.r.A, q.r.tau, q.r.p, q.b.data(), q.r.tol, q.r.m_init, q.r.m_o,
                                       q.r.prec, q.r.w, &st, nullptr, 0, nullptr);
    std::vector<int64_t> w(16, 0);
    w[0] = st.substeps; w[1] = st.rejected; w[2] = st.matvecs; w[3] = st.iterations; w[4] = st.expm_calls;
    w[5] = st.m_last; w[6] = rc;
    std::memcpy(&w[10], &st.err_est, sizeof(double));
    S->finished[q.ticket] = w;
  }
  if (S->solo.empty()) __atomic_store_n(&S->q->stop[0], 0, __ATOMIC_RELEASE);
  return KIOPS_OK;
}

kiops_status server_pump(kiops_ctx* ctx, KiopsServer* S, bool allow_solo = false) {
  kiops_status xs = server_check_exit(ctx, S);
  if (!xs) xs = server_collect(ctx, S);
  if (xs) return xs;
  if (!S->solo.empty()) {  // drain, then run alone (only from kiops_poll: it blocks for the solve)
    if (!allow_solo) {
      __atomic_store_n(&S->q->stop[0], 1, __ATOMIC_RELEASE);
      return KIOPS_OK;
    }
    xs = server_run_solo(ctx, S);
    if (xs) return xs;
    if (!S->solo.empty()) return KIOPS_OK;  // still draining
  }
  // admissions, in arrival order per class (a request that does not fit waits; later ones may pass it)
  bool enqueued = false;
  for (auto it = S->pending.begin(); it != S->pending.end();) {
    Pending& pd = *it;
    const int c = pd.cls;
    const int slot = (int)(S->next_index[c] % (unsigned)S->cfg.queue_slots);
    size_t off = 0;
    if (S->slot_busy[c][slot] || !S->arena.alloc(pd.P.L.total, off)) {
      ++it;
      continue;
    }
    bind(pd.P, S->arena_base + off);
    pd.P.args.ticket = pd.ticket;
    pd.P.args.timeout_ns = (long long)(ctx->cfg.timeout_s * 1e9);
    // No device work here: a memset is a kernel, and it could not start while the server kernel holds every
    // SM, so admission would wait for the kernel to go idle.  Nothing of the workspace needs clearing: the
    // teams use their own barrier words and the abort word of the server, and the solve writes every stats
    // word the host reads.
    S->done_h[c][slot] = 0;
    std::memcpy((void*)(S->slots_h[c] + slot), &pd.P.args, sizeof(SolveArgs));
    InFlight f;
    f.cls = c;
    f.slot = slot;
    f.index = S->next_index[c];
    f.off = off;
    f.bytes = pd.P.L.total;
    f.stats_dev = pd.P.args.stats;
    S->inflight[pd.ticket] = f;
    S->slot_busy[c][slot] = 1;
    __atomic_thread_fence(__ATOMIC_SEQ_CST);  // the slot is written before the tail moves
    S->next_index[c] += 1;
    __atomic_store_n(&S->q->tail[c][0], S->next_index[c], __ATOMIC_RELEASE);
    enqueued = true;
    it = S->pending.erase(it);
  }
  if ((enqueued || !S->inflight.empty()) && !server_kernel_running(S)) {
    // the kernel may have exited after the check at the top: collect what an abort left before the
    // relaunch clears the abort word
    kiops_status xs2 = server_check_exit(ctx, S);
    if (!xs2) xs2 = server_collect(ctx, S);
    if (xs2) return xs2;
    if (S->inflight.empty()) return KIOPS_OK;
    kiops_status st = server_launch(ctx, S);
    if (st) return st;
  }
  return KIOPS_OK;
}

}  // namespace

extern "C" {

kiops_status kiops_server_config_default(kiops_server_config* cfg) {
  if (!cfg) return KIOPS_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->hbm_budget_bytes = 120e9;
  cfg->queue_slots = 512;
  cfg->small_team_blocks = 8;
  cfg->large_team_blocks = 0;
  cfg->large_teams = 2;  // measured on the 3D request mix with n <= 64: 415 (one team) -> 555 solves/s
  cfg->large_work_threshold = 2e8;
  cfg->idle_timeout_s = 2.0;
  cfg->solo_min_unknowns = 1e6;
  return KIOPS_OK;
}

kiops_status kiops_server_start(kiops_ctx* ctx, const kiops_server_config* cfg_in) {
  if (!ctx) return KIOPS_EINVAL;
  if (ctx->server) return fail(ctx, KIOPS_EBUSY, "a server is already running on this context");
  kiops_server_config cfg;
  if (cfg_in) cfg = *cfg_in; else kiops_server_config_default(&cfg);
  if (!(cfg.hbm_budget_bytes > 0) || cfg.queue_slots < 1 || cfg.small_team_blocks < 1 || cfg.large_teams < 0 ||
      !(cfg.idle_timeout_s > 0) || cfg.idle_timeout_s >= ctx->cfg.timeout_s)
    return fail(ctx, KIOPS_EINVAL, "invalid server configuration (the idle timeout must be below cfg.timeout_s)");
  void* fn = kiops_k::server_kernel();
  kiops_status st = prepare_kernel(ctx, fn);
  if (st) return st;
  int per_sm = 0;
  KCHECK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, kDynSmem));
  const int G = per_sm * ctx->sms;
  if (G < 2) return fail(ctx, KIOPS_ECUDA, "server kernel does not fit");
  std::unique_ptr<KiopsServer> S(new KiopsServer());
  int large_K = cfg.large_team_blocks > 0 ? cfg.large_team_blocks : G / (2 * std::max(cfg.large_teams, 1));
  int large_T = cfg.large_teams;
  if (large_T * large_K >= G) large_T = 0;
  const int small_K = std::min(cfg.small_team_blocks, G);
  const int small_T = (G - large_T * large_K) / small_K;
  if (small_T < 1) return fail(ctx, KIOPS_EINVAL, "team sizes leave no small team");
  cfg.large_team_blocks = large_K;
  cfg.large_teams = large_T;
  S->cfg = cfg;
  ServerDev& sd = S->sd;
  sd.n_classes = kServerClasses;
  sd.team_blocks[0] = small_K;
  sd.teams[0] = small_T;
  sd.first_block[0] = 0;
  sd.team_blocks[1] = std::max(large_K, 1);
  sd.teams[1] = large_T;
  sd.first_block[1] = small_T * small_K;
  S->grid = small_T * small_K + large_T * large_K;
  sd.slots_per_class = cfg.queue_slots;
  const int n_teams = small_T + large_T;
  // mapped host memory: queue words, request slots, completion words
  const size_t slots_bytes = (size_t)kServerClasses * cfg.queue_slots * sizeof(SolveArgs);
  const size_t done_bytes = (size_t)kServerClasses * cfg.queue_slots * 8;
  const size_t mapped = align_up(sizeof(MappedQueues), 256) + align_up(slots_bytes, 256) + done_bytes;
  KCHECK(ctx, cudaHostAlloc(&S->mapped_base, mapped, cudaHostAllocMapped | cudaHostAllocPortable));
  std::memset(S->mapped_base, 0, mapped);
  char* hb = (char*)S->mapped_base;
  S->q = (MappedQueues*)hb;
  char* dp = nullptr;
  KCHECK(ctx, cudaHostGetDevicePointer((void**)&dp, S->mapped_base, 0));
  const size_t o_slots = align_up(sizeof(MappedQueues), 256), o_done = o_slots + align_up(slots_bytes, 256);
  for (int c = 0; c < kServerClasses; ++c) {
    S->slots_h[c] = (SolveArgs*)(hb + o_slots) + (size_t)c * cfg.queue_slots;
    S->done_h[c] = (unsigned long long*)(hb + o_done) + (size_t)c * cfg.queue_slots;
    sd.tail[c] = (const unsigned int*)(dp + offsetof(MappedQueues, tail) + (size_t)c * 16 * 4);
    sd.slots[c] = (const SolveArgs*)(dp + o_slots) + (size_t)c * cfg.queue_slots;
    sd.done[c] = (unsigned long long*)(dp + o_done) + (size_t)c * cfg.queue_slots;
    S->slot_busy[c].assign((size_t)cfg.queue_slots, 0);
  }
  sd.stop = (const int*)(dp + offsetof(MappedQueues, stop));
  // device memory: heads, team counters, claims, abort flag, team partials; then the arena
  const size_t stride = (size_t)2 * kMaxRed * std::max(large_K, small_K);
  const size_t dev_small = 256 * 2 + (size_t)n_teams * 64 * 4 * 2 + 256 + (size_t)n_teams * stride * 8 + 4096;
  const size_t arena_bytes = (size_t)cfg.hbm_budget_bytes;
  cudaError_t e = cudaMalloc(&S->dev_base, align_up(dev_small, 256) + arena_bytes);
  if (e != cudaSuccess) {
    cudaFreeHost(S->mapped_base);
    return fail(ctx, KIOPS_ENOMEM, "server memory (budget %.3g bytes): %s", cfg.hbm_budget_bytes, cudaGetErrorString(e));
  }
  char* db = (char*)S->dev_base;
  KCHECK(ctx, cudaMemset(db, 0, dev_small));
  sd.head[0] = (unsigned int*)db;
  sd.head[1] = (unsigned int*)(db + 256);
  sd.team_ctr = (unsigned int*)(db + 512);
  sd.team_claim = (int*)(db + 512 + (size_t)n_teams * 64 * 4);
  sd.abort_flag = (int*)(db + 512 + (size_t)n_teams * 64 * 8);
  sd.team_partials = (double*)(db + align_up(512 + (size_t)n_teams * 64 * 8 + 256, 256));
  sd.team_partials_stride = stride;
  sd.timeout_ns = (long long)(ctx->cfg.timeout_s * 1e9);
  sd.idle_ns = (long long)(cfg.idle_timeout_s * 1e9);
  S->arena_base = db + align_up(dev_small, 256);
  S->arena.init(arena_bytes);
  KCHECK(ctx, cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking));
  KCHECK(ctx, cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking));
  KCHECK(ctx, cudaEventCreateWithFlags(&S->kdone, cudaEventDisableTiming));
  ctx->server = S.release();
  return KIOPS_OK;
}

kiops_status kiops_submit(kiops_ctx* ctx, const kiops_request* r, uint64_t* ticket) {
  if (!ctx || !r || !ticket) return KIOPS_EINVAL;
  KiopsServer* S = ctx->server;
  if (!S) return fail(ctx, KIOPS_EINVAL, "no server: call kiops_server_start first");
  if (!r->A || !r->b || !r->w) return fail(ctx, KIOPS_EINVAL, "NULL operator, b or w");
  if (!(r->tau > 0.0)) return fail(ctx, KIOPS_EINVAL, "served requests need tau > 0");
  if (S->cfg.solo_min_unknowns > 0 && (double)r->A->d.n >= S->cfg.solo_min_unknowns) {
    Prepared P;  // validates the request as kiops_solve does
    kiops_status st = prepare(ctx, r->A, r->tau, r->p, r->b, r->tol, r->m_init, r->m_o, r->prec, r->w, 1, 0, P);
    if (st) return st;
    SoloReq q;
    q.ticket = S->next_ticket++;
    q.r = *r;
    q.b.assign(r->b, r->b + r->p + 1);
    S->solo.push_back(q);
    *ticket = q.ticket;
    return server_pump(ctx, S);
  }
  const int cls = (S->cfg.large_teams > 0 && estimate_work(ctx, *r) > S->cfg.large_work_threshold) ? 1 : 0;
  Pending pd;
  pd.ticket = S->next_ticket++;
  pd.cls = cls;
  kiops_status st = prepare(ctx, r->A, r->tau, r->p, r->b, r->tol, r->m_init, r->m_o, r->prec, r->w,
                            S->sd.team_blocks[cls], 0, pd.P);
  if (st) return st;
  if (pd.P.L.total > S->arena.bytes)
    return fail(ctx, KIOPS_ENOMEM, "request workspace %zu bytes exceeds the HBM budget %zu", pd.P.L.total, S->arena.bytes);
  S->pending.push_back(pd);
  *ticket = pd.ticket;
  return server_pump(ctx, S);
}

kiops_status kiops_poll(kiops_ctx* ctx, uint64_t ticket, double timeout_s, int* done, kiops_stats* stats) {
  if (!ctx || !done) return KIOPS_EINVAL;
  KiopsServer* S = ctx->server;
  if (!S) return fail(ctx, KIOPS_EINVAL, "no server");
  *done = 0;
  auto t0 = std::chrono::steady_clock::now();
  while (true) {
    kiops_status st = server_pump(ctx, S, true);
    if (st) return st;
    auto it = S->finished.find(ticket);
    if (it != S->finished.end()) {
      const std::vector<int64_t>& sv = it->second;
      fill_stats(stats, sv.data(), (const double*)(sv.data() + 10), KIOPS_ENGINE_GRID,
                 (int)S->sd.team_blocks[0]);
      const int dst = (int)sv[6];
      S->finished.erase(it);
      *done = 1;
      if (dst != ST_OK) return fail(ctx, (kiops_status)dst, "served request %llu: device status %d",
                                    (unsigned long long)ticket, dst);
      return KIOPS_OK;
    }
    const bool known = S->inflight.count(ticket) ||
                       std::any_of(S->pending.begin(), S->pending.end(), [&](const Pending& p) { return p.ticket == ticket; }) ||
                       std::any_of(S->solo.begin(), S->solo.end(), [&](const SoloReq& q) { return q.ticket == ticket; });
    if (!known) return fail(ctx, KIOPS_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el >= timeout_s) return KIOPS_OK;
  }
}

kiops_status kiops_server_stop(kiops_ctx* ctx) {
  if (!ctx) return KIOPS_EINVAL;
  KiopsServer* S = ctx->server;
  if (!S) return KIOPS_OK;
  __atomic_store_n(&S->q->stop[0], 1, __ATOMIC_RELEASE);
  kiops_status rc = KIOPS_OK;
  if (S->launched && cudaStreamSynchronize(S->kstream) != cudaSuccess) rc = fail(ctx, KIOPS_ECUDA, "server kernel failed");
  cudaEventDestroy(S->kdone);
  cudaStreamDestroy(S->kstream);
  cudaStreamDestroy(S->cstream);
  cudaFree(S->dev_base);
  cudaFreeHost(S->mapped_base);
  delete S;
  ctx->server = nullptr;
  return rc;
}

kiops_status kiops_server_info(kiops_ctx* ctx, int64_t info[8]) {
  if (!ctx || !info || !ctx->server) return KIOPS_EINVAL;
  KiopsServer* S = ctx->server;
  size_t free_bytes = 0;
  for (auto& kv : S->arena.free_) free_bytes += kv.second;
  info[0] = (int64_t)(S->pending.size() + S->solo.size());
  info[1] = (int64_t)S->inflight.size();
  info[2] = (int64_t)(S->arena.bytes - free_bytes);
  info[3] = S->sd.teams[0];
  info[4] = S->sd.teams[1];
  info[5] = S->sd.team_blocks[1];
  unsigned int heads[kServerClasses] = {};  // copy-engine reads: they proceed while the kernel runs
  for (int c = 0; c < kServerClasses; ++c)
    KCHECK(ctx, cudaMemcpyAsync(heads + c, S->sd.head[c], sizeof(unsigned int), cudaMemcpyDeviceToHost, S->cstream));
  KCHECK(ctx, cudaStreamSynchronize(S->cstream));
  info[6] = heads[0];
  info[7] = heads[1];
  return KIOPS_OK;
}

kiops_status kiops_server_selftest_abort(kiops_ctx* ctx) {
  if (!ctx || !ctx->server) return KIOPS_EINVAL;
  KiopsServer* S = ctx->server;
  // a copy-engine write, so it lands while the server kernel occupies every SM
  const int v = ST_ETIMEOUT;
  KCHECK(ctx, cudaMemcpyAsync(S->sd.abort_flag, &v, sizeof(int), cudaMemcpyHostToDevice, S->cstream));
  KCHECK(ctx, cudaStreamSynchronize(S->cstream));
  return KIOPS_OK;
}

// ---- FP64 throughput probe -------------------------------------------------------------------------------
kiops_status kiops_probe_fp64(kiops_ctx* ctx, double* flops_per_s) {
  if (!ctx || !flops_per_s) return KIOPS_EINVAL;
  *flops_per_s = 0.0;
  const int iters = 4096, max_blocks = 4 * ctx->sms;
  void* buf = nullptr;
  KCHECK(ctx, cudaMalloc(&buf, (size_t)max_blocks * kiops_k::probe_threads() * sizeof(double)));
  std::unique_ptr<void, cudaError_t (*)(void*)> guard(buf, cudaFree);
  cudaEvent_t e0, e1;
  KCHECK(ctx, cudaEventCreate(&e0));
  KCHECK(ctx, cudaEventCreate(&e1));
  double best = 0.0;
  for (int chains : {8, 16})
    for (int per_sm : {2, 4}) {
      const int blocks = per_sm * ctx->sms;
      KCHECK(ctx, kiops_k::launch_fp64_probe(chains, blocks, iters, (double*)buf, ctx->stream));  // warm-up
      for (int r = 0; r < 3; ++r) {
        KCHECK(ctx, cudaEventRecord(e0, ctx->stream));
        KCHECK(ctx, kiops_k::launch_fp64_probe(chains, blocks, iters, (double*)buf, ctx->stream));
        KCHECK(ctx, cudaEventRecord(e1, ctx->stream));
        KCHECK(ctx, cudaEventSynchronize(e1));
        float ms = 0.0f;
        KCHECK(ctx, cudaEventElapsedTime(&ms, e0, e1));
        const double f = kiops_k::probe_flops_per_thread(chains, iters) * (double)blocks * kiops_k::probe_threads();
        if (ms > 0.0f) best = std::max(best, f / (1e-3 * (double)ms));
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *flops_per_s = best;
  return KIOPS_OK;
}

// ---- Self-test of the bounded device-side waits ----------------------------------------------------------
kiops_status kiops_selftest_wait_timeout(kiops_ctx* ctx, double timeout_s) {
  if (!ctx) return KIOPS_EINVAL;
  if (!(timeout_s > 0.0) || timeout_s > 5.0) return fail(ctx, KIOPS_EINVAL, "timeout_s must be in (0, 5]");
  void* buf = nullptr;  // counter line, abort flag, results
  KCHECK(ctx, cudaMalloc(&buf, 512));
  std::unique_ptr<void, cudaError_t (*)(void*)> guard(buf, cudaFree);
  char* b = (char*)buf;
  KCHECK(ctx, cudaMemsetAsync(buf, 0, 512, ctx->stream));
  barrier_timeout_kernel<<<1, 64, 0, ctx->stream>>>((unsigned int*)b, (int*)(b + 128), (long long)(timeout_s * 1e9),
                                                    (int*)(b + 256));
  KCHECK(ctx, cudaGetLastError());
  int out[2] = {0, 0};
  KCHECK(ctx, cudaMemcpyAsync(out, b + 256, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  if (out[0] == 0 && out[1] == ST_ETIMEOUT)
    return fail(ctx, KIOPS_ETIMEOUT, "a device-side wait exceeded %.3g s (self-test: expected)", timeout_s);
  return fail(ctx, KIOPS_ECUDA, "wait self-test: barrier passed = %d, abort flag = %d", out[0], out[1]);
}

// ---- Exponential integrators (section 4) -------------------------------------------------------------
static kiops_status pde_dev(kiops_ctx* ctx, const kiops_pde* pde, kiops_k::PdeDev& P) {
  if (!pde) return fail(ctx, KIOPS_EINVAL, "NULL problem");
  if (pde->kind != KIOPS_PDE_ADR2D && pde->kind != KIOPS_PDE_GRAY_SCOTT2D)
    return fail(ctx, KIOPS_EINVAL, "unknown test problem %d", pde->kind);
  if (pde->n < 2 || (pde->kind == KIOPS_PDE_GRAY_SCOTT2D ? 2 : 1) * pde->n * pde->n > INT32_MAX)
    return fail(ctx, KIOPS_EINVAL, "grid size n = %lld outside [2, 2^31-1 unknowns]", (long long)pde->n);
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(pde->param[k])) return fail(ctx, KIOPS_EINVAL, "parameter %d is not finite", k);
  std::memset(&P, 0, sizeof(P));
  P.kind = pde->kind;
  P.n = pde->n;
  if (pde->kind == KIOPS_PDE_ADR2D) {
    P.ns = 1;
    P.bc = KIOPS_BC_NEUMANN;
    P.dx = 1.0 / (double)(pde->n - 1);
  } else {
    P.ns = 2;
    P.bc = KIOPS_BC_PERIODIC;
    P.dx = 1.0 / (double)pde->n;
  }
  for (int k = 0; k < 4; ++k) P.prm[k] = pde->param[k];
  return KIOPS_OK;
}

kiops_status kiops_pde_rhs(kiops_ctx* ctx, const kiops_pde* pde, const double* u, double* f) {
  if (!ctx) return KIOPS_EINVAL;
  if (!u || !f) return fail(ctx, KIOPS_EINVAL, "NULL u or f");
  kiops_k::PdeDev P;
  kiops_status st = pde_dev(ctx, pde, P);
  if (st) return st;
  KCHECK(ctx, kiops_k::launch_pde_eval(P, u, 1.0, f, nullptr, ctx->sms, ctx->stream));
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  return KIOPS_OK;
}

kiops_status kiops_integrate(kiops_ctx* ctx, const kiops_pde* pde, int scheme, double t0, double t1, int64_t nsteps,
                             double tol, int m_init, double* u, kiops_integrate_stats* stats) {
  NvtxRange nvtx_range("kiops integrate");
  if (!ctx) return KIOPS_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  kiops_k::PdeDev P;
  kiops_status st = pde_dev(ctx, pde, P);
  if (st) return st;
  if (scheme < KIOPS_EPIRK4S3 || scheme > KIOPS_EXPRB5S3) return fail(ctx, KIOPS_EINVAL, "unknown scheme %d", scheme);
  if (!u) return fail(ctx, KIOPS_EINVAL, "NULL u");
  if (!(t1 > t0) || !std::isfinite(t0) || !std::isfinite(t1) || nsteps < 1)
    return fail(ctx, KIOPS_EINVAL, "need t1 > t0 (finite) and nsteps >= 1");
  if (!(tol > 0.0) || m_init < 1) return fail(ctx, KIOPS_EINVAL, "tol must be > 0 and m_init >= 1");
  // stage nodes (increasing, as Task I wants them) and the b_3, b_4 weights: eqs 50, 51, 53 (eq 11 grouping)
  double c2, c3;
  kiops_k::SchemeDev S{};
  if (scheme == KIOPS_EPIRK4S3) {
    c2 = 1.0 / 8.0;
    c3 = 1.0 / 9.0;
    S = {1892.0, 1458.0, -42336.0, -34992.0, -2.0};
  } else if (scheme == KIOPS_EPIRK4S3A) {
    c2 = 0.5;
    c3 = 2.0 / 3.0;
    S = {32.0, -13.5, -144.0, 81.0, 0.0};
  } else {
    c2 = 0.5;
    c3 = 0.9;
    S = {18.0, -250.0 / 81.0, -60.0, 500.0 / 27.0, 0.0};
  }
  const double nodes[2] = {std::min(c2, c3), std::max(c2, c3)};
  const int64_t npts = P.n * P.n, N = npts * P.ns;
  // workspace: zero, hf, W[2], U2, U3, b3, b4, Z[2], w, h r2 (N each), coupling fields (4 x npts)
  const size_t need = (size_t)(12 * N + 4 * npts) * sizeof(double);
  if (need > ctx->integ_bytes) {
    if (ctx->integ) cudaFree(ctx->integ);
    ctx->integ = nullptr;
    ctx->integ_bytes = 0;
    KCHECK(ctx, cudaMalloc((void**)&ctx->integ, need));
    ctx->integ_bytes = need;
  }
  double* base = ctx->integ;
  double *zero = base, *hf = base + N, *U2 = base + 4 * N, *U3 = base + 5 * N;
  double* W[2] = {base + 2 * N, base + 3 * N};
  double *b3 = base + 6 * N, *b4 = base + 7 * N, *w = base + 10 * N, *hr2 = base + 11 * N;
  double* Z[2] = {base + 8 * N, base + 9 * N};
  double* fields[4] = {base + 12 * N, base + 12 * N + npts, base + 12 * N + 2 * npts, base + 12 * N + 3 * npts};
  KCHECK(ctx, cudaMemsetAsync(zero, 0, (size_t)N * sizeof(double), ctx->stream));
  // A = h J_n: the stencil part scaled by h, the coupling fields h dR(u_n) (rewritten every step)
  const double h = (t1 - t0) / (double)nsteps;
  kiops_stencil2d_desc d;
  std::memset(&d, 0, sizeof(d));
  d.nx = d.ny = P.n;
  d.nspecies = P.ns;
  d.bc = P.bc;
  const double idx2 = 1.0 / (P.dx * P.dx);
  for (int sp = 0; sp < P.ns; ++sp) {
    double dd, aa = 0.0;
    if (P.kind == KIOPS_PDE_ADR2D) {
      dd = P.prm[0] * idx2;
      aa = P.prm[1] / (2.0 * P.dx);
    } else {
      dd = P.prm[sp] * idx2;
    }
    const double cf[5] = {-4.0 * dd, dd + aa, dd - aa, dd + aa, dd - aa};
    for (int k = 0; k < 5; ++k) d.coef[sp][k] = h * cf[k];
  }
  d.diag[0][0] = fields[0];
  if (P.ns == 2) {
    d.diag[0][1] = fields[1];
    d.diag[1][0] = fields[2];
    d.diag[1][1] = fields[3];
  }
  kiops_op* A = nullptr;
  st = kiops_op_stencil2d(ctx, &A, &d);
  if (st) return st;
  std::unique_ptr<kiops_op, kiops_status (*)(kiops_op*)> A_guard(A, kiops_op_destroy);
  int m_slot[3] = {m_init, m_init, m_init};
  auto tally = [&](const kiops_stats& s, int slot) {
    m_slot[slot] = s.m_last;
    if (stats) {
      stats->kiops_calls += 1;
      stats->matvecs += s.matvecs;
      stats->substeps += s.substeps;
      stats->rejected += s.rejected;
      stats->m_last[slot] = s.m_last;
    }
  };
  for (int64_t n = 0; n < nsteps; ++n) {
    NvtxRange step_range("integrator step");
    // h f(u_n) and the fields of A = h J_n
    KCHECK(ctx, kiops_k::launch_pde_eval(P, u, h, hf, fields, ctx->sms, ctx->stream));
    // Task I: phi_1(c A) h f(u_n) at both nodes
    {
      const double* bb[2] = {zero, hf};
      double* const ww[2] = {W[0], W[1]};
      kiops_stats s1{};
      st = kiops_solve_task1(ctx, A, nodes, 2, 1, bb, tol, m_slot[0], 2, KIOPS_FP64, ww, &s1);
      if (st) return st;
      tally(s1, 0);
    }
    const double* W2 = c2 == nodes[0] ? W[0] : W[1];
    const double* W3 = c3 == nodes[0] ? W[0] : W[1];
    KCHECK(ctx, kiops_k::launch_stages(N, u, W2, c2, W3, c3, U2, U3, ctx->sms, ctx->stream));
    if (scheme == KIOPS_EXPRB5S3) {
      // Task I: phi_3(c A) h r(U_n2) at c = 1/2, 9/10; U_n3 += 27/25 Z(1/2) + 729/125 Z(9/10)
      KCHECK(ctx, kiops_k::launch_remainder(P, u, U2, h, hr2, ctx->sms, ctx->stream));
      const double* bb[4] = {zero, zero, zero, hr2};
      double* const zz[2] = {Z[0], Z[1]};
      kiops_stats s2{};
      st = kiops_solve_task1(ctx, A, nodes, 2, 3, bb, tol, m_slot[1], 2, KIOPS_FP64, zz, &s2);
      if (st) return st;
      tally(s2, 1);
      KCHECK(ctx, kiops_k::launch_axpy2(N, U3, 27.0 / 25.0, Z[0], 729.0 / 125.0, Z[1], ctx->sms, ctx->stream));
    }
    // b_3, b_4 from r(U_n2), r(U_n3); Task II (eq 10, tau = 1) gives u_{n+1} - u_n
    KCHECK(ctx, kiops_k::launch_assemble(P, u, U2, U3, h, S, b3, b4, ctx->sms, ctx->stream));
    {
      const double* bb[5] = {zero, hf, zero, b3, b4};
      kiops_stats s3{};
      st = kiops_solve(ctx, A, 1.0, 4, bb, tol, m_slot[2], 2, KIOPS_FP64, w, &s3);
      if (st) return st;
      tally(s3, 2);
    }
    KCHECK(ctx, kiops_k::launch_axpy2(N, u, 1.0, w, 0.0, nullptr, ctx->sms, ctx->stream));
    if (stats) stats->steps = n + 1;
  }
  KCHECK(ctx, cudaStreamSynchronize(ctx->stream));
  return KIOPS_OK;
}

}  // extern "C"
