// lbm_api.cu - host implementation of the C ABI declared in include/lbm.h.
//
// A domain owns one device workspace holding, 256-byte aligned:
//   h[2][q_phase][N], g[2][27][N], f[2][Q_f][N]     PDF double buffers (storage type)
//   T[N], u[3][N], S_a[N], S_b[N], acc[N]           RK thermal fields (compute type)
//   diagnostics partials [grid][7], result [8]      FP64 reduction scratch
//   droplet table [LBM_MAX_DROPLETS][7]             FP64 init input
// Each step reads buffer `cur` and writes `cur ^ 1`, then flips `cur`.  With
// the in-place (AA) layout there is one PDF set, stepped in place, plus a
// (phi, T) field [N] of the compute type that each step refreshes first.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/lbm.h"
#include "launchers.h"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

lbm_status fail(lbm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int thermal_q(lbm_thermal th) {
  switch (th) {
    case LBM_TH_D3Q7: return 7;
    case LBM_TH_D3Q15: return 15;
    case LBM_TH_D3Q19: return 19;
    case LBM_TH_D3Q27: return 27;
    default: return 0;
  }
}

size_t store_bytes(lbm_precision p) { return p == LBM_FP64 ? 8 : (p == LBM_FP32 ? 4 : 2); }
size_t field_bytes(lbm_precision p) { return p == LBM_FP64 ? 8 : 4; }

struct Layout {
  size_t h[2], g[2], f[2], T, u, sa, sb, acc, phi, phiT, partials, diag, drops, errflag, total;
};

// Launch geometry of the step kernel: TX x rows columns, z split into chunks;
// the bulk kernel's grid is one-dimensional (sched, see BulkSched).
struct Geometry {
  dim3 grid;       // generic kernel: (tiles x, tiles y, chunks); bulk: the same counts (reported only)
  int zchunk;
  int nblocks;     // blocks of one launch (diagnostics partials)
  int bulk;        // 2: skewed kernel, 1: bulk kernel (tensor-TMA staging), 0: generic kernel
  BulkSched sched;
};

int thermal_q(lbm_thermal th);

// The bulk kernel needs 16-byte aligned rows, rows at least one staged
// row long, at least two tiles of rows, and shared memory that fits.
bool bulk_ok(int nx, int ny, lbm_precision prec, int qh, int qf) {
  const char* env = std::getenv("LBM_KERNEL");
  if (env && std::strcmp(env, "generic") == 0) return false;
  if (nx < bulk_box_cols((int)prec)) return false;
  const int rows = bulk_tile_rows((int)prec, qh, qf);
  if (ny < 2 * rows || (ny + rows - 1) / rows > 65535) return false;
  return bulk_smem_bytes((int)prec, qh, qf) <= kMaxDynSmem;
}

// Bulk kernel: one CTA per SM.  The schedule minimises the modelled time of
// the launch, (waves of whole units) x (planes + prologue) + (waves of tail
// pieces) x (planes / npiece + prologue), over the chunk count (>= 16 planes
// per chunk) and the tail split (>= 8 planes per piece); the prologue (three
// h/f stages and one g stage before the first plane) costs about two planes.
BulkSched bulk_schedule(int bx, int by, int nz, int sms, int forced_zchunk) {
  const long long cols = (long long)bx * by;
  BulkSched best{bx, by, 1, nz, (int)cols, 1};
  if (forced_zchunk > 0) {
    best.zchunk = forced_zchunk;
    best.nchunk = (nz + forced_zchunk - 1) / forced_zchunk;
    best.nfull = (int)(cols * best.nchunk);
    return best;
  }
  const double prologue = 2.0;
  double best_cost = 1e300;
  const int max_chunks = nz / 16 > 1 ? nz / 16 : 1;
  for (int k = 1; k <= max_chunks; ++k) {
    const int zc = (nz + k - 1) / k;
    const int nchunk = (nz + zc - 1) / zc;
    const long long units = cols * nchunk;
    const long long full_waves = units / sms;
    const long long rem = units - full_waves * sms;
    for (int p = 1; p <= 8; ++p) {
      if (p > 1 && (rem == 0 || zc / p < 8)) break;
      double cost = (double)full_waves * (zc + prologue);
      if (rem > 0) cost += (double)((rem * p + sms - 1) / sms) * ((double)zc / p + prologue);
      if (cost < best_cost - 1e-9) {
        best_cost = cost;
        // p == 1: every unit runs whole; else the units past the last full
        // wave are cut into p pieces
        best = BulkSched{bx, by, nchunk, zc, (int)(p == 1 ? units : units - rem), p};
      }
    }
  }
  return best;
}

Geometry geometry(int nx, int ny, int nz, lbm_precision prec, int qh, int qf, int sms, bool allow_bulk = true) {
  Geometry g;
  g.bulk = allow_bulk && bulk_ok(nx, ny, prec, qh, qf) ? 1 : 0;
  const int rows = g.bulk ? bulk_tile_rows((int)prec, qh, qf) : TY;
  const int cols_ = g.bulk ? bulk_tile_cols((int)prec) : TX;
  const int bx = (nx + cols_ - 1) / cols_, by = (ny + rows - 1) / rows;
  const long long cols = (long long)bx * by;
  const char* env = std::getenv("LBM_ZCHUNK");
  const int forced = env ? std::atoi(env) : 0;
  if (g.bulk) {
    // the skewed kernel where its layout fits (LBM_KERNEL=bulk keeps the bulk one)
    const char* kenv = std::getenv("LBM_KERNEL");
    const bool no_skew = kenv && std::strcmp(kenv, "bulk") == 0;
    if (!no_skew && skew_smem_bytes((int)prec, qh, qf) > 0 && skew_smem_bytes((int)prec, qh, qf) <= kMaxDynSmem)
      g.bulk = 2;
    g.sched = bulk_schedule(bx, by, nz, sms > 0 ? sms : 1, forced);
    g.zchunk = g.sched.zchunk;
    g.grid = dim3(bx, by, g.sched.nchunk);
    g.nblocks = bulk_sched_blocks(g.sched);
    return g;
  }
  int zc = forced;
  if (zc <= 0) {
    // generic: ~8 CTAs per SM, chunks of >= 8 planes
    const long long want = (long long)(sms > 0 ? sms : 1) * 8;
    int nchunks = (int)((want + cols - 1) / cols);
    if (nchunks > nz / 8) nchunks = nz / 8;
    if (nchunks < 1) nchunks = 1;
    zc = (nz + nchunks - 1) / nchunks;
  }
  const int nchunks = (nz + zc - 1) / zc;
  g.grid = dim3(bx, by, nchunks);
  g.zchunk = zc;
  g.nblocks = (int)(cols * nchunks);
  g.sched = BulkSched{bx, by, nchunks, zc, g.nblocks, 1};
  return g;
}

// Padded PDF geometry: GX = 16 / sizeof(storage) ghost columns and
// kGhostRows ghost rows on each side; the row pitch is a multiple of 16 bytes.
struct Pad {
  int GX, GY, NXP, NYP;
  size_t Np;
};

Pad padding(int nx, int ny, int nz, lbm_precision prec) {
  Pad p;
  const int s = (int)store_bytes(prec);
  p.GX = 16 / s;
  p.GY = kGhostRows;
  const int align = 16 / s;
  p.NXP = ((nx + 2 * p.GX + align - 1) / align) * align;
  p.NYP = ny + 2 * p.GY;
  p.Np = (size_t)nz * p.NYP * p.NXP;
  return p;
}

bool layout(int nx, int ny, int nz, lbm_precision prec, lbm_thermal th, int qh, Layout* L, bool aa = false) {
  // launch grids put nz (one plane per z block) and ny / 4 on the 16-bit grid axes
  if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || ny > 262140) return false;
  if (qh != 15 && qh != 27) return false;
  if (prec < LBM_FP64 || prec > LBM_FP16_STORE) return false;
  if (th < LBM_TH_D3Q7 || th > LBM_TH_RK4) return false;
  const size_t N = (size_t)nx * ny * nz;
  if (N >= (size_t(1) << 40)) return false;
  const Pad pd = padding(nx, ny, nz, prec);
  const size_t sb = store_bytes(prec), fb = field_bytes(prec);
  const int qf = thermal_q(th);
  size_t off = 0;
  // one PDF set = [h (qh) | g (27) | f (qf)] directions of Np elements each,
  // contiguous, so that one ghost-fill launch covers the whole set
  for (int k = 0; k < 2; ++k) {
    if (aa && k == 1) {
      // in-place layout: one set, both indices name it
      L->h[1] = L->h[0];
      L->g[1] = L->g[0];
      L->f[1] = L->f[0];
      break;
    }
    L->h[k] = off;
    L->g[k] = off + (size_t)qh * pd.Np * sb;
    L->f[k] = L->g[k] + (size_t)27 * pd.Np * sb;
    off = align256(L->f[k] + (size_t)qf * pd.Np * sb);
  }
  const bool rk = qf == 0;
  const bool rk4 = th == LBM_TH_RK4;
  L->T = off; off = align256(off + (rk ? N * fb : 0));
  L->u = off; off = align256(off + (rk ? 3 * N * fb : 0));
  L->sa = off; off = align256(off + (rk ? N * fb : 0));
  L->sb = off; off = align256(off + (rk4 ? N * fb : 0));
  L->acc = off; off = align256(off + (rk4 ? N * fb : 0));
  L->phi = off; off = align256(off + (rk ? N * fb : 0));   // phi of the step (conductivity ratio)
  L->phiT = off; off = align256(off + (aa ? 2 * N * fb : 0));   // (phi, T) of the level (in-place layout)
  // room for the largest grid any kernel / z-chunk choice can produce
  const size_t max_blocks = (size_t)((nx + TX - 1) / TX) * ((ny + 3) / 4) * nz;
  L->partials = off; off = align256(off + max_blocks * kDiagVals * 8);
  L->diag = off; off = align256(off + 8 * 8);
  L->drops = off; off = align256(off + (size_t)LBM_MAX_DROPLETS * 7 * 8);
  L->errflag = off; off = align256(off + sizeof(int));
  L->total = off;
  return true;
}

}  // namespace

struct lbm_domain {
  int nx, ny, nz;
  long long N;
  lbm_precision prec;
  lbm_thermal th;
  int qh, qf;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  bool owns_ws;
  Layout L;
  Geometry geo;
  Geometry geo_aa{};     // in-place layout: the tiled kernels' geometry (bulk == 2 when they apply)
  int diag_nblocks = 0;  // CTAs of the last step launch (diagnostics partials)
  bool aa = false;  // in-place (AA) layout
  int sms;  // multiprocessors of the device (launch geometry)
  int cur;
  bool params_set, inited;
  long long level;
  lbm_params params;
  DevParams dp;
  void* staging;  // device buffer for host-bound field copies (lazy)
  size_t staging_bytes;
  lbm_status sticky;
  std::string sticky_msg;
  TMaps maps[2];  // tensor maps of PDF set 0 / 1 (bulk kernel)
  int test_stall = 0;  // LBM_TEST_STALL at creation
  // MODE_SAVE target of the next passes (FP64 adjoint; [SAVE_N][N] doubles)
  double* save_ptr = nullptr;
  // step-kernel timing (lbm_profile_steps): event pairs around each launch
  std::vector<cudaEvent_t> prof_ev;
  bool prof_on = false;
  int prof_n = 0;
};

namespace {

lbm_status check_cuda(lbm_domain* d, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LBM_OK;
  const std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  if (d) {
    d->sticky = LBM_ERR_CUDA;
    d->sticky_msg = msg;
  }
  return fail(LBM_ERR_CUDA, msg);
}

lbm_status check_launch(lbm_domain* d, const char* what) {
  return check_cuda(d, cudaGetLastError(), what);
}

lbm_status usable(lbm_domain* d) {
  if (!d) return fail(LBM_ERR_ARG, "null domain");
  if (d->sticky != LBM_OK) return fail(d->sticky, "domain has a sticky error: " + d->sticky_msg);
  return LBM_OK;
}

void* at(lbm_domain* d, size_t off) { return d->ws + off; }
// the current PDF set ([h | g | f], padded, storage precision)
char* cur_set_ptr(lbm_domain* d) { return d->ws + d->L.h[d->cur]; }

// ----------------------------------------------------------------- dispatch
template <class S>
StepPtrs<S, typename Store<S>::R> ptrs(lbm_domain* d) {
  using R = typename Store<S>::R;
  StepPtrs<S, R> A{};
  const int c = d->cur;
  A.h_src = (const S*)at(d, d->L.h[c]);
  A.h_dst = (S*)at(d, d->L.h[c ^ 1]);
  A.g_src = (const S*)at(d, d->L.g[c]);
  A.g_dst = (S*)at(d, d->L.g[c ^ 1]);
  A.f_src = (const S*)at(d, d->L.f[c]);
  A.f_dst = (S*)at(d, d->L.f[c ^ 1]);
  A.T = (const R*)at(d, d->L.T);
  A.u_out = (R*)at(d, d->L.u);
  A.s1_out = (R*)at(d, d->L.sa);
  A.acc_out = (R*)at(d, d->L.acc);
  A.phi_out = (R*)at(d, d->L.phi);
  A.rk_acc = d->th == LBM_TH_RK4;
  A.diag_partials = (double*)at(d, d->L.partials);
  A.save = std::is_same<R, double>::value ? (R*)d->save_ptr : nullptr;
  A.error_flag = (int*)at(d, d->L.errflag);
  const size_t np = (size_t)d->dp.Np;
  for (int i = 0; i < 27; ++i) {
    A.hd[i] = i < d->qh ? A.h_dst + (size_t)i * np : nullptr;
    A.gd[i] = A.g_dst + (size_t)i * np;
    A.fd[i] = i < d->qf ? A.f_dst + (size_t)i * np : nullptr;
  }
  return A;
}

template <class S, int QH>
void step_qf(lbm_domain* d, const StepPtrs<S, typename Store<S>::R>& A, int mode) {
  switch (d->qf) {
    case 0: launch_step<S, QH, 0>(d->dp, A, d->maps[d->cur], d->geo.grid, d->geo.zchunk, d->geo.sched, mode, d->geo.bulk, d->stream); break;
    case 7: launch_step<S, QH, 7>(d->dp, A, d->maps[d->cur], d->geo.grid, d->geo.zchunk, d->geo.sched, mode, d->geo.bulk, d->stream); break;
    case 15: launch_step<S, QH, 15>(d->dp, A, d->maps[d->cur], d->geo.grid, d->geo.zchunk, d->geo.sched, mode, d->geo.bulk, d->stream); break;
    case 19: launch_step<S, QH, 19>(d->dp, A, d->maps[d->cur], d->geo.grid, d->geo.zchunk, d->geo.sched, mode, d->geo.bulk, d->stream); break;
    default: launch_step<S, QH, 27>(d->dp, A, d->maps[d->cur], d->geo.grid, d->geo.zchunk, d->geo.sched, mode, d->geo.bulk, d->stream); break;
  }
}

template <class S>
void step_launch(lbm_domain* d, const StepPtrs<S, typename Store<S>::R>& A, int mode) {
  d->diag_nblocks = d->geo.nblocks;
  if (d->qh == 15) step_qf<S, 15>(d, A, mode);
  else step_qf<S, 27>(d, A, mode);
}

// In-place layout: (phi, T) of the level, then the step (gathers from the
// neighbours when the level is even, locally when it is odd), on the tiled
// kernels where they apply (all but the density ratio, whose forces need
// the moments and stencils of one plane together, and sub-domains) and on
// the generic tiles otherwise.
bool aa_tiled(const lbm_domain* d) {
  const DevParams& q = d->dp;
  return d->aa && d->geo_aa.bulk == 2 && !(q.sub || q.rho_ratio);
}

template <class S>
void aa_launch(lbm_domain* d, const StepPtrs<S, typename Store<S>::R>& A, int mode) {
  using R = typename Store<S>::R;
  const int nb = (d->level & 1) == 0 ? 1 : 0;
  void* phiT = at(d, d->L.phiT);
  const bool tiled = aa_tiled(d);
  d->diag_nblocks = tiled ? d->geo_aa.nblocks : d->geo.nblocks;
  auto qf = [&](auto qh_tag) {
    constexpr int QH = decltype(qh_tag)::value;
    auto go = [&](auto qf_tag) {
      constexpr int QF = decltype(qf_tag)::value;
      if (tiled)
        launch_aa_tiled<S, QH, QF>(d->dp, A, d->maps[0], phiT, nb, d->geo_aa.sched, mode, d->stream);
      else
        launch_aa_step<S, QH, QF>(d->dp, A, phiT, nb, d->geo.grid, d->geo.zchunk, mode, d->stream);
    };
    switch (d->qf) {
      case 0: go(std::integral_constant<int, 0>{}); break;
      case 7: go(std::integral_constant<int, 7>{}); break;
      case 15: go(std::integral_constant<int, 15>{}); break;
      case 19: go(std::integral_constant<int, 19>{}); break;
      default: go(std::integral_constant<int, 27>{}); break;
    }
  };
  (void)sizeof(R);
  if (d->qh == 15) qf(std::integral_constant<int, 15>{});
  else qf(std::integral_constant<int, 27>{});
}

template <class S>
void rk_tail(lbm_domain* d) {
  using R = typename Store<S>::R;
  R* T = (R*)at(d, d->L.T);
  R* u = (R*)at(d, d->L.u);
  R* sa = (R*)at(d, d->L.sa);
  R* sb = (R*)at(d, d->L.sb);
  R* acc = (R*)at(d, d->L.acc);
  const R* phi = d->dp.alpha_ratio ? (const R*)at(d, d->L.phi) : nullptr;
  if (d->th == LBM_TH_RK2) {
    launch_rk_stage<S>(d->dp, sa, T, u, phi, nullptr, nullptr, 0, d->stream);
  } else {
    launch_rk_stage<S>(d->dp, sa, T, u, phi, acc, sb, 1, d->stream);   // S2 -> sb
    launch_rk_stage<S>(d->dp, sb, T, u, phi, acc, sa, 2, d->stream);   // S3 -> sa
    launch_rk_stage<S>(d->dp, sa, T, u, phi, acc, nullptr, 3, d->stream);
  }
}

// Direction i of stencil Q (7, 15, 19, 27): its velocity components.
static void stencil_c(int Q, int i, int c[3]) {
  const int k = (Q == 15 && i >= 7) ? i + 12 : i;   // D3Q15 indexes into D3Q27 past the faces
  c[0] = q27_cx(k);
  c[1] = q27_cy(k);
  c[2] = q27_cz(k);
}

// The ghost sides the tiled two-grid kernels read, per array of a PDF set
// (the bits of GhostSides).  g is only pulled into the tile's own cells, so
// direction c reads the ghosts at depth 1 on the side -c points to: x < 0
// for c_x = 1, x >= nx for c_x = -1, none for c_x = 0 (y alike).  h and f are
// also summed into phi and T over the tile's one-cell halo ring, whose pulls
// reach x = -1 - c_x and x = nx - c_x: the columns x < 0 unless c_x = -1, the
// columns x >= nx unless c_x = 1.  Beyond a z wall the bounce-back source of
// a halo cell is the opposite direction at that cell itself, so on plane 0
// the arrays with c_z = -1 (the opposites of c_z = 1) are read on every side
// at depth 1, and on plane nz - 1 those with c_z = 1.
static void ghost_sides(const lbm_domain* d, unsigned char* m) {
  int q = 0, c[3];
  auto halo = [&](int Q, int n) {
    for (int i = 0; i < n; ++i) {
      stencil_c(Q, i, c);
      unsigned v = (c[0] >= 0 ? 1u : 0u) | (c[0] <= 0 ? 2u : 0u) | (c[1] >= 0 ? 4u : 0u) | (c[1] <= 0 ? 8u : 0u);
      if (d->dp.walls) v |= (c[2] < 0 ? 16u : 0u) | (c[2] > 0 ? 32u : 0u);
      m[q++] = (unsigned char)v;
    }
  };
  halo(d->qh, d->qh);
  for (int i = 0; i < 27; ++i) {
    stencil_c(27, i, c);
    m[q++] = (unsigned char)((c[0] > 0 ? 1u : 0u) | (c[0] < 0 ? 2u : 0u) | (c[1] > 0 ? 4u : 0u) |
                             (c[1] < 0 ? 8u : 0u));
  }
  if (d->qf > 0) halo(d->qf, d->qf);
}

// Refresh the periodic ghost cells of PDF set k that the tiled kernels read
// (bulk and skewed kernels only).
void ghost_fill(lbm_domain* d, int k) {
  if (!d->geo.bulk) return;
  void* base = at(d, d->L.h[k]);
  const int nq = d->qh + 27 + d->qf;
  unsigned char sides[27 + 27 + 27];
  ghost_sides(d, sides);
  if (d->prec == LBM_FP64) launch_ghost_fill<double>(d->dp, base, nq, d->stream, sides);
  else if (d->prec == LBM_FP32) launch_ghost_fill<float>(d->dp, base, nq, d->stream, sides);
  else launch_ghost_fill<__half>(d->dp, base, nq, d->stream, sides);
}

// One step (mode: MODE_COLLIDE [| MODE_DIAG]), or a read-only pass.
lbm_status run_pass(lbm_domain* d, int mode, void* macro_out = nullptr, int macro_dtype = 0,
                    unsigned mask = 0) {
  auto go = [&](auto tag) {
    using S = decltype(tag);
    auto A = ptrs<S>(d);
    A.macro_out = macro_out;
    A.macro_dtype = macro_dtype;
    A.macro_mask = mask;
    const bool timed = d->prof_on && (size_t)(2 * d->prof_n + 1) < d->prof_ev.size();
    if (timed) cudaEventRecord(d->prof_ev[2 * d->prof_n], d->stream);
    if (d->aa) aa_launch<S>(d, A, mode);
    else step_launch<S>(d, A, mode);
    if (timed) cudaEventRecord(d->prof_ev[2 * d->prof_n++ + 1], d->stream);
    if (mode & MODE_COLLIDE) ghost_fill(d, d->cur ^ 1);
    if ((mode & MODE_COLLIDE) && d->qf == 0) rk_tail<S>(d);
  };
  if (d->prec == LBM_FP64) go(double{});
  else if (d->prec == LBM_FP32) go(float{});
  else go(__half{});
  lbm_status s = check_launch(d, "step kernel launch");
  if (s != LBM_OK) return s;
  if (mode & MODE_COLLIDE) {
    if (!d->aa) d->cur ^= 1;
    d->level += 1;
  }
  return LBM_OK;
}

// A kernel whose bounded wait ran out raised the device error flag; read it
// after a synchronisation and make it sticky.
lbm_status check_error_flag(lbm_domain* d) {
  int flag = 0;
  lbm_status s = check_cuda(d, cudaMemcpy(&flag, at(d, d->L.errflag), sizeof(int), cudaMemcpyDeviceToHost),
                            "error flag read");
  if (s != LBM_OK) return s;
  if (flag) {
    d->sticky = LBM_ERR_TIMEOUT;
    d->sticky_msg = "a step kernel's bounded wait for its bulk copies ran out";
    return fail(LBM_ERR_TIMEOUT, d->sticky_msg);
  }
  return LBM_OK;
}

lbm_status finish_diag(lbm_domain* d, long long level, lbm_diag* out) {
  launch_diag_finalize((const double*)at(d, d->L.partials), d->diag_nblocks,
                       (double*)at(d, d->L.diag), d->stream);
  lbm_status s = check_launch(d, "diagnostics reduction");
  if (s != LBM_OK) return s;
  double v[kDiagVals];
  s = check_cuda(d, cudaMemcpyAsync(v, at(d, d->L.diag), sizeof(v), cudaMemcpyDeviceToHost, d->stream),
                 "diagnostics copy");
  if (s != LBM_OK) return s;
  s = check_cuda(d, cudaStreamSynchronize(d->stream), "diagnostics sync");
  if (s != LBM_OK) return s;
  s = check_error_flag(d);
  if (s != LBM_OK) return s;
  out->mass = v[0];
  out->heat = v[1];
  out->kinetic = v[2];
  out->mx = v[3];
  out->my = v[4];
  out->mz = v[5];
  out->level = level;
  out->nonfinite = v[6] != 0.0 || !std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2]);
  out->pad_ = 0;
  if (out->nonfinite) return fail(LBM_ERR_NONFINITE, "non-finite value in the state");
  return LBM_OK;
}

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// rho c_p of the light phase; the constant heat capacity when neither rho nor
// c_p differs between the phases (1 at the defaults, so alpha = kappa).
double heat_capacity_L(const lbm_params& p) { return p.rho_L * p.cp_L; }
bool varying_heat_capacity(const lbm_params& p) { return p.rho_L != p.rho_H || p.cp_L != p.cp_H; }

template <class R>
void fill_real(RealParams<R>& r, const lbm_params& p, lbm_precision prec) {
  const double cs2 = 1.0 / 3.0;
  const double alpha_L = p.alpha_L / heat_capacity_L(p);
  r.omega_phi = (R)(1.0 / (0.5 + p.mobility / cs2));
  r.omega_T = (R)(1.0 / (0.5 + alpha_L / cs2));
  r.tau_L = (R)(p.nu_L / cs2 + 0.5);
  r.tau_H = (R)(p.nu_H / cs2 + 0.5);
  r.rho_L = (R)p.rho_L; r.rho_H = (R)p.rho_H; r.xi = (R)p.xi;
  r.sigma_ref = (R)p.sigma_ref; r.sigma_T = (R)p.sigma_T; r.T_ref = (R)p.T_ref; r.alpha = (R)alpha_L;

  for (int k = 0; k < 3; ++k) {
    r.gravity[k] = (R)p.gravity[k];
    r.grad[k] = (R)p.grad_T[k];
    r.origin[k] = (R)p.grad_T_origin[k];
  }
  r.T_bottom = (R)p.T_bottom; r.T_top = (R)p.T_top;

  r.eps_n = (R)p.eps_n;
  r.shift_h = (R)(prec == LBM_FP64 ? 0.0 : 0.5);
  r.shift_f = (R)(prec == LBM_FP64 ? 0.0 : p.T_ref);
}

void refresh_devparams(lbm_domain* d) {
  DevParams& q = d->dp;
  const lbm_params& p = d->params;
  q.nx = d->nx; q.ny = d->ny; q.nz = d->nz; q.N = d->N;
  const Pad pd = padding(d->nx, d->ny, d->nz, d->prec);
  q.GX = pd.GX; q.GY = pd.GY; q.NXP = pd.NXP; q.NYP = pd.NYP; q.Np = (long long)pd.Np;
  q.walls = p.walls_z ? 1 : 0;
  q.rk_iso = p.rk_isotropic_fd ? 1 : 0;
  q.heat_cap = varying_heat_capacity(p) ? 1 : 0;
  q.alpha_ratio = (p.alpha_H != p.alpha_L || q.heat_cap) ? 1 : 0;
  q.tw_waves = p.T_bottom_amp != 0.0 ? p.T_bottom_waves : 0;
  q.dalpha_d = (p.alpha_H - p.alpha_L) / heat_capacity_L(p);
  q.dalpha_f = (float)q.dalpha_d;
  {
    const double hc[6] = {p.alpha_L, p.alpha_H - p.alpha_L, p.rho_L, p.rho_H - p.rho_L, p.cp_L, p.cp_H - p.cp_L};
    for (int k = 0; k < 6; ++k) {
      q.hc_d[k] = hc[k];
      q.hc_f[k] = (float)hc[k];
    }
  }
  q.T_bottom_amp_d = p.T_bottom_amp;
  q.T_bottom_amp_f = (float)p.T_bottom_amp;
  q.test_stall = d->test_stall;
  fill_real(q.pd, p, d->prec);
  fill_real(q.pf, p, d->prec);
  q.moving_walls = (p.walls_z && (p.wall_u_bottom[0] != 0.0 || p.wall_u_bottom[1] != 0.0 ||
                                  p.wall_u_top[0] != 0.0 || p.wall_u_top[1] != 0.0)) ? 1 : 0;
  q.wetting = (p.walls_z && (p.theta_bottom != 90.0 || p.theta_top != 90.0)) ? 1 : 0;
  q.wall_ext = (q.moving_walls || q.wetting) ? 1 : 0;
  for (int c = 0; c < 2; ++c) {
    q.uw_d[0][c] = p.wall_u_bottom[c];
    q.uw_d[1][c] = p.wall_u_top[c];
    q.uw_f[0][c] = (float)p.wall_u_bottom[c];
    q.uw_f[1][c] = (float)p.wall_u_top[c];
  }
  const double pi = 3.14159265358979323846;
  q.kw_d[0] = p.theta_bottom == 90.0 ? 0.0 : 4.0 / p.xi * std::cos(p.theta_bottom * pi / 180.0);
  q.kw_d[1] = p.theta_top == 90.0 ? 0.0 : 4.0 / p.xi * std::cos(p.theta_top * pi / 180.0);
  q.kw_f[0] = (float)q.kw_d[0];
  q.kw_f[1] = (float)q.kw_d[1];
  q.uniform_rho = p.rho_L == p.rho_H ? 1 : 0;
  q.rho_ratio = q.uniform_rho ? 0 : 1;
  q.uniform_tau = p.nu_L == p.nu_H ? 1 : 0;
  q.four_over_xi_d = 4.0 / p.xi;
  q.twelve_over_xi_d = 12.0 / p.xi;
  q.inv_rho_d = 1.0 / p.rho_L;
  q.omega_g_d = 1.0 / q.pd.tau_L;
  q.four_over_xi_f = (float)q.four_over_xi_d;
  q.twelve_over_xi_f = (float)q.twelve_over_xi_d;
  q.inv_rho_f = (float)q.inv_rho_d;
  q.omega_g_f = 1.0f / q.pf.tau_L;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  }
  return fn;
}

// 4D map (x, y, z, direction) over one padded PDF array of Q directions,
// boxes of box_w x box_rows x 1 x 1 elements.
bool make_map(CUtensorMap* m, void* base, lbm_precision prec, const DevParams& P, int Q, int box_w,
              int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const size_t s = store_bytes(prec);
  const CUtensorMapDataType dt = prec == LBM_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                               : prec == LBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t dims[4] = {(cuuint64_t)P.NXP, (cuuint64_t)P.NYP, (cuuint64_t)P.nz, (cuuint64_t)Q};
  const cuuint64_t strides[3] = {(cuuint64_t)P.NXP * s, (cuuint64_t)P.NXP * P.NYP * s,
                                 (cuuint64_t)P.Np * s};
  const cuuint32_t box[4] = {(cuuint32_t)box_w, (cuuint32_t)box_rows, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, dt, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// In-place layout: maps over the one set, every box the tile's own rows.
bool make_maps_aa(lbm_domain* d) {
  const int w = bulk_box_cols((int)d->prec), rows = bulk_tile_rows((int)d->prec, d->qh, d->qf);
  TMaps& t = d->maps[0];
  if (!make_map(&t.h, at(d, d->L.h[0]), d->prec, d->dp, d->qh, w, rows)) return false;
  if (!make_map(&t.g, at(d, d->L.g[0]), d->prec, d->dp, 27, w, rows)) return false;
  if (d->qf > 0) return make_map(&t.f, at(d, d->L.f[0]), d->prec, d->dp, d->qf, w, rows);
  t.f = t.h;  // unused with an RK energy solver
  return true;
}

bool make_maps(lbm_domain* d) {
  const int w = bulk_box_cols((int)d->prec), rows = bulk_tile_rows((int)d->prec, d->qh, d->qf);
  for (int k = 0; k < 2; ++k) {
    TMaps& t = d->maps[k];
    if (!make_map(&t.h, at(d, d->L.h[k]), d->prec, d->dp, d->qh, w, rows + 2)) return false;
    if (!make_map(&t.g, at(d, d->L.g[k]), d->prec, d->dp, 27, w, rows)) return false;
    if (d->qf > 0) {
      if (!make_map(&t.f, at(d, d->L.f[k]), d->prec, d->dp, d->qf, w, rows + 2)) return false;
    } else {
      t.f = t.h;  // unused with an RK energy solver
    }
  }
  return true;
}

}  // namespace

// ===================================================================== ABI
extern "C" {

void lbm_default_params(lbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nu_L = p->nu_H = 0.1;
  p->rho_L = p->rho_H = 1.0;
  p->mobility = 0.02;
  p->xi = 5.0;
  p->sigma_ref = 5e-3;
  p->sigma_T = -5e-4;
  p->T_ref = 0.0;
  p->alpha_L = p->alpha_H = 0.05;
  p->eps_n = 1e-12;
  p->theta_bottom = p->theta_top = 90.0;
  p->omega_high = 1.0;
  p->cp_L = p->cp_H = 1.0;
}

size_t lbm_workspace_bytes_layout(int nx, int ny, int nz, lbm_precision prec, lbm_thermal thermal,
                                  int q_phase, lbm_layout pdf_layout) {
  Layout L;
  if (pdf_layout != LBM_LAYOUT_TWO_GRID && pdf_layout != LBM_LAYOUT_AA) return 0;
  if (!layout(nx, ny, nz, prec, thermal, q_phase, &L, pdf_layout == LBM_LAYOUT_AA)) return 0;
  return L.total;
}

size_t lbm_workspace_bytes(int nx, int ny, int nz, lbm_precision prec, lbm_thermal thermal,
                           int q_phase) {
  return lbm_workspace_bytes_layout(nx, ny, nz, prec, thermal, q_phase, LBM_LAYOUT_TWO_GRID);
}

lbm_status lbm_create_domain(int nx, int ny, int nz, lbm_precision prec, lbm_thermal thermal,
                             int q_phase, void* stream, void* workspace, size_t workspace_bytes,
                             lbm_domain** out) {
  return lbm_create_domain_layout(nx, ny, nz, prec, thermal, q_phase, LBM_LAYOUT_TWO_GRID, stream, workspace,
                                  workspace_bytes, out);
}

lbm_status lbm_create_domain_layout(int nx, int ny, int nz, lbm_precision prec, lbm_thermal thermal,
                                    int q_phase, lbm_layout pdf_layout, void* stream, void* workspace,
                                    size_t workspace_bytes, lbm_domain** out) {
  g_last_error.clear();
  if (!out) return fail(LBM_ERR_ARG, "out is null");
  *out = nullptr;
  if (pdf_layout != LBM_LAYOUT_TWO_GRID && pdf_layout != LBM_LAYOUT_AA)
    return fail(LBM_ERR_ARG, "unknown PDF layout");
  const bool aa = pdf_layout == LBM_LAYOUT_AA;
  Layout L;
  if (!layout(nx, ny, nz, prec, thermal, q_phase, &L, aa))
    return fail(LBM_ERR_ARG, "invalid lattice size, precision, thermal scheme or q_phase");
  if (workspace && workspace_bytes < L.total)
    return fail(LBM_ERR_OOM, "workspace smaller than lbm_workspace_bytes()");
  if (workspace && ((uintptr_t)workspace & 255))
    return fail(LBM_ERR_ARG, "workspace must be 256-byte aligned");
  lbm_domain* d = new (std::nothrow) lbm_domain();
  if (!d) return fail(LBM_ERR_OOM, "host allocation failed");
  d->nx = nx; d->ny = ny; d->nz = nz;
  d->N = (long long)nx * ny * nz;
  d->prec = prec; d->th = thermal; d->qh = q_phase; d->qf = thermal_q(thermal);
  d->stream = (cudaStream_t)stream;
  d->L = L;
  d->aa = aa;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      sms = 152;
    }
    d->sms = sms;
  }
  // the in-place layout runs its own kernels: on the skewed kernel's tiles
  // where they fit (geo_aa), else on the generic kernel's (geo)
  d->geo = geometry(nx, ny, nz, prec, q_phase, thermal_q(thermal), d->sms, !aa);
  d->diag_nblocks = d->geo.nblocks;
  if (aa) {
    const size_t ab = aa_skew_smem_bytes((int)prec, q_phase, thermal_q(thermal));
    if (bulk_ok(nx, ny, prec, q_phase, thermal_q(thermal)) && ab > 0 && ab <= kMaxDynSmem) {
      d->geo_aa = geometry(nx, ny, nz, prec, q_phase, thermal_q(thermal), d->sms, true);
      d->geo_aa.bulk = 2;
    }
  }
  d->sticky = LBM_OK;
  if (const char* env = std::getenv("LBM_TEST_STALL")) d->test_stall = std::atoi(env) != 0;
  lbm_default_params(&d->params);
  if (workspace) {
    d->ws = (char*)workspace;
    d->ws_bytes = workspace_bytes;
    d->owns_ws = false;
  } else {
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete d;
      return fail(LBM_ERR_OOM, std::string("cudaMalloc of the workspace failed: ") + cudaGetErrorString(e));
    }
    d->ws = (char*)p;
    d->ws_bytes = L.total;
    d->owns_ws = true;
  }
  refresh_devparams(d);
  if (d->geo.bulk && !make_maps(d)) {
    // no tensor-map support: run the generic kernel
    d->geo = geometry(nx, ny, nz, prec, q_phase, thermal_q(thermal), d->sms, false);
    d->diag_nblocks = d->geo.nblocks;
  }
  if (d->geo_aa.bulk && !make_maps_aa(d)) d->geo_aa.bulk = 0;
  {
    const cudaError_t e = cudaMemsetAsync(at(d, L.errflag), 0, sizeof(int), d->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (d->owns_ws) cudaFree(d->ws);
      delete d;
      return fail(LBM_ERR_CUDA, std::string("workspace init failed: ") + cudaGetErrorString(e));
    }
  }
  *out = d;
  return LBM_OK;
}

lbm_status lbm_destroy_domain(lbm_domain* d) {
  if (!d) return fail(LBM_ERR_ARG, "null domain");
  cudaStreamSynchronize(d->stream);
  for (cudaEvent_t e : d->prof_ev) cudaEventDestroy(e);
  if (d->owns_ws) cudaFree(d->ws);
  if (d->staging) cudaFree(d->staging);
  delete d;
  return LBM_OK;
}

lbm_status lbm_set_params(lbm_domain* d, const lbm_params* p) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!p) return fail(LBM_ERR_ARG, "params is null");
  const double vals[] = {p->nu_L, p->nu_H, p->rho_L, p->rho_H, p->mobility, p->xi, p->sigma_ref,
                         p->sigma_T, p->T_ref, p->alpha_L, p->alpha_H, p->gravity[0], p->gravity[1],
                         p->gravity[2], p->T_bottom, p->T_top, p->grad_T[0], p->grad_T[1],
                         p->grad_T[2], p->grad_T_origin[0], p->grad_T_origin[1],
                         p->grad_T_origin[2], p->eps_n, p->omega_high, p->T_bottom_amp, p->cp_L, p->cp_H};
  if (!finite_all(vals, (int)(sizeof(vals) / sizeof(vals[0]))))
    return fail(LBM_ERR_ARG, "non-finite parameter");
  if (p->nu_L <= 0 || p->nu_H <= 0) return fail(LBM_ERR_ARG, "viscosity must be > 0");
  if (p->mobility <= 0) return fail(LBM_ERR_ARG, "mobility must be > 0");
  if (p->xi <= 0) return fail(LBM_ERR_ARG, "interface width must be > 0");
  if (p->alpha_L <= 0 || p->alpha_H <= 0) return fail(LBM_ERR_ARG, "conductivity must be > 0");
  if (p->cp_L <= 0 || p->cp_H <= 0) return fail(LBM_ERR_ARG, "heat capacity must be > 0");
  if (p->rho_L <= 0 || p->rho_H <= 0) return fail(LBM_ERR_ARG, "density must be > 0");
  if (p->eps_n < 0) return fail(LBM_ERR_ARG, "eps_n must be >= 0");
  if (p->T_bottom_waves < 0) return fail(LBM_ERR_ARG, "T_bottom_waves must be >= 0");
  {
    const double w[6] = {p->wall_u_bottom[0], p->wall_u_bottom[1], p->wall_u_top[0], p->wall_u_top[1],
                         p->theta_bottom, p->theta_top};
    if (!finite_all(w, 6)) return fail(LBM_ERR_ARG, "non-finite wall velocity or contact angle");
    if (std::hypot(w[0], w[1]) >= 0.3 || std::hypot(w[2], w[3]) >= 0.3)
      return fail(LBM_ERR_ARG, "wall speed must be < 0.3 (lattice units)");
    if (!(w[4] > 0 && w[4] < 180) || !(w[5] > 0 && w[5] < 180))
      return fail(LBM_ERR_ARG, "contact angle must lie in (0, 180) degrees");
  }
  if (p->omega_high != 1.0)
    return fail(LBM_ERR_UNSUPPORTED, "higher-order central-moment rate != 1 not built");
  d->params = *p;
  d->params_set = true;
  refresh_devparams(d);
  return LBM_OK;
}

lbm_status lbm_set_heat_sources(lbm_domain* d, int n, const lbm_heat_source* src) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (n < 0 || n > LBM_MAX_SOURCES) return fail(LBM_ERR_ARG, "number of heat sources out of range");
  if (n > 0 && !src) return fail(LBM_ERR_ARG, "sources is null");
  for (int k = 0; k < n; ++k) {
    const double v[5] = {src[k].x, src[k].y, src[k].z, src[k].Q, src[k].w};
    if (!finite_all(v, 5) || src[k].w <= 0) return fail(LBM_ERR_ARG, "invalid heat source");
    if (std::isnan(src[k].d)) return fail(LBM_ERR_ARG, "invalid heat source cut-off");
  }
  d->dp.nsrc = n;
  for (int k = 0; k < n; ++k) {
    const double v[6] = {src[k].x, src[k].y, src[k].z, src[k].Q, src[k].w,
                         (src[k].d > 0 && std::isfinite(src[k].d)) ? src[k].d * src[k].d : -1.0};
    for (int j = 0; j < 6; ++j) {
      d->dp.pd.src[k][j] = v[j];
      d->dp.pf.src[k][j] = (float)v[j];
    }
  }
  return LBM_OK;
}

lbm_status lbm_set_heater_patches(lbm_domain* d, int z, int sx, int sy, int n, const int32_t* x0,
                                  const int32_t* y0, const double* intensity) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (n < 0 || n > LBM_MAX_PATCHES) return fail(LBM_ERR_ARG, "number of patches out of range");
  if (n > 0 && (!x0 || !y0 || !intensity)) return fail(LBM_ERR_ARG, "patch arrays are null");
  if (n > 0 && (sx < 1 || sy < 1 || z < 0 || z >= d->nz)) return fail(LBM_ERR_ARG, "invalid patch geometry");
  if (n > 0 && !finite_all(intensity, n)) return fail(LBM_ERR_ARG, "non-finite patch intensity");
  d->dp.npatch = n;
  d->dp.patch_z = z;
  d->dp.patch_sx = sx;
  d->dp.patch_sy = sy;
  for (int k = 0; k < n; ++k) {
    d->dp.px0[k] = x0[k];
    d->dp.py0[k] = y0[k];
    d->dp.pd.pI[k] = intensity[k];
    d->dp.pf.pI[k] = (float)intensity[k];
  }
  return LBM_OK;
}

lbm_status lbm_set_heater_field(lbm_domain* d, const void* q_dev, int dtype) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!q_dev) {
    d->dp.qfield = nullptr;
    d->dp.qfield_f32 = 0;
    return LBM_OK;
  }
  if (dtype != LBM_FP64 && dtype != LBM_FP32) return fail(LBM_ERR_ARG, "heater field dtype must be LBM_FP64 or LBM_FP32");
  const size_t esz = dtype == LBM_FP64 ? sizeof(double) : sizeof(float);
  if (reinterpret_cast<uintptr_t>(q_dev) % esz != 0) return fail(LBM_ERR_ARG, "heater field is not aligned to its element size");
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, q_dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_ERR_ARG, std::string("heater field is not a device pointer: ") + cudaGetErrorString(e));
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(LBM_ERR_ARG, "heater field is not device memory");
  int dev = -1;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return check_cuda(d, e, "cudaGetDevice");
  if (a.device != dev) return fail(LBM_ERR_ARG, "heater field lives on another device");
  d->dp.qfield = q_dev;
  d->dp.qfield_f32 = dtype == LBM_FP32 ? 1 : 0;
  return LBM_OK;
}

lbm_status lbm_init_droplets(lbm_domain* d, int n, const lbm_droplet* drops) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (n < 0 || n > LBM_MAX_DROPLETS) return fail(LBM_ERR_ARG, "number of droplets out of range");
  if (n > 0 && !drops) return fail(LBM_ERR_ARG, "droplets is null");
  std::vector<double> tab((size_t)n * 7);
  for (int k = 0; k < n; ++k) {
    const double v[7] = {drops[k].cx, drops[k].cy, drops[k].cz, drops[k].R,
                         drops[k].ux, drops[k].uy, drops[k].uz};
    if (!finite_all(v, 7) || drops[k].R < 0) return fail(LBM_ERR_ARG, "invalid droplet");
    std::memcpy(&tab[(size_t)k * 7], v, sizeof(v));
  }
  double* dev = (double*)at(d, d->L.drops);
  if (n > 0) {
    s = check_cuda(d, cudaMemcpyAsync(dev, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, d->stream),
                   "droplet upload");
    if (s != LBM_OK) return s;
  }
  d->cur = 0;
  auto go = [&](auto tag) {
    using S = decltype(tag);
    using R = typename Store<S>::R;
    S* h = (S*)at(d, d->L.h[0]);
    S* g = (S*)at(d, d->L.g[0]);
    S* f = (S*)at(d, d->L.f[0]);
    R* T = (R*)at(d, d->L.T);
    auto qf = [&](auto qh_tag) {
      constexpr int QH = decltype(qh_tag)::value;
      switch (d->qf) {
        case 0: launch_init<S, QH, 0>(d->dp, dev, n, h, g, f, T, d->stream); break;
        case 7: launch_init<S, QH, 7>(d->dp, dev, n, h, g, f, T, d->stream); break;
        case 15: launch_init<S, QH, 15>(d->dp, dev, n, h, g, f, T, d->stream); break;
        case 19: launch_init<S, QH, 19>(d->dp, dev, n, h, g, f, T, d->stream); break;
        default: launch_init<S, QH, 27>(d->dp, dev, n, h, g, f, T, d->stream); break;
      }
    };
    if (d->qh == 15) qf(std::integral_constant<int, 15>{});
    else qf(std::integral_constant<int, 27>{});
  };
  if (d->prec == LBM_FP64) go(double{});
  else if (d->prec == LBM_FP32) go(float{});
  else go(__half{});
  ghost_fill(d, 0);
  if (d->aa) {
    // level 0 of the in-place layout: p_i(x) in slot opp(i)
    auto sw = [&](auto tag) {
      using S = decltype(tag);
      launch_aa_swap<S>(d->dp, d->qh, (S*)at(d, d->L.h[0]), d->stream);
      launch_aa_swap<S>(d->dp, 27, (S*)at(d, d->L.g[0]), d->stream);
      if (d->qf > 0) launch_aa_swap<S>(d->dp, d->qf, (S*)at(d, d->L.f[0]), d->stream);
    };
    if (d->prec == LBM_FP64) sw(double{});
    else if (d->prec == LBM_FP32) sw(float{});
    else sw(__half{});
  }
  s = check_launch(d, "init kernel launch");
  if (s != LBM_OK) return s;
  if (n > 0) {
    // the pageable upload above must complete before `tab` goes out of scope
    s = check_cuda(d, cudaStreamSynchronize(d->stream), "init sync");
    if (s != LBM_OK) return s;
  }
  d->inited = true;
  d->level = 0;
  return LBM_OK;
}

lbm_status lbm_step(lbm_domain* d, int nsteps) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
  if (!d->inited) return fail(LBM_ERR_STATE, "lbm_init_droplets (or lbm_set_pdfs) has not been called");
  for (int k = 0; k < nsteps; ++k) {
    s = run_pass(d, MODE_COLLIDE);
    if (s != LBM_OK) return s;
  }
  return LBM_OK;
}

lbm_status lbm_step_diagnostics(lbm_domain* d, int nsteps, lbm_diag* out) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (nsteps < 1 || !out) return fail(LBM_ERR_ARG, "nsteps must be >= 1 and out non-null");
  if (!d->inited) return fail(LBM_ERR_STATE, "domain not initialised");
  s = lbm_step(d, nsteps - 1);
  if (s != LBM_OK) return s;
  const long long level = d->level;
  s = run_pass(d, MODE_COLLIDE | MODE_DIAG);
  if (s != LBM_OK) return s;
  return finish_diag(d, level, out);
}

lbm_status lbm_get_diagnostics(lbm_domain* d, lbm_diag* out) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!out) return fail(LBM_ERR_ARG, "out is null");
  if (!d->inited) return fail(LBM_ERR_STATE, "domain not initialised");
  s = run_pass(d, MODE_DIAG);
  if (s != LBM_OK) return s;
  return finish_diag(d, d->level, out);
}

lbm_status lbm_get_fields(lbm_domain* d, unsigned mask, void* dst, int dst_on_device, int dtype) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!dst) return fail(LBM_ERR_ARG, "dst is null");
  if (mask == 0 || (mask & ~15u)) return fail(LBM_ERR_ARG, "invalid field mask");
  if (dtype != 0 && dtype != 1) return fail(LBM_ERR_ARG, "dtype must be 0 (f64) or 1 (f32)");
  if (!d->inited) return fail(LBM_ERR_STATE, "domain not initialised");
  const int comps = ((mask & 1u) ? 1 : 0) + ((mask & 2u) ? 3 : 0) + ((mask & 4u) ? 1 : 0) + ((mask & 8u) ? 1 : 0);
  const size_t bytes = (size_t)comps * d->N * (dtype == 0 ? 8 : 4);
  void* target = dst;
  if (!dst_on_device) {
    if (d->staging_bytes < bytes) {
      if (d->staging) cudaFree(d->staging);
      d->staging = nullptr;
      d->staging_bytes = 0;
      if (cudaMalloc(&d->staging, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_OOM, "staging allocation failed");
      }
      d->staging_bytes = bytes;
    }
    target = d->staging;
  }
  s = run_pass(d, MODE_MACRO, target, dtype, mask);
  if (s != LBM_OK) return s;
  if (!dst_on_device) {
    s = check_cuda(d, cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, d->stream), "field copy");
    if (s != LBM_OK) return s;
    s = check_cuda(d, cudaStreamSynchronize(d->stream), "field sync");
  }
  return s;
}

static lbm_status pdf_io(lbm_domain* d, int which, double* host, bool to_host) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!host) return fail(LBM_ERR_ARG, "host buffer is null");
  if (which < 0 || which > 3) return fail(LBM_ERR_ARG, "which must be 0..3");
  if (which == 2 && d->qf == 0) return fail(LBM_ERR_ARG, "no thermal PDFs with an RK solver");
  if (which == 3 && d->qf != 0) return fail(LBM_ERR_ARG, "no T field with an LB thermal solver");
  const size_t N = (size_t)d->N;
  if (which == 3) {
    // the T field is dense, in the compute type, not shifted: convert on the host
    void* buf = at(d, d->L.T);
    if (d->prec == LBM_FP64) {
      s = check_cuda(d, cudaMemcpyAsync(to_host ? (void*)host : buf, to_host ? buf : (void*)host, N * 8,
                                        to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice, d->stream),
                     "T copy");
      if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "T sync");
      return s;
    }
    std::vector<float> tmpf(N);
    if (to_host) {
      s = check_cuda(d, cudaMemcpyAsync(tmpf.data(), buf, N * 4, cudaMemcpyDeviceToHost, d->stream), "T copy");
      if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "T sync");
      if (s == LBM_OK)
        for (size_t k = 0; k < N; ++k) host[k] = tmpf[k];
    } else {
      for (size_t k = 0; k < N; ++k) tmpf[k] = (float)host[k];
      s = check_cuda(d, cudaMemcpyAsync(buf, tmpf.data(), N * 4, cudaMemcpyHostToDevice, d->stream), "T copy");
      if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "T sync");
    }
    return s;
  }
  const int Q = which == 0 ? d->qh : (which == 1 ? 27 : d->qf);
  const double shift = which == 0 ? d->dp.pd.shift_h : (which == 2 ? d->dp.pd.shift_f : 0.0);
  void* buf = which == 0 ? at(d, d->L.h[d->cur]) : which == 1 ? at(d, d->L.g[d->cur]) : at(d, d->L.f[d->cur]);
  const size_t bytes = (size_t)Q * N * 8;
  double* tmp = nullptr;
  s = check_cuda(d, cudaMalloc(&tmp, bytes), "conversion buffer");
  if (s != LBM_OK) return s;
  auto conv = [&](auto tag, bool dir) {
    using S = decltype(tag);
    if (d->aa) launch_aa_convert<S>(d->dp, Q, dir, buf, tmp, shift, (int)(d->level & 1), d->stream);
    else launch_pdf_convert<S>(d->dp, Q, dir, buf, tmp, shift, d->stream);
  };
  if (!to_host) s = check_cuda(d, cudaMemcpyAsync(tmp, host, bytes, cudaMemcpyHostToDevice, d->stream), "upload");
  if (s == LBM_OK) {
    if (d->prec == LBM_FP64) conv(double{}, to_host);
    else if (d->prec == LBM_FP32) conv(float{}, to_host);
    else conv(__half{}, to_host);
    s = check_launch(d, "conversion kernel");
  }
  if (s == LBM_OK && !to_host) ghost_fill(d, d->cur);
  if (s == LBM_OK && to_host)
    s = check_cuda(d, cudaMemcpyAsync(host, tmp, bytes, cudaMemcpyDeviceToHost, d->stream), "download");
  if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "conversion sync");
  cudaFree(tmp);
  return s;
}

lbm_status lbm_get_pdfs(lbm_domain* d, int which, double* dst_host) {
  return pdf_io(d, which, dst_host, true);
}

lbm_status lbm_set_pdfs(lbm_domain* d, int which, const double* src_host) {
  lbm_status s = pdf_io(d, which, const_cast<double*>(src_host), false);
  if (s == LBM_OK) d->inited = true;
  return s;
}

// ---------------------------------------------------------------- checkpoint

}  // extern "C"

namespace {

// Header of a saved state: the domain description it belongs to.
struct StateHeader {
  char magic[8];
  int32_t version, nx, ny, nz, prec, thermal, q_phase, pad_;   // pad_: PDF layout (1 = in place)
  int64_t level;
  uint64_t pdf_bytes, field_bytes;
};
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', 'E'};

size_t state_pdf_bytes(const lbm_domain* d) {
  return (size_t)(d->qh + 27 + d->qf) * (size_t)d->dp.Np * store_bytes(d->prec);
}
size_t state_field_bytes(const lbm_domain* d) {
  return d->qf == 0 ? (size_t)d->N * field_bytes(d->prec) : 0;   // T of the RK solvers
}

}  // namespace

extern "C" {

size_t lbm_state_bytes(lbm_domain* d) {
  if (!d) return 0;
  return sizeof(StateHeader) + state_pdf_bytes(d) + state_field_bytes(d);
}

lbm_status lbm_save_state(lbm_domain* d, void* host_buf, size_t bytes) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!host_buf) return fail(LBM_ERR_ARG, "buffer is null");
  if (bytes < lbm_state_bytes(d)) return fail(LBM_ERR_ARG, "buffer smaller than lbm_state_bytes");
  if (!d->inited) return fail(LBM_ERR_STATE, "domain not initialised");
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kStateMagic, 8);
  h.version = 1;
  h.nx = d->nx; h.ny = d->ny; h.nz = d->nz;
  h.prec = (int32_t)d->prec; h.thermal = (int32_t)d->th; h.q_phase = d->qh;
  h.pad_ = d->aa ? 1 : 0;   // PDF layout
  h.level = d->level;
  h.pdf_bytes = state_pdf_bytes(d);
  h.field_bytes = state_field_bytes(d);
  char* out = (char*)host_buf;
  std::memcpy(out, &h, sizeof(h));
  s = check_cuda(d, cudaMemcpyAsync(out + sizeof(h), cur_set_ptr(d), h.pdf_bytes, cudaMemcpyDeviceToHost,
                                    d->stream), "state copy");
  if (s == LBM_OK && h.field_bytes)
    s = check_cuda(d, cudaMemcpyAsync(out + sizeof(h) + h.pdf_bytes, at(d, d->L.T), h.field_bytes,
                                      cudaMemcpyDeviceToHost, d->stream), "state field copy");
  if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "state sync");
  return s;
}

lbm_status lbm_load_state(lbm_domain* d, const void* host_buf, size_t bytes) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!host_buf) return fail(LBM_ERR_ARG, "buffer is null");
  if (bytes < sizeof(StateHeader)) return fail(LBM_ERR_ARG, "buffer too small for a state header");
  StateHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1)
    return fail(LBM_ERR_ARG, "not a saved state (bad magic or version)");
  if (h.nx != d->nx || h.ny != d->ny || h.nz != d->nz || h.prec != (int32_t)d->prec ||
      h.thermal != (int32_t)d->th || h.q_phase != d->qh || h.pad_ != (d->aa ? 1 : 0))
    return fail(LBM_ERR_ARG, "saved state belongs to a domain of another size, precision, stencil or layout");
  if (h.pdf_bytes != state_pdf_bytes(d) || h.field_bytes != state_field_bytes(d) ||
      bytes < lbm_state_bytes(d))
    return fail(LBM_ERR_ARG, "saved state has an unexpected size");
  const char* in = (const char*)host_buf;
  s = check_cuda(d, cudaMemcpyAsync(cur_set_ptr(d), in + sizeof(h), h.pdf_bytes, cudaMemcpyHostToDevice,
                                    d->stream), "state copy");
  if (s == LBM_OK && h.field_bytes)
    s = check_cuda(d, cudaMemcpyAsync(at(d, d->L.T), in + sizeof(h) + h.pdf_bytes, h.field_bytes,
                                      cudaMemcpyHostToDevice, d->stream), "state field copy");
  // pageable source: complete before returning
  if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "state sync");
  if (s != LBM_OK) return s;
  d->level = h.level;
  d->inited = true;
  return LBM_OK;
}

lbm_status lbm_get_level(lbm_domain* d, int64_t* level) {
  if (!d || !level) return fail(LBM_ERR_ARG, "null argument");
  *level = d->level;
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm_domain* d, int timeout_ms) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  cudaEvent_t ev;
  s = check_cuda(d, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
  if (s != LBM_OK) return s;
  s = check_cuda(d, cudaEventRecord(ev, d->stream), "event record");
  const auto t0 = std::chrono::steady_clock::now();
  while (s == LBM_OK) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      s = check_cuda(d, e, "event query");
      break;
    }
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                        std::chrono::steady_clock::now() - t0).count();
    if (timeout_ms >= 0 && ms > timeout_ms) {
      s = fail(LBM_ERR_TIMEOUT, "stream did not finish within the timeout");
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  cudaEventDestroy(ev);
  if (s == LBM_OK) s = check_error_flag(d);
  return s;
}

lbm_status lbm_stencil(int Q, int32_t* c_out, double* w_out) {
  if (Q != 7 && Q != 15 && Q != 19 && Q != 27) return fail(LBM_ERR_ARG, "Q must be 7, 15, 19 or 27");
  for (int i = 0; i < Q; ++i) {
    int c[3];
    double w;
    switch (Q) {
      case 7: c[0] = cx<7>(i); c[1] = cy<7>(i); c[2] = cz<7>(i); w = weight<7>(i); break;
      case 15: c[0] = cx<15>(i); c[1] = cy<15>(i); c[2] = cz<15>(i); w = weight<15>(i); break;
      case 19: c[0] = cx<19>(i); c[1] = cy<19>(i); c[2] = cz<19>(i); w = weight<19>(i); break;
      default: c[0] = cx<27>(i); c[1] = cy<27>(i); c[2] = cz<27>(i); w = weight<27>(i); break;
    }
    if (c_out)
      for (int a = 0; a < 3; ++a) c_out[3 * i + a] = c[a];
    if (w_out) w_out[i] = w;
  }
  return LBM_OK;
}

// ---------------------------------------------------------------- slab halos

lbm_status lbm_set_subdomain(lbm_domain* d, int x_offset, int nx_global) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (nx_global < d->nx) return fail(LBM_ERR_ARG, "nx_global must be >= nx");
  if (d->aa) return fail(LBM_ERR_UNSUPPORTED, "sub-domains are built for the two-grid layout");
  const bool plain = x_offset == 0 && nx_global == d->nx;
  d->dp.sub = plain ? 0 : 1;
  d->dp.sub_x0 = x_offset;
  d->dp.gnx = nx_global;
  return LBM_OK;
}

static size_t halo_pdf_bytes(const lbm_domain* d, int width) {
  return (size_t)(d->qh + 27 + d->qf) * d->nz * d->ny * (size_t)width * store_bytes(d->prec);
}

size_t lbm_halo_bytes(lbm_domain* d, int width) {
  if (!d || width < 1 || width > d->nx) return 0;
  const size_t pdf = (halo_pdf_bytes(d, width) + 15) & ~size_t(15);
  return pdf + (d->qf == 0 ? (size_t)d->nz * d->ny * width * field_bytes(d->prec) : 0);
}

static lbm_status halo_io(lbm_domain* d, int x0, int width, void* buf, bool to_buf) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!buf) return fail(LBM_ERR_ARG, "buffer is null");
  if (width < 1 || x0 < 0 || x0 + width > d->nx) return fail(LBM_ERR_ARG, "columns outside the lattice");
  if (d->aa) return fail(LBM_ERR_UNSUPPORTED, "halo exchange is built for the two-grid layout");
  if (!d->inited) return fail(LBM_ERR_STATE, "domain not initialised");
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, buf) != cudaSuccess ||
      (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail(LBM_ERR_ARG, "halo buffer must be device memory");
  }
  const size_t t_off = (halo_pdf_bytes(d, width) + 15) & ~size_t(15);
  const int nq = d->qh + 27 + d->qf;
  auto go = [&](auto tag) {
    using S = decltype(tag);
    using R = typename Store<S>::R;
    launch_halo_x<S>(d->dp, (S*)cur_set_ptr(d), nq, d->qf == 0 ? (R*)at(d, d->L.T) : nullptr, x0, width, buf,
                     t_off, to_buf, d->stream);
  };
  if (d->prec == LBM_FP64) go(double{});
  else if (d->prec == LBM_FP32) go(float{});
  else go(__half{});
  s = check_launch(d, "halo kernel");
  // the tiled kernels read periodic ghost copies of the edge columns
  if (s == LBM_OK && !to_buf) {
    ghost_fill(d, d->cur);
    s = check_launch(d, "ghost fill");
  }
  return s;
}

lbm_status lbm_pack_halo_x(lbm_domain* d, int x0, int width, void* dst_dev) {
  return halo_io(d, x0, width, dst_dev, true);
}

lbm_status lbm_unpack_halo_x(lbm_domain* d, int x0, int width, const void* src_dev) {
  return halo_io(d, x0, width, const_cast<void*>(src_dev), false);
}

lbm_status lbm_kernel_info(lbm_domain* d, int32_t* info) {
  if (!d || !info) return fail(LBM_ERR_ARG, "null argument");
  const bool tiled_aa = aa_tiled(d);
  const Geometry& g = tiled_aa ? d->geo_aa : d->geo;
  info[0] = d->aa ? (tiled_aa ? 4 : 3) : d->geo.bulk;
  info[1] = (int32_t)g.grid.x;
  info[2] = (int32_t)g.grid.y;
  info[3] = (int32_t)g.grid.z;
  info[4] = g.zchunk;
  info[5] = tiled_aa             ? (int32_t)aa_skew_smem_bytes((int)d->prec, d->qh, d->qf)
            : d->aa              ? 0
            : d->geo.bulk == 2   ? (int32_t)skew_smem_bytes((int)d->prec, d->qh, d->qf)
            : d->geo.bulk == 1   ? (int32_t)bulk_smem_bytes((int)d->prec, d->qh, d->qf)
                                 : 0;
  return LBM_OK;
}

// ---------------------------------------------------------------- adjoint

}  // extern "C"

namespace {

// Device buffers of an adjoint computation (one allocation, released by the caller).
struct AdjBuffers {
  char* base = nullptr;
  double *lam_a = nullptr, *lam_b = nullptr, *lstar = nullptr, *fld = nullptr, *tot = nullptr;
  double *dJdphi = nullptr, *dJdI = nullptr;
  char* sets = nullptr;   // nsets states (checkpoints): padded PDF set, then T (RK)
  size_t set_bytes = 0;   // one state
  size_t pdf_bytes = 0;   // its PDF set
  double* saves = nullptr;  // nsaves x [SAVE_N][N] step intermediates
  size_t save_elems = 0;
  AdjRK rk{};             // RK energy solvers only
};

size_t pdf_set_bytes(const lbm_domain* d) {
  return (size_t)(d->qh + 27 + d->qf) * (size_t)d->dp.Np * sizeof(double);
}

// Slots of the dense adjoint arrays: h, g, then f (LB) or the T field (RK).
size_t adj_slots(const lbm_domain* d) { return (size_t)(d->qh + 27 + (d->qf > 0 ? d->qf : 1)); }

lbm_status adj_alloc(lbm_domain* d, int nsets, int nsaves, AdjBuffers* B) {
  const size_t N = (size_t)d->N, nq = adj_slots(d);
  const bool rk = d->qf == 0;
  B->pdf_bytes = pdf_set_bytes(d);
  B->set_bytes = align256(B->pdf_bytes + (rk ? N * 8 : 0));
  size_t off = 0;
  size_t o_la = off; off = align256(off + nq * N * 8);
  size_t o_lb = off; off = align256(off + nq * N * 8);
  size_t o_ls = off; off = align256(off + nq * N * 8);
  size_t o_fl = off; off = align256(off + 9 * N * 8);
  size_t o_to = off; off = align256(off + 2 * N * 8);
  size_t o_dp = off; off = align256(off + N * 8);
  size_t o_di = off; off = align256(off + LBM_MAX_PATCHES * 8);
  size_t o_rk = off; off = align256(off + (rk ? 13 * N * 8 : 0));   // u 3, psi 3, lk 2, lT 1, lu 3, lq 1
  size_t o_se = off; off = align256(off + (size_t)nsets * B->set_bytes);
  B->save_elems = (size_t)SAVE_N * N;
  size_t o_sv = off; off = align256(off + (size_t)nsaves * B->save_elems * 8);
  if (cudaMalloc(&B->base, off) != cudaSuccess) {
    cudaGetLastError();
    B->base = nullptr;
    return fail(LBM_ERR_OOM, "adjoint: device allocation of checkpoint and adjoint buffers failed");
  }
  B->lam_a = (double*)(B->base + o_la);
  B->lam_b = (double*)(B->base + o_lb);
  B->lstar = (double*)(B->base + o_ls);
  B->fld = (double*)(B->base + o_fl);
  B->tot = (double*)(B->base + o_to);
  B->dJdphi = (double*)(B->base + o_dp);
  B->dJdI = (double*)(B->base + o_di);
  if (rk) {
    double* r = (double*)(B->base + o_rk);
    B->rk.u = r;
    B->rk.psi[0] = r + 3 * N;
    B->rk.psi[1] = r + 4 * N;
    B->rk.psi[2] = r + 5 * N;
    B->rk.lk[0] = r + 6 * N;
    B->rk.lk[1] = r + 7 * N;
    B->rk.lT = r + 8 * N;
    B->rk.lu = r + 9 * N;
    B->rk.lq = r + 12 * N;
  }
  B->sets = B->base + o_se;
  B->saves = (double*)(B->base + o_sv);
  return LBM_OK;
}

char* cur_set(lbm_domain* d) { return d->ws + d->L.h[d->cur]; }

// lam_out = (dPhi/ds)^T lam_in for the step whose intermediates (MODE_SAVE)
// are in 'save'.  Also accumulates dJ/dI from lam_in into B.dJdI if patches.
lbm_status adj_one_step(lbm_domain* d, const double* save, const double* lam_in, double* lam_out,
                        AdjBuffers& B, bool patch_grad, double ncap) {
  AdjPtrs A;
  A.save = save;
  A.lam_in = lam_in;
  A.lstar = B.lstar;
  A.fld = B.fld;
  A.tot = B.tot;
  A.lam_out = lam_out;
  A.ncap = ncap;
  if (d->qf == 0) {
    // RK energy solver: the stage reverse first (it gives the u adjoint of
    // pass A, the T adjoint of pass B2 and the q_T adjoint of the patches)
    adj_rk(d->dp, save, lam_in + (size_t)(d->qh + 27) * (size_t)d->N, B.rk, d->th == LBM_TH_RK4, d->stream);
    if (patch_grad) adj_patch_grad(d->dp, B.rk.lq, B.dJdI, d->qh, 0, d->stream);
  } else if (patch_grad) {
    adj_patch_grad(d->dp, lam_in, B.dJdI, d->qh, d->qf, d->stream);
  }
  adj_cell(d->dp, A, d->qh, d->qf, B.rk.lu, d->stream);
  adj_fields(d->dp, A, d->stream);
  adj_pull(d->dp, A, d->qh, d->qf, B.rk.lT, d->stream);
  return check_launch(d, "adjoint step kernels");
}

lbm_status adj_check(lbm_domain* d) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!d->inited) return fail(LBM_ERR_STATE, "domain not initialised");
  if (d->prec != LBM_FP64 || !adj_supported(d->qh, d->qf))
    return fail(LBM_ERR_UNSUPPORTED, "the adjoint needs FP64 storage");
  if (d->dp.alpha_ratio)
    return fail(LBM_ERR_UNSUPPORTED, "the adjoint is built for a uniform diffusivity (kappa and rho c_p equal in both phases)");
  if (d->dp.rho_ratio)
    return fail(LBM_ERR_UNSUPPORTED, "the adjoint is built for equal densities (rho_L == rho_H)");
  if (d->dp.wall_ext)
    return fail(LBM_ERR_UNSUPPORTED, "the adjoint is built for walls at rest with neutral wetting");
  if (d->aa) return fail(LBM_ERR_UNSUPPORTED, "the adjoint is built for the two-grid layout");
  if (d->dp.sub) return fail(LBM_ERR_UNSUPPORTED, "the adjoint is built for whole lattices");
  if ((long long)d->nx * d->ny >= (1LL << 31))
    return fail(LBM_ERR_UNSUPPORTED, "the adjoint needs nx * ny < 2^31");
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_adjoint_step(lbm_domain* d, const double* lam_in_host, double* lam_out_host, double normal_cap) {
  lbm_status s = adj_check(d);
  if (s != LBM_OK) return s;
  if (!lam_in_host || !lam_out_host) return fail(LBM_ERR_ARG, "null argument");
  AdjBuffers B;
  s = adj_alloc(d, 0, 1, &B);
  if (s != LBM_OK) return s;
  const size_t bytes = adj_slots(d) * (size_t)d->N * 8;
  s = check_cuda(d, cudaMemcpyAsync(B.lam_a, lam_in_host, bytes, cudaMemcpyHostToDevice, d->stream),
                 "adjoint input copy");
  // intermediates of the step from the current state (read-only pass)
  d->save_ptr = B.saves;
  if (s == LBM_OK) s = run_pass(d, MODE_SAVE);
  d->save_ptr = nullptr;
  if (s == LBM_OK) s = adj_one_step(d, B.saves, B.lam_a, B.lam_b, B, false, normal_cap);
  if (s == LBM_OK)
    s = check_cuda(d, cudaMemcpyAsync(lam_out_host, B.lam_b, bytes, cudaMemcpyDeviceToHost, d->stream),
                   "adjoint output copy");
  if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "adjoint sync");
  cudaFree(B.base);
  return s;
}

lbm_status lbm_adjoint_run(lbm_domain* d, int nsteps, int ckpt_every, const double* target, double normal_cap,
                           double* J_out, double* dJdI_host) {
  lbm_status s = adj_check(d);
  if (s != LBM_OK) return s;
  if (nsteps < 1 || ckpt_every < 1 || !target || !J_out || !(normal_cap == normal_cap))
    return fail(LBM_ERR_ARG, "invalid argument");
  if (ckpt_every > nsteps) ckpt_every = nsteps;
  const int K = ckpt_every;
  const int nseg = (nsteps + K - 1) / K;
  AdjBuffers B;
  // sets: nseg checkpoints and the final state; K step-intermediate slots
  s = adj_alloc(d, nseg + 1, K, &B);
  if (s != LBM_OK) return s;
  auto set_ptr = [&](int k) { return B.sets + (size_t)k * B.set_bytes; };
  auto save_slot = [&](int k) { return B.saves + (size_t)k * B.save_elems; };
  char* ckpt0 = set_ptr(0);
  char* final_set = set_ptr(nseg);
  // a state is the current PDF set, and with an RK energy solver the T field
  char* T_field = (char*)at(d, d->L.T);
  auto save_state = [&](char* dst) {
    lbm_status r = check_cuda(d, cudaMemcpyAsync(dst, cur_set(d), B.pdf_bytes, cudaMemcpyDeviceToDevice, d->stream),
                              "adjoint state copy");
    if (r == LBM_OK && d->qf == 0)
      r = check_cuda(d, cudaMemcpyAsync(dst + B.pdf_bytes, T_field, (size_t)d->N * 8, cudaMemcpyDeviceToDevice,
                                        d->stream),
                     "adjoint state copy");
    return r;
  };
  auto restore_state = [&](const char* src) {
    lbm_status r = check_cuda(d, cudaMemcpyAsync(cur_set(d), src, B.pdf_bytes, cudaMemcpyDeviceToDevice, d->stream),
                              "adjoint state copy");
    if (r == LBM_OK && d->qf == 0)
      r = check_cuda(d, cudaMemcpyAsync(T_field, src + B.pdf_bytes, (size_t)d->N * 8, cudaMemcpyDeviceToDevice,
                                        d->stream),
                     "adjoint state copy");
    return r;
  };
  const long long level0 = d->level;
  // forward, checkpoint every K steps
  for (int n = 0; n < nsteps && s == LBM_OK; ++n) {
    if (n % K == 0) s = save_state(ckpt0 + (size_t)(n / K) * B.set_bytes);
    if (s == LBM_OK) s = run_pass(d, MODE_COLLIDE);
  }
  if (s == LBM_OK) s = save_state(final_set);
  lbm_diag dg;
  if (s == LBM_OK) s = lbm_get_diagnostics(d, &dg);
  double J = 0.0;
  if (s == LBM_OK) {
    if (!(dg.mass != 0.0)) s = fail(LBM_ERR_STATE, "adjoint: zero phi mass");
  }
  if (s == LBM_OK) {
    const double c[3] = {dg.mx / dg.mass, dg.my / dg.mass, dg.mz / dg.mass};
    for (int a = 0; a < 3; ++a) J += (c[a] - target[a]) * (c[a] - target[a]);
    adj_centroid_seed(d->dp, dg.mass, c, target, B.dJdphi, d->stream);
    adj_seed(d->dp, B.dJdphi, B.lam_a, d->qh, d->qf, d->stream);
    s = check_launch(d, "adjoint seed");
  }
  if (s == LBM_OK) s = check_cuda(d, cudaMemsetAsync(B.dJdI, 0, LBM_MAX_PATCHES * 8, d->stream), "adjoint memset");
  // backward over the segments, replaying each from its checkpoint; the
  // replayed steps save the intermediates the adjoint steps read
  for (int seg = nseg - 1; seg >= 0 && s == LBM_OK; --seg) {
    const int n0 = seg * K, n1 = std::min(n0 + K, nsteps);
    s = restore_state(ckpt0 + (size_t)seg * B.set_bytes);
    for (int n = n0; n < n1 && s == LBM_OK; ++n) {
      d->save_ptr = save_slot(n - n0);
      // the last step of a segment only needs its intermediates
      s = run_pass(d, n + 1 < n1 ? (MODE_COLLIDE | MODE_SAVE) : MODE_SAVE);
    }
    d->save_ptr = nullptr;
    for (int n = n1 - 1; n >= n0 && s == LBM_OK; --n) {
      s = adj_one_step(d, save_slot(n - n0), B.lam_a, B.lam_b, B, true, normal_cap);
      std::swap(B.lam_a, B.lam_b);
    }
  }
  d->save_ptr = nullptr;
  // leave the domain at the forward result
  if (s == LBM_OK) s = restore_state(final_set);
  if (s == LBM_OK && d->dp.npatch > 0 && dJdI_host)
    s = check_cuda(d, cudaMemcpyAsync(dJdI_host, B.dJdI, (size_t)d->dp.npatch * 8, cudaMemcpyDeviceToHost,
                                      d->stream),
                   "adjoint gradient copy");
  if (s == LBM_OK) s = check_cuda(d, cudaStreamSynchronize(d->stream), "adjoint sync");
  d->level = level0 + nsteps;
  cudaFree(B.base);
  if (s == LBM_OK) *J_out = J;
  return s;
}

lbm_status lbm_profile_steps(lbm_domain* d, int enable) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (enable && d->prof_ev.empty()) {
    d->prof_ev.resize(2 * LBM_MAX_PROFILED);
    for (cudaEvent_t& e : d->prof_ev) {
      s = check_cuda(d, cudaEventCreate(&e), "profiling event creation");
      if (s != LBM_OK) return s;
    }
  }
  d->prof_on = enable != 0;
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_domain* d, double* ms_total, int32_t* launches) {
  lbm_status s = usable(d);
  if (s != LBM_OK) return s;
  if (!ms_total || !launches) return fail(LBM_ERR_ARG, "null argument");
  s = check_cuda(d, cudaStreamSynchronize(d->stream), "profiling sync");
  if (s != LBM_OK) return s;
  double total = 0.0;
  for (int k = 0; k < d->prof_n; ++k) {
    float ms = 0.f;
    s = check_cuda(d, cudaEventElapsedTime(&ms, d->prof_ev[2 * k], d->prof_ev[2 * k + 1]),
                   "profiling event time");
    if (s != LBM_OK) return s;
    total += ms;
  }
  *ms_total = total;
  *launches = d->prof_n;
  d->prof_n = 0;
  return LBM_OK;
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// Record a failure for lbm_last_error from another translation unit.
lbm_status lbm::set_error(lbm_status s, const char* msg) { return fail(s, msg); }

extern "C" {

const char* lbm_version(void) { return "thermocap-lbm-gb300 0.1 (sm_103a)"; }

}  // extern "C"
