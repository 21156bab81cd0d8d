// lbm_device.cuh - device-side building blocks of the GB300 thermocapillary
// phase-field LBM: lattice tables, storage traits, launch parameter structs.
//
// Lattices (App. B): velocity classes rest / 6 faces / 12 edges / 8 corners,
// in the order rest; +x,-x,+y,-y,+z,-z; the twelve edges; the eight corners.
// D3Q7 = rest + faces (w_0 = 0, w_face = 1/6), D3Q15 = rest + faces + corners,
// D3Q19 = rest + faces + edges, D3Q27 = all.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// Compile-time loop: f(std::integral_constant<int, i>) for i in [B, E).  Every
// direction loop uses it, so lattice velocities and weights are constants by
// construction (no reliance on the unroller).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ----------------------------------------------------------------- lattices
// Direction k of D3Q27 (the superset).  Other stencils index into it.
__host__ __device__ constexpr int q27_cx(int k) {
  constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0,
                         1, -1, 1, -1, 1, -1, -1, 1};
  return t[k];
}
__host__ __device__ constexpr int q27_cy(int k) {
  constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1,
                         1, -1, 1, -1, -1, 1, 1, -1};
  return t[k];
}
__host__ __device__ constexpr int q27_cz(int k) {
  constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1,
                         1, -1, -1, 1, 1, -1, 1, -1};
  return t[k];
}

// Map direction i of stencil Q to its D3Q27 index.
template <int Q>
__host__ __device__ constexpr int to27(int i) {
  return (Q == 15 && i >= 7) ? i + 12 : i;
}
template <int Q> __host__ __device__ constexpr int cx(int i) { return q27_cx(to27<Q>(i)); }
template <int Q> __host__ __device__ constexpr int cy(int i) { return q27_cy(to27<Q>(i)); }
template <int Q> __host__ __device__ constexpr int cz(int i) { return q27_cz(to27<Q>(i)); }

// Opposite direction: same stencil, negated velocity.
template <int Q>
__host__ __device__ constexpr int opp(int i) {
  int r = 0;
  for (int j = 0; j < Q; ++j)
    if (cx<Q>(j) == -cx<Q>(i) && cy<Q>(j) == -cy<Q>(i) && cz<Q>(j) == -cz<Q>(i)) r = j;
  return r;
}

// Weights per velocity class, App. B.
template <int Q>
__host__ __device__ constexpr double weight(int i) {
  const int n = (cx<Q>(i) != 0) + (cy<Q>(i) != 0) + (cz<Q>(i) != 0);
  if (Q == 7) return n == 0 ? 0.0 : 1.0 / 6.0;
  if (Q == 15) return n == 0 ? 16.0 / 72.0 : (n == 1 ? 8.0 / 72.0 : 1.0 / 72.0);
  if (Q == 19) return n == 0 ? 12.0 / 36.0 : (n == 1 ? 2.0 / 36.0 : 1.0 / 36.0);
  return n == 0 ? 64.0 / 216.0 : (n == 1 ? 16.0 / 216.0 : (n == 2 ? 4.0 / 216.0 : 1.0 / 216.0));
}

// ----------------------------------------------------------------- storage
template <class S> struct Store;
template <> struct Store<double> {
  using R = double;
  __device__ __forceinline__ static R ld(const double* p) { return __ldg(p); }
  __device__ __forceinline__ static R ld_s(const double* p) { return *p; }
  __device__ __forceinline__ static void st(double* p, R v) { *p = v; }
};
template <> struct Store<float> {
  using R = float;
  __device__ __forceinline__ static R ld(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static R ld_s(const float* p) { return *p; }
  __device__ __forceinline__ static void st(float* p, R v) { *p = v; }
};
template <> struct Store<__half> {
  using R = float;
  __device__ __forceinline__ static R ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ __forceinline__ static R ld_s(const __half* p) { return __half2float(*p); }
  __device__ __forceinline__ static void st(__half* p, R v) { *p = __float2half_rn(v); }
};

// Step-kernel tile: a CTA of TX x TY threads owns a TX x TY column of cells.
constexpr int TX = 32;
constexpr int TY = 8;

// ----------------------------------------------------------------- params
constexpr int kMaxSources = 64;
constexpr int kMaxPatches = 64;

// Scalar model parameters in one precision.  The kernels read the copy of
// their compute type, so the FP32 path carries no double arithmetic or
// conversions.
template <class R>
struct RealParams {
  R omega_phi, omega_T, tau_L, tau_H;
  R rho_L, rho_H, xi, sigma_ref, sigma_T, T_ref, alpha;
  R gravity[3];
  R T_bottom, T_top;
  R grad[3], origin[3];
  R eps_n;
  R shift_h, shift_f;             // storage shifts (w_i * shift) for h and f
  R src[kMaxSources][6];          // x, y, z, Q, w, d^2 (d^2 < 0: no cut-off)
  R pI[kMaxPatches];
};

// Everything a kernel needs, passed by value (lives in the constant bank).
// PDF arrays are stored with periodic ghost cells: GX columns on each side
// in x and GY rows on each side in y (no ghosts in z), row pitch NXP and NYP
// rows per plane; Np = nz * NYP * NXP elements per direction.  Cell (x, y, z)
// of direction i lives at i * Np + pdf_index(x, y, z).  Fields (T, u, stage
// buffers, outputs) are dense [z][y][x] arrays of N = nx * ny * nz.
constexpr int kGhostRows = 2;

struct DevParams {
  int nx, ny, nz, walls;
  long long N;
  int NXP, NYP, GX, GY;
  long long Np;
  int rk_iso;
  int test_stall;  // test of the timeout path: the bulk kernel's first copy wait runs out
  int qfield_f32;  // element type of qfield: 0 double, 1 float
  const void* qfield;  // caller-owned dense [z][y][x] heat-source density, or null
  int nsrc;
  int npatch, patch_z, patch_sx, patch_sy;
  int px0[kMaxPatches], py0[kMaxPatches];
  RealParams<double> pd;
  RealParams<float> pf;
  // Extensions of the uniform-property model, kept after everything else so
  // that the fields above keep their constant-bank offsets.
  int alpha_ratio;  // alpha_H != alpha_L: alpha(phi) per cell and the grad alpha terms
  int tw_waves;     // k > 0: modulated bottom wall temperature (T_bottom_amp != 0)
  double dalpha_d, T_bottom_amp_d;  // alpha_H - alpha_L; bottom wall modulation amplitude
  float dalpha_f, T_bottom_amp_f;
  // Constants derived once on the host, so that no kernel divides by a
  // parameter: 4/xi, 12/xi, and for uniform density / viscosity (flags set)
  // 1/rho and 1/tau of the g collision.
  int uniform_rho, uniform_tau;
  int rho_ratio;   // rho_H != rho_L: the pressure and viscous correction forces F_p, F_mu
  double four_over_xi_d, twelve_over_xi_d, inv_rho_d, omega_g_d;
  float four_over_xi_f, twelve_over_xi_f, inv_rho_f, omega_g_f;
  // Walls with a tangential velocity or a contact angle other than 90
  // degrees ([0] bottom, [1] top); kw = (4 / xi) cos(theta).  wall_ext
  // selects the extension kernels.
  int wall_ext, moving_walls, wetting;
  double uw_d[2][2], kw_d[2];
  float uw_f[2][2], kw_f[2];
  // Sub-domain (a slab of a larger lattice): local column x is global column
  // (x + sub_x0) mod gnx for every position-dependent term.
  int sub, sub_x0, gnx;
  // Volumetric heat capacity C = rho c_p that varies with phi (rho or c_p
  // unequal in the two phases): kappa_L, kappa_H - kappa_L, rho_L,
  // rho_H - rho_L, c_p,L, c_p,H - c_p,L.  With a constant C the host folds
  // 1 / C into alpha and its slope instead and leaves heat_cap 0.
  int heat_cap;
  double hc_d[6];
  float hc_f[6];
};

// Global column of local column x (positions of sources, patches, the
// background gradient, the modulated wall, droplets, first moments).
__host__ __device__ __forceinline__ int global_x(const DevParams& P, int x) {
  if (!P.sub) return x;
  int g = (x + P.sub_x0) % P.gnx;
  return g < 0 ? g + P.gnx : g;
}

template <class R> __host__ __device__ __forceinline__ const RealParams<R>& RP(const DevParams& P);
template <> __host__ __device__ __forceinline__ const RealParams<double>& RP<double>(const DevParams& P) { return P.pd; }
template <> __host__ __device__ __forceinline__ const RealParams<float>& RP<float>(const DevParams& P) { return P.pf; }

template <class R> __device__ __forceinline__ R dalpha_of(const DevParams& P);
template <> __device__ __forceinline__ double dalpha_of<double>(const DevParams& P) { return P.dalpha_d; }
template <> __device__ __forceinline__ float dalpha_of<float>(const DevParams& P) { return P.dalpha_f; }
template <class R> __device__ __forceinline__ const R* hc_of(const DevParams& P);
template <> __device__ __forceinline__ const double* hc_of<double>(const DevParams& P) { return P.hc_d; }
template <> __device__ __forceinline__ const float* hc_of<float>(const DevParams& P) { return P.hc_f; }
template <class R> struct Derived { R four_over_xi, twelve_over_xi, inv_rho, omega_g; };
template <class R> __device__ __forceinline__ Derived<R> derived(const DevParams& P);
template <> __device__ __forceinline__ Derived<double> derived<double>(const DevParams& P) {
  return {P.four_over_xi_d, P.twelve_over_xi_d, P.inv_rho_d, P.omega_g_d};
}
template <> __device__ __forceinline__ Derived<float> derived<float>(const DevParams& P) {
  return {P.four_over_xi_f, P.twelve_over_xi_f, P.inv_rho_f, P.omega_g_f};
}

template <class R> __device__ __forceinline__ R t_amp_of(const DevParams& P);
template <> __device__ __forceinline__ double t_amp_of<double>(const DevParams& P) { return P.T_bottom_amp_d; }
template <> __device__ __forceinline__ float t_amp_of<float>(const DevParams& P) { return P.T_bottom_amp_f; }

__device__ __forceinline__ double cos_pi(double a) { return cospi(a); }
__device__ __forceinline__ float cos_pi(float a) { return cospif(a); }

// Wall temperature above column x (0 <= x < nx): T_top at the top wall; at
// the bottom T_bottom, plus T_bottom_amp cos(omega (x + 1/2)) with
// omega = 2 pi k / nx when a modulation is set.
template <class R>
__device__ __forceinline__ R wall_T(const DevParams& P, int x, bool bottom) {
  const auto& rp = RP<R>(P);
  if (!bottom) return (R)rp.T_top;
  R t = (R)rp.T_bottom;
  if (P.tw_waves)
    t += t_amp_of<R>(P) * cos_pi((R)(2 * P.tw_waves) * ((R)global_x(P, x) + (R)0.5) / (R)(P.sub ? P.gnx : P.nx));
  return t;
}

// Work assignment of the bulk step kernel's one-dimensional grid.  The
// lattice is bx x by tile columns; each column is cut into nchunk z-chunks of
// zchunk planes (the last may be shorter).  A unit is one (chunk, column)
// pair, numbered chunk-major so that the CTAs of one wave hold neighbouring
// columns at the same planes (their shared halo rows then meet in L2).  The
// first nfull units run whole, one CTA each; every remaining unit is cut into
// npiece z-pieces, one CTA each, so that what would be a partial last wave of
// whole units becomes npiece times as many short pieces spread over all SMs.
struct BulkSched {
  int bx, by, nchunk, zchunk, nfull, npiece;
};

__host__ __device__ __forceinline__ int bulk_sched_units(const BulkSched& s) { return s.bx * s.by * s.nchunk; }
__host__ __device__ __forceinline__ int bulk_sched_blocks(const BulkSched& s) {
  return s.nfull + (bulk_sched_units(s) - s.nfull) * s.npiece;
}

// Tile column (tx, ty) and plane range [z0, z1) of block b.
__host__ __device__ __forceinline__ void bulk_unit(const BulkSched& s, int nz, int b, int& tx, int& ty, int& z0,
                                                   int& z1) {
  const int cols = s.bx * s.by;
  int u, piece = 0;
  if (b < s.nfull) {
    u = b;
  } else {
    const int rem = bulk_sched_units(s) - s.nfull;
    const int r = b - s.nfull;
    piece = r / rem;
    u = s.nfull + r % rem;
  }
  const int c = u / cols, t = u % cols;
  tx = t % s.bx;
  ty = t / s.bx;
  int lo = c * s.zchunk, hi = lo + s.zchunk;
  if (hi > nz) hi = nz;
  if (b >= s.nfull) {
    const int len = hi - lo;
    const int a = lo + (int)((long long)len * piece / s.npiece);
    hi = lo + (int)((long long)len * (piece + 1) / s.npiece);
    lo = a;
  }
  z0 = lo;
  z1 = hi;
}

template <class R> __device__ __forceinline__ R wall_u(const DevParams& P, int top, int c);
template <> __device__ __forceinline__ double wall_u<double>(const DevParams& P, int top, int c) { return P.uw_d[top][c]; }
template <> __device__ __forceinline__ float wall_u<float>(const DevParams& P, int top, int c) { return P.uw_f[top][c]; }
template <class R> __device__ __forceinline__ R wall_k(const DevParams& P, int top);
template <> __device__ __forceinline__ double wall_k<double>(const DevParams& P, int top) { return P.kw_d[top]; }
template <> __device__ __forceinline__ float wall_k<float>(const DevParams& P, int top) { return P.kw_f[top]; }

// Ghost phi beyond a wall with contact angle theta (k = (4 / xi) cos theta,
// a the first fluid cell): the root of g - a = k w (1 - w), w = (a + g) / 2,
// that tends to the mirror g = a as k -> 0, written s = a + g = 4 a / ((1 -
// k/2) + sqrt((1 - k/2)^2 + 2 k a)) so that it has no cancellation.
template <class R>
__device__ __forceinline__ R wet_ghost(R a, R k) {
  const R b = (R)1 - (R)0.5 * k;
  const R d = b * b + (R)2 * k * a;
  const R sum = (R)4 * a / (b + sqrt(d > (R)0 ? d : (R)0));
  return sum - a;
}

// Moving wall: the momentum a population coming off the wall takes, by the
// equilibrium's linear term, 2 w_I (c_I . u_w) / c_s^2 (times phi for h);
// top = 1 for the wall above.
template <int Q, int I, class R>
__device__ __forceinline__ R wall_momentum(const DevParams& P, int top) {
  constexpr R w6 = (R)(6.0 * weight<Q>(I));
  R cu = (R)0;
  if constexpr (cx<Q>(I) != 0) cu = cx<Q>(I) > 0 ? wall_u<R>(P, top, 0) : -wall_u<R>(P, top, 0);
  if constexpr (cy<Q>(I) != 0) cu = cy<Q>(I) > 0 ? cu + wall_u<R>(P, top, 1) : cu - wall_u<R>(P, top, 1);
  return w6 * cu;
}

// Moving wall, thermal anti-bounce-back: the even part of the equilibrium at
// u_w, 1 + (c_I . u_w)^2 / (2 c_s^4) - u_w^2 / (2 c_s^2).
template <int Q, int I, class R>
__device__ __forceinline__ R wall_even(const DevParams& P, int top) {
  const R ux = wall_u<R>(P, top, 0), uy = wall_u<R>(P, top, 1);
  R cu = (R)0;
  if constexpr (cx<Q>(I) != 0) cu = cx<Q>(I) > 0 ? ux : -ux;
  if constexpr (cy<Q>(I) != 0) cu = cy<Q>(I) > 0 ? cu + uy : cu - uy;
  return (R)1 + (R)4.5 * cu * cu - (R)1.5 * (ux * ux + uy * uy);
}

// Kernel modes (bit set).
enum : int { MODE_COLLIDE = 1, MODE_DIAG = 2, MODE_MACRO = 4, MODE_SAVE = 8 };

// Per-cell quantities of a step written in MODE_SAVE (the adjoint's inputs):
// dense [SAVE_N][N] arrays of the compute type.
enum : int {
  SAVE_PHI = 0, SAVE_T, SAVE_GPX, SAVE_GPY, SAVE_GPZ, SAVE_LP, SAVE_GTX, SAVE_GTY, SAVE_GTZ,
  SAVE_PST, SAVE_JX, SAVE_JY, SAVE_JZ, SAVE_SXX, SAVE_SYY, SAVE_SZZ, SAVE_SXY, SAVE_SXZ, SAVE_SYZ, SAVE_N
};

constexpr int kDiagVals = 7;  // mass, heat, kinetic, mx, my, mz, nonfinite count

template <class S, class RF>
struct StepPtrs {
  const S* h_src; S* h_dst;
  const S* g_src; S* g_dst;
  const S* f_src; S* f_dst;
  // RK thermal fields (RF = double in FP64 mode, float otherwise)
  const RF* T; RF* u_out; RF* s1_out; RF* acc_out;
  int rk_acc;                     // RK4: write acc = K1/6
  // macroscopic output (MODE_MACRO): order phi, u(3), p, T, selected by mask
  void* macro_out; int macro_dtype; unsigned macro_mask;
  double* diag_partials;          // [grid blocks][kDiagVals] (MODE_DIAG)
  RF* save;                       // [SAVE_N][N] (MODE_SAVE)
  int* error_flag;                // set to 1 by a CTA whose bounded wait ran out
  // per-direction destination rows (dst + i * N), so a store address is one
  // multiply-add of the cell index onto a constant-bank pointer
  S* hd[27];
  S* gd[27];
  S* fd[27];
  RF* phi_out;                    // RK with a conductivity ratio: phi for stages 2..4
};

// Buffers of one adjoint step (lbm_adjoint.cuh): dense FP64 arrays (N values
// per direction or field).
struct AdjPtrs {
  const double* save;     // intermediates of step n (MODE_SAVE), [SAVE_N][N]
  const double* lam_in;   // lam^{n+1}, dense [(QH + 27 + QF)][N]
  double* lstar;          // lam* (direct parts), dense [(QH + 27 + QF)][N]
  double* fld;            // [9][N]: local adjoints of phi, T, grad phi (3), lap phi, grad T (3)
  double* tot;            // [2][N]: total adjoints of phi and T
  double* lam_out;        // lam^n, dense [(QH + 27 + QF)][N]
  double ncap;            // > 0: interface normal differentiated only where |4 phi (1 - phi) / xi| <= ncap |grad phi|
};

}  // namespace lbm
