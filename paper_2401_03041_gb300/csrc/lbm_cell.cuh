// lbm_cell.cuh - the per-cell part of one time step (a4-a9 of the sweep),
// shared by the generic and the bulk step kernels.
//
// Inputs: the zeroth moments phi and T of the pulled PDFs, their finite
// differences (isotropic D3Q27 gradient and Laplacian), the RK stencil values,
// and accessors returning the pulled PDF values h*_i, g*_i, f*_i as stored
// (h and f shifted by w_i s, g unshifted; wall rules applied).  Outputs:
// post-collision PDFs (stored shifted),
// RK stage-1 fields, optional macroscopic fields and FP64 diagnostics.
//
// Central-moment collision in closed form.  With y = g* - g^eq + S/2 (S the
// Guo source), relaxing each central moment kappa_k at rate w_k gives
// g' = g^eq + S/2 + K(u)^-1 [(1 - w_k) kappa_k(y)].  The zeroth and first
// central moments of y vanish identically (p* = sum g*, u = sum c g* + a/2)
// and orders >= 3 have w_k = 1, so only the six second-order moments survive,
// relaxed with w = 1/tau(phi):
//   Pi_ab = sum g* c_a c_b - p* c_s^2 d_ab - u_a u_b + (u_a a_b + a_a u_b)/2.
// K(u)^-1 is the tensor product of 1D inverse shifts; a unit central moment of
// order e along one axis maps to the populations (c = 0, +1, -1)
//   P0 = {1 - u^2, (u^2 + u)/2, (u^2 - u)/2},  P1 = {-2u, u + 1/2, u - 1/2},
//   P2 = {-1, 1/2, 1/2},
// and (K^-1 Pi)_i = sum over the six moments of P_ex(cx) P_ey(cy) P_ez(cz).
// g^eq + S/2 splits into a part even and a part odd under c -> -c, evaluated
// once per opposite pair.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ size_t cell_index(const DevParams& P, int x, int y, int z) {
  return ((size_t)z * P.ny + y) * P.nx + x;
}

// Element offset of cell (x, y, z) inside one direction of a padded PDF array
// (x in [-GX, nx + GX), y in [-GY, ny + GY) address the ghost cells).
__device__ __forceinline__ size_t pdf_index(const DevParams& P, int x, int y, int z) {
  return ((size_t)z * P.NYP + (y + P.GY)) * P.NXP + (x + P.GX);
}

// Heat source density q_T at cell (x, y, z) (centre (x+1/2, y+1/2, z+1/2)):
// Gaussian sources (Eq. HeatSource, r <= d) plus heater patches (by index)
// plus the caller's per-cell heater field.
template <class R>
__device__ __forceinline__ R heat_source(const DevParams& P, int x, int y, int z) {
  const auto& rp = RP<R>(P);
  R q = 0;
  const int xg = global_x(P, x);
  for (int k = 0; k < P.nsrc; ++k) {
    const R dx = (R)xg + (R)0.5 - (R)rp.src[k][0];
    const R dy = (R)y + (R)0.5 - (R)rp.src[k][1];
    const R dz = (R)z + (R)0.5 - (R)rp.src[k][2];
    const R r2 = dx * dx + dy * dy + dz * dz;
    const R w = (R)rp.src[k][4];
    if (rp.src[k][5] < (R)0 || r2 <= (R)rp.src[k][5]) q += (R)rp.src[k][3] * exp((R)-2 * r2 / (w * w));
  }
  if (P.npatch > 0 && z == P.patch_z) {
    for (int k = 0; k < P.npatch; ++k) {
      if (xg >= P.px0[k] && xg < P.px0[k] + P.patch_sx && y >= P.py0[k] && y < P.py0[k] + P.patch_sy)
        q += (R)rp.pI[k];
    }
  }
  if (P.qfield) {
    const size_t c = cell_index(P, x, y, z);
    q += P.qfield_f32 ? (R)__ldg(static_cast<const float*>(P.qfield) + c)
                      : (R)__ldg(static_cast<const double*>(P.qfield) + c);
  }
  return q;
}

template <class R>
__device__ __forceinline__ R basis_pick(int c, R z, R p, R m) { return c == 0 ? z : (c > 0 ? p : m); }

// Thermal coefficients of a cell (Eq. temperature; Sec. 2.3: kappa and c_p
// linear in phi, rho linear in phi, C = rho c_p): the diffusivity
// alpha = kappa / C, the conduction cross coefficient (kappa_H - kappa_L) / C
// of grad phi . (grad T + G), and C' / C (d C / d phi over C).  With a
// constant C the host has folded 1 / C into alpha and dalpha, and C' = 0.
template <class R>
struct ThermCoef {
  R alpha, dk_C, dC_C;
};

template <class R>
__device__ __forceinline__ ThermCoef<R> therm_coef(const DevParams& P, R phi) {
  if (!P.heat_cap) {
    const auto& rp = RP<R>(P);
    return {(R)rp.alpha + phi * dalpha_of<R>(P), dalpha_of<R>(P), (R)0};
  }
  const R* hc = hc_of<R>(P);
  const R kap = hc[0] + phi * hc[1];
  const R rho = hc[2] + phi * hc[3];
  const R cp = hc[4] + phi * hc[5];
  const R iC = (R)1 / (rho * cp);
  return {kap * iC, hc[1] * iC, (hc[3] * cp + rho * hc[5]) * iC};
}

// c . v for a lattice velocity c with components in {-1, 0, 1} known at
// compile time: only the non-zero components are summed (x * 0 cannot be
// folded away under IEEE rules, so the plain product form costs a multiply
// per zero component); the sum order is x, y, z as in the full product.
template <int EX, int EY, int EZ, class R>
__device__ __forceinline__ R cdot(R vx, R vy, R vz) {
  if constexpr (EX != 0) {
    R s = EX > 0 ? vx : -vx;
    if constexpr (EY != 0) s = EY > 0 ? s + vy : s - vy;
    if constexpr (EZ != 0) s = EZ > 0 ? s + vz : s - vz;
    return s;
  } else if constexpr (EY != 0) {
    R s = EY > 0 ? vy : -vy;
    if constexpr (EZ != 0) s = EZ > 0 ? s + vz : s - vz;
    return s;
  } else if constexpr (EZ != 0) {
    return EZ > 0 ? vz : -vz;
  } else {
    return (R)0;
  }
}

// Where a collision writes its post-collision populations: StdPut stores
// direction i of the cell at dst[i] + pcell (the two-grid layout); another
// policy is a callable put(std::integral_constant<int, i>, value) (the
// in-place AA layout, whose destinations depend on the step's phase).
struct StdPut {};

// Is direction i the first of its opposite pair (first non-zero component > 0)?
template <int Q>
__host__ __device__ constexpr bool pair_first(int i) {
  return cx<Q>(i) > 0 || (cx<Q>(i) == 0 && (cy<Q>(i) > 0 || (cy<Q>(i) == 0 && cz<Q>(i) > 0)));
}

// Finite differences of one plane triple: the isotropic D3Q27 gradient and
// Laplacian of phi and T from three shared-memory planes (row pitch HXv),
// summed over opposite pairs so that uniform fields give exact zeros.
template <class R>
struct Stencil27 {
  R gpx, gpy, gpz, lp, gtx, gty, gtz, lt;
  template <int HXv>
  __device__ __forceinline__ void eval(const R* pm, const R* pc, const R* pp, const R* tm,
                                       const R* tc, const R* tp, int c0) {
    // sum over the 13 opposite pairs (c, -c): gradient from v(c) - v(-c),
    // Laplacian from v(c) + v(-c) - 2 v(0) (exact zeros on uniform fields)
    const R phi = pc[c0], T = tc[c0];
    gpx = gpy = gpz = lp = gtx = gty = gtz = lt = 0;
    static_for<1, 27>([&](auto K) {
      constexpr int k = decltype(K)::value;
      if constexpr (pair_first<27>(k)) {
        constexpr int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
        const R* P_ = ez == 0 ? pc : (ez > 0 ? pp : pm);
        const R* T_ = ez == 0 ? tc : (ez > 0 ? tp : tm);
        const R* Pm = ez == 0 ? pc : (ez > 0 ? pm : pp);
        const R* Tm = ez == 0 ? tc : (ez > 0 ? tm : tp);
        constexpr int o = ey * HXv + ex;
        const R vp = P_[c0 + o], vm = Pm[c0 - o], tp_ = T_[c0 + o], tm_ = Tm[c0 - o];
        constexpr R w = (R)weight<27>(k);
        lp += w * ((vp - phi) + (vm - phi));
        lt += w * ((tp_ - T) + (tm_ - T));
        const R dp = vp - vm, dt = tp_ - tm_;
        if constexpr (ex != 0) { gpx += (R)ex * w * dp; gtx += (R)ex * w * dt; }
        if constexpr (ey != 0) { gpy += (R)ey * w * dp; gty += (R)ey * w * dt; }
        if constexpr (ez != 0) { gpz += (R)ez * w * dp; gtz += (R)ez * w * dt; }
      }
    });
    gpx *= (R)3; gpy *= (R)3; gpz *= (R)3; lp *= (R)6;
    gtx *= (R)3; gty *= (R)3; gtz *= (R)3; lt *= (R)6;
  }
};

// (phi, T) pairs of the bulk kernel's interleaved shared-memory planes.
template <class R> struct PairOf;
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<double> { using type = double2; };

// Stencil27 from interleaved (phi, T) planes.  FP32: both fields at once with
// packed FP32 arithmetic (same per-lane operations and rounding as eval).
template <int HXv>
__device__ __forceinline__ void eval_pairs(Stencil27<float>& fd, const float2* pm, const float2* pc,
                                           const float2* pp, int c0) {
  // Laplacian as sum_k w_k (v(c) + v(-c)) - (sum_k 2 w_k) v(0): one packed
  // add per pair instead of three (uniform fields then give zeros to
  // rounding rather than exactly)
  const float2 c = pc[c0];
  const float2 m1 = make_float2(-1.f, -1.f);
  float2 L = make_float2(0.f, 0.f), Gx = L, Gy = L, Gz = L;
  static_for<1, 27>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if constexpr (pair_first<27>(k)) {
      constexpr int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
      const float2* P_ = ez == 0 ? pc : (ez > 0 ? pp : pm);
      const float2* Pm = ez == 0 ? pc : (ez > 0 ? pm : pp);
      constexpr int o = ey * HXv + ex;
      const float2 vp = P_[c0 + o], vm = Pm[c0 - o];
      constexpr float w = (float)weight<27>(k);
      L = __ffma2_rn(make_float2(w, w), __fadd2_rn(vp, vm), L);
      const float2 d = __ffma2_rn(vm, m1, vp);  // vp - vm
      if constexpr (ex != 0) Gx = __ffma2_rn(make_float2((float)ex * w, (float)ex * w), d, Gx);
      if constexpr (ey != 0) Gy = __ffma2_rn(make_float2((float)ey * w, (float)ey * w), d, Gy);
      if constexpr (ez != 0) Gz = __ffma2_rn(make_float2((float)ez * w, (float)ez * w), d, Gz);
    }
  });
  // sum over the 13 pairs of 2 w_k = 1 - w_0 = 1 - 8/27 = 19/27
  constexpr float w2 = (float)(1.0 - weight<27>(0));
  L = __ffma2_rn(make_float2(-w2, -w2), c, L);
  fd.gpx = 3.f * Gx.x; fd.gpy = 3.f * Gy.x; fd.gpz = 3.f * Gz.x; fd.lp = 6.f * L.x;
  fd.gtx = 3.f * Gx.y; fd.gty = 3.f * Gy.y; fd.gtz = 3.f * Gz.y; fd.lt = 6.f * L.y;
}

template <int HXv>
__device__ __forceinline__ void eval_pairs(Stencil27<double>& fd, const double2* pm, const double2* pc,
                                           const double2* pp, int c0) {
  const double phi = pc[c0].x, T = pc[c0].y;
  fd.gpx = fd.gpy = fd.gpz = fd.lp = fd.gtx = fd.gty = fd.gtz = fd.lt = 0;
  static_for<1, 27>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if constexpr (pair_first<27>(k)) {
      constexpr int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
      const double2* P_ = ez == 0 ? pc : (ez > 0 ? pp : pm);
      const double2* Pm = ez == 0 ? pc : (ez > 0 ? pm : pp);
      constexpr int o = ey * HXv + ex;
      const double2 vp = P_[c0 + o], vm = Pm[c0 - o];
      constexpr double w = weight<27>(k);
      fd.lp += w * ((vp.x - phi) + (vm.x - phi));
      fd.lt += w * ((vp.y - T) + (vm.y - T));
      const double dp = vp.x - vm.x, dt = vp.y - vm.y;
      if constexpr (ex != 0) { fd.gpx += (double)ex * w * dp; fd.gtx += (double)ex * w * dt; }
      if constexpr (ey != 0) { fd.gpy += (double)ey * w * dp; fd.gty += (double)ey * w * dt; }
      if constexpr (ez != 0) { fd.gpz += (double)ez * w * dp; fd.gtz += (double)ez * w * dt; }
    }
  });
  fd.gpx *= 3.0; fd.gpy *= 3.0; fd.gpz *= 3.0; fd.lp *= 6.0;
  fd.gtx *= 3.0; fd.gty *= 3.0; fd.gtz *= 3.0; fd.lt *= 6.0;
}

// RK stage-1 operator values from interleaved (phi, T) planes (T = .y).
template <class P2, class R, int HXv>
__device__ __forceinline__ void rk_std_pairs(const P2* tm, const P2* tc, const P2* tp, int c0, R& gx, R& gy,
                                             R& gz, R& lap) {
  gx = (R)0.5 * (tc[c0 + 1].y - tc[c0 - 1].y);
  gy = (R)0.5 * (tc[c0 + HXv].y - tc[c0 - HXv].y);
  gz = (R)0.5 * (tp[c0].y - tm[c0].y);
  lap = tc[c0 + 1].y + tc[c0 - 1].y + tc[c0 + HXv].y + tc[c0 - HXv].y + tp[c0].y + tm[c0].y - (R)6 * tc[c0].y;
}

// Central gradient of phi (.x) from interleaved (phi, T) planes.
template <class P2, class R, int HXv>
__device__ __forceinline__ void central_phi_pairs(const P2* tm, const P2* tc, const P2* tp, int c0, R& gx, R& gy,
                                                  R& gz) {
  gx = (R)0.5 * (tc[c0 + 1].x - tc[c0 - 1].x);
  gy = (R)0.5 * (tc[c0 + HXv].x - tc[c0 - HXv].x);
  gz = (R)0.5 * (tp[c0].x - tm[c0].x);
}

// RK stage-1 operator values at the cell (7-point Laplacian, central gradient)
template <class R, int HXv>
__device__ __forceinline__ void rk_std(const R* tm, const R* tc, const R* tp, int c0, R& gx, R& gy,
                                       R& gz, R& lap) {
  gx = (R)0.5 * (tc[c0 + 1] - tc[c0 - 1]);
  gy = (R)0.5 * (tc[c0 + HXv] - tc[c0 - HXv]);
  gz = (R)0.5 * (tp[c0] - tm[c0]);
  lap = tc[c0 + 1] + tc[c0 - 1] + tc[c0 + HXv] + tc[c0 - HXv] + tp[c0] + tm[c0] - (R)6 * tc[c0];
}

// ---------------------------------------------------------------- pieces
// The cell update a2-a9 in pieces, so that the bulk kernel can hand the g part
// and the h / f part of one cell to two threads (roles) while the generic
// kernel runs them in sequence (cell_update).

// a2: zeroth, first and second moments of the pulled g, per opposite pair
// (s = g(c) + g(-c) enters even moments, d = g(c) - g(-c) odd ones).
template <class R>
struct GMoments {
  R pst, jx, jy, jz, sxx, syy, szz, sxy, sxz, syz;
};

template <class R, class GG>
__device__ __forceinline__ GMoments<R> g_moments(GG getg) {
  GMoments<R> m;
  m.pst = getg(std::integral_constant<int, 0>{});
  m.jx = m.jy = m.jz = m.sxx = m.syy = m.szz = m.sxy = m.sxz = m.syz = 0;
  static_for<1, 27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (pair_first<27>(i)) {
      const R a_ = getg(I), b_ = getg(std::integral_constant<int, opp<27>(i)>{});
      const R s_ = a_ + b_, d_ = a_ - b_;
      constexpr int ex = cx<27>(i), ey = cy<27>(i), ez = cz<27>(i);
      m.pst += s_;
      if constexpr (ex != 0) { m.jx += (R)ex * d_; m.sxx += s_; }
      if constexpr (ey != 0) { m.jy += (R)ey * d_; m.syy += s_; }
      if constexpr (ez != 0) { m.jz += (R)ez * d_; m.szz += s_; }
      if constexpr (ex * ey != 0) m.sxy += (R)(ex * ey) * s_;
      if constexpr (ex * ez != 0) m.sxz += (R)(ex * ez) * s_;
      if constexpr (ey * ez != 0) m.syz += (R)(ey * ez) * s_;
    }
  });
  return m;
}

// a4-a5: surface-tension and Marangoni force and body force of one cell from
// phi, T and their finite differences, as the acceleration a = F / rho.
// Everything here is known before the moments of the pulled g, so the bulk
// kernel's stencil role computes it alone and hands a to the g role.
template <class R>
struct CellForce {
  R ax, ay, az, rho;
};

// GX: positions may be those of a sub-domain (global_x); the tiled kernels'
// builds without the extensions pass false.
template <class R, bool GX = true>
__device__ __forceinline__ CellForce<R> cell_force(const DevParams& P, int x, int y, int z, R phi, R Tc,
                                                   R gpx, R gpy, R gpz, R lp, R gtx, R gty, R gtz) {
  const auto& rp = RP<R>(P);
  const Derived<R> dv = derived<R>(P);
  const R Gx = (R)rp.grad[0], Gy = (R)rp.grad[1], Gz = (R)rp.grad[2];
  if constexpr (GX) x = global_x(P, x);
  const R Ttot = Tc + Gx * ((R)x + (R)0.5 - (R)rp.origin[0]) + Gy * ((R)y + (R)0.5 - (R)rp.origin[1]) +
                 Gz * ((R)z + (R)0.5 - (R)rp.origin[2]);
  const R gTx = gtx + Gx, gTy = gty + Gy, gTz = gtz + Gz;
  const R xi = (R)rp.xi;
  const R sigma = (R)rp.sigma_ref + (R)rp.sigma_T * (Ttot - (R)rp.T_ref);
  const R beta = sigma * dv.twelve_over_xi;   // 12 sigma / xi
  const R kap = (R)1.5 * sigma * xi;
  const R mu = (R)4 * beta * phi * (phi - (R)1) * (phi - (R)0.5) - kap * lp;
  const R g2 = gpx * gpx + gpy * gpy + gpz * gpz;
  const R tdp = gTx * gpx + gTy * gpy + gTz * gpz;
  const R cm = (R)1.5 * xi * (R)rp.sigma_T;
  CellForce<R> f;
  f.rho = (R)rp.rho_L + phi * (R)(rp.rho_H - rp.rho_L);
  const R Fx = mu * gpx + cm * (g2 * gTx - tdp * gpx) + f.rho * (R)rp.gravity[0];
  const R Fy = mu * gpy + cm * (g2 * gTy - tdp * gpy) + f.rho * (R)rp.gravity[1];
  const R Fz = mu * gpz + cm * (g2 * gTz - tdp * gpz) + f.rho * (R)rp.gravity[2];
  const R irho = P.uniform_rho ? dv.inv_rho : (R)1 / f.rho;
  f.ax = Fx * irho; f.ay = Fy * irho; f.az = Fz * irho;
  return f;
}

// a5 with a density ratio (Sec. 2.2): adds the pressure and viscous
// correction forces of the velocity-based formulation to a = (F_s + F_b) / rho,
//   F_p  = -p* c_s^2 (rho_H - rho_L) grad phi,
//   F_mu = nu (rho_H - rho_L) [grad u + (grad u)^T] . grad phi,
// nu = c_s^2 (tau(phi) - 1/2).  The strain rate is taken from the second
// moments of the pulled g (no finite differences of u): with u0 = j + a0/2,
// a0 = (F_s + F_b + F_p) / rho,
//   Pi_ab = sum_i g*_i c_ia c_ib - p* c_s^2 d_ab - u0_a u0_b + (u0_a a0_b + a0_a u0_b) / 2
// (the non-equilibrium second moment plus half the Guo source's) equals
// -tau c_s^2 (d_a u_b + d_b u_a), so F_mu = -((tau - 1/2) / tau) (rho_H - rho_L) Pi . grad phi.
template <class R>
__device__ __forceinline__ void density_ratio_accel(const DevParams& P, R phi, R gpx, R gpy, R gpz,
                                                    const GMoments<R>& m, CellForce<R>& F) {
  const auto& rp = RP<R>(P);
  const R drho = (R)(rp.rho_H - rp.rho_L);
  const R irho = (R)1 / F.rho;
  const R fp = -m.pst * (R)(1.0 / 3.0) * drho * irho;
  const R a0x = F.ax + fp * gpx, a0y = F.ay + fp * gpy, a0z = F.az + fp * gpz;
  const R ux = m.jx + (R)0.5 * a0x, uy = m.jy + (R)0.5 * a0y, uz = m.jz + (R)0.5 * a0z;
  const R p3 = m.pst * (R)(1.0 / 3.0);
  const R Pxx = m.sxx - p3 - ux * ux + ux * a0x;
  const R Pyy = m.syy - p3 - uy * uy + uy * a0y;
  const R Pzz = m.szz - p3 - uz * uz + uz * a0z;
  const R Pxy = m.sxy - ux * uy + (R)0.5 * (ux * a0y + a0x * uy);
  const R Pxz = m.sxz - ux * uz + (R)0.5 * (ux * a0z + a0x * uz);
  const R Pyz = m.syz - uy * uz + (R)0.5 * (uy * a0z + a0y * uz);
  const R tau = (R)rp.tau_L + phi * (R)(rp.tau_H - rp.tau_L);
  const R coef = -(tau - (R)0.5) / tau * drho * irho;
  F.ax = a0x + coef * (Pxx * gpx + Pxy * gpy + Pxz * gpz);
  F.ay = a0y + coef * (Pxy * gpx + Pyy * gpy + Pyz * gpz);
  F.az = a0z + coef * (Pxz * gpx + Pyz * gpy + Pzz * gpz);
}

// a6: velocity u = j + a/2 (Guo) from the first moment j of the pulled g.
template <class R>
struct CellFlow {
  R ux, uy, uz, ax, ay, az, uu, rho;
};

template <class R>
__device__ __forceinline__ CellFlow<R> cell_velocity(R ax, R ay, R az, R rho, R jx, R jy, R jz) {
  CellFlow<R> f;
  f.ax = ax; f.ay = ay; f.az = az; f.rho = rho;
  f.ux = jx + (R)0.5 * ax; f.uy = jy + (R)0.5 * ay; f.uz = jz + (R)0.5 * az;
  f.uu = f.ux * f.ux + f.uy * f.uy + f.uz * f.uz;
  return f;
}

// a4-a6 in one piece.
template <class R>
__device__ __forceinline__ CellFlow<R> cell_flow(const DevParams& P, int x, int y, int z, R phi, R Tc,
                                                 R gpx, R gpy, R gpz, R lp, R gtx, R gty, R gtz, R jx, R jy,
                                                 R jz) {
  const CellForce<R> F = cell_force<R>(P, x, y, z, phi, Tc, gpx, gpy, gpz, lp, gtx, gty, gtz);
  return cell_velocity<R>(F.ax, F.ay, F.az, F.rho, jx, jy, jz);
}

// Per-thread accumulators of the FP64 diagnostics (a10).  With an FP64
// compute type they are doubles.  With FP32 they are unevaluated sums hi + lo
// of two floats (Knuth's TwoSum for every addition; a product enters with its
// exact rounding error from an FMA), about 48 significant bits, so that the
// FP64 pipe, a small fraction of the FP32 rate on this GPU, is used once per
// thread (flush) instead of for every cell.
template <class R>
struct DiagAcc {
  double s[kDiagVals];
  __device__ __forceinline__ DiagAcc() {
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) s[k] = 0.0;
  }
  __device__ __forceinline__ void add(int k, double v) { s[k] += v; }
  __device__ __forceinline__ void flush(double* out) const {
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) out[k] = s[k];
  }
};

template <>
struct DiagAcc<float> {
  float hi[kDiagVals], lo[kDiagVals];
  __device__ __forceinline__ DiagAcc() {
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) hi[k] = lo[k] = 0.f;
  }
  // the _rn intrinsics keep the compiler from contracting these into FMAs
  __device__ __forceinline__ void add(int k, float v) {
    const float t = __fadd_rn(hi[k], v);
    const float bv = __fsub_rn(t, hi[k]);
    lo[k] = __fadd_rn(lo[k], __fadd_rn(__fsub_rn(hi[k], __fsub_rn(t, bv)), __fsub_rn(v, bv)));
    hi[k] = t;
  }
  __device__ __forceinline__ void add_prod(int k, float a, float b) {
    const float p = __fmul_rn(a, b);
    lo[k] = __fadd_rn(lo[k], fmaf(a, b, -p));
    add(k, p);
  }
  __device__ __forceinline__ void flush(double* out) const {
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) out[k] = (double)hi[k] + (double)lo[k];
  }
};


// a10 diagnostics (FP64 partial sums) and the macroscopic output pass.
template <class S>
__device__ __forceinline__ void cell_outputs(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                             int x, int y, int z, size_t cell, int mode,
                                             typename Store<S>::R phi, typename Store<S>::R Tc,
                                             typename Store<S>::R pst,
                                             const CellFlow<typename Store<S>::R>& f,
                                             DiagAcc<typename Store<S>::R>& dsum) {
  using R = typename Store<S>::R;
  if (mode & MODE_DIAG) {
    if constexpr (std::is_same<R, double>::value) {
      const double dphi = (double)phi;
      dsum.s[0] += dphi;
      dsum.s[1] += (double)Tc;
      dsum.s[2] += 0.5 * (double)f.rho * (double)f.uu;
      dsum.s[3] += dphi * (global_x(P, x) + 0.5);
      dsum.s[4] += dphi * (y + 0.5);
      dsum.s[5] += dphi * (z + 0.5);
      if (!isfinite(dphi) || !isfinite((double)Tc) || !isfinite((double)f.uu)) dsum.s[6] += 1.0;
    } else {
      // cell centres are exact in FP32 below 2^23; 0.5 rho is exact
      dsum.add(0, phi);
      dsum.add(1, Tc);
      dsum.add_prod(2, (R)0.5 * f.rho, f.uu);
      dsum.add_prod(3, phi, (R)global_x(P, x) + (R)0.5);
      dsum.add_prod(4, phi, (R)y + (R)0.5);
      dsum.add_prod(5, phi, (R)z + (R)0.5);
      if (!isfinite(phi) || !isfinite(Tc) || !isfinite(f.uu)) dsum.hi[6] += 1.f;
    }
  }
  if (mode & MODE_MACRO) {
    const double vals[6] = {(double)phi, (double)f.ux, (double)f.uy, (double)f.uz, (double)pst, (double)Tc};
    const unsigned cnt[4] = {1u, 3u, 1u, 1u};
    int slot = 0, v = 0;
    for (int k = 0; k < 4; ++k) {
      if (A.macro_mask & (1u << k)) {
        for (unsigned c = 0; c < cnt[k]; ++c) {
          const size_t at = (size_t)(slot + c) * P.N + cell;
          if (A.macro_dtype == 0) ((double*)A.macro_out)[at] = vals[v + c];
          else ((float*)A.macro_out)[at] = (float)vals[v + c];
        }
        slot += cnt[k];
      }
      v += cnt[k];
    }
  }
}

// a8: g collision (central moments, closed form)
template <class S, class PUT = StdPut>
__device__ __forceinline__ void collide_g(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                          size_t pcell, typename Store<S>::R phi,
                                          const GMoments<typename Store<S>::R>& m,
                                          const CellFlow<typename Store<S>::R>& f, PUT put = PUT{}) {
  using R = typename Store<S>::R;
  const auto& rp = RP<R>(P);
  const R ux = f.ux, uy = f.uy, uz = f.uz, ax = f.ax, ay = f.ay, az = f.az, uu = f.uu;
  const R om = P.uniform_tau ? derived<R>(P).omega_g : (R)1 / ((R)rp.tau_L + phi * (R)(rp.tau_H - rp.tau_L));
  const R k1 = (R)1 - om;
  const R p3 = m.pst * (R)(1.0 / 3.0);
  const R Pxx = k1 * (m.sxx - p3 - ux * ux + ux * ax);
  const R Pyy = k1 * (m.syy - p3 - uy * uy + uy * ay);
  const R Pzz = k1 * (m.szz - p3 - uz * uz + uz * az);
  const R Pxy = k1 * (m.sxy - ux * uy + (R)0.5 * (ux * ay + ax * uy));
  const R Pxz = k1 * (m.sxz - ux * uz + (R)0.5 * (ux * az + ax * uz));
  const R Pyz = k1 * (m.syz - uy * uz + (R)0.5 * (uy * az + ay * uz));
  // per-axis inverse-shift bases
  const R X0z = (R)1 - ux * ux, X0p = (R)0.5 * (ux * ux + ux), X0m = (R)0.5 * (ux * ux - ux);
  const R X1z = (R)-2 * ux, X1p = ux + (R)0.5, X1m = ux - (R)0.5;
  const R Y0z = (R)1 - uy * uy, Y0p = (R)0.5 * (uy * uy + uy), Y0m = (R)0.5 * (uy * uy - uy);
  const R Y1z = (R)-2 * uy, Y1p = uy + (R)0.5, Y1m = uy - (R)0.5;
  const R Z0z = (R)1 - uz * uz, Z0p = (R)0.5 * (uz * uz + uz), Z0m = (R)0.5 * (uz * uz - uz);
  const R Z1z = (R)-2 * uz, Z1p = uz + (R)0.5, Z1m = uz - (R)0.5;
  R A00[3], A10[3], A01[3], A20[3], A02[3], A11[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int zc = c == 0 ? 0 : (c == 1 ? 1 : -1);
    const R p0 = basis_pick(zc, Z0z, Z0p, Z0m);
    const R p1 = basis_pick(zc, Z1z, Z1p, Z1m);
    const R p2 = zc == 0 ? (R)-1 : (R)0.5;
    A00[c] = p2 * Pzz; A10[c] = p1 * Pxz; A01[c] = p1 * Pyz;
    A20[c] = p0 * Pxx; A02[c] = p0 * Pyy; A11[c] = p0 * Pxy;
  }
  const R ua = ux * ax + uy * ay + uz * az;
  const R base = m.pst - (R)1.5 * (uu + ua);
  const R u3x = (R)3 * ux, u3y = (R)3 * uy, u3z = (R)3 * uz;
  const R a15x = (R)1.5 * ax, a15y = (R)1.5 * ay, a15z = (R)1.5 * az;
  auto neq_of = [&](int ex, int ey, int ez) -> R {
    const int c = ez == 0 ? 0 : (ez > 0 ? 1 : 2);
    const R q0 = basis_pick(ey, Y0z, Y0p, Y0m);
    const R q1 = basis_pick(ey, Y1z, Y1p, Y1m);
    const R q2 = ey == 0 ? (R)-1 : (R)0.5;
    const R B0 = q0 * A00[c] + q1 * A01[c] + q2 * A02[c];
    const R B1 = q0 * A10[c] + q1 * A11[c];
    const R B2 = q0 * A20[c];
    const R r0 = basis_pick(ex, X0z, X0p, X0m);
    const R r1 = basis_pick(ex, X1z, X1p, X1m);
    const R r2 = ex == 0 ? (R)-1 : (R)0.5;
    return r0 * B0 + r1 * B1 + r2 * B2;
  };
  auto out = [&](auto I, R v) {
    if constexpr (std::is_same<PUT, StdPut>::value) Store<S>::st(A.gd[decltype(I)::value] + pcell, v);
    else put(I, v);
  };
  out(std::integral_constant<int, 0>{}, (R)weight<27>(0) * base + neq_of(0, 0, 0));
  static_for<1, 27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (pair_first<27>(i)) {
      constexpr int ex = cx<27>(i), ey = cy<27>(i), ez = cz<27>(i);
      constexpr R w = (R)weight<27>(i);
      // g^eq + S/2 = w [p* + 3cu + 9/2 cu^2 - 3/2 uu + 3/2 (ca - ua) + 9/2 cu ca]
      //            = w [(base + (3cu / 2)(3cu + 3ca)) +- (3cu + 3ca / 2)]
      const R cu3 = cdot<ex, ey, ez>(u3x, u3y, u3z);
      const R ca15 = cdot<ex, ey, ez>(a15x, a15y, a15z);
      const R odd = cu3 + ca15;
      const R even = (R)0.5 * cu3 * (odd + ca15) + base;
      out(I, w * (even + odd) + neq_of(ex, ey, ez));
      out(std::integral_constant<int, opp<27>(i)>{}, w * (even - odd) + neq_of(-ex, -ey, -ez));
    }
  });
}

// a7: h collision (single rate + Guo source of the interface force).
// geth(I) returns the pulled population as STORED, hs_i = h*_i - w_i s
// (s = shift_h, 0 in FP64).  With h^eq_i = w_i phi E_i the relaxation
//   h'_i - w_i s = hs_i - omega (hs_i - w_i (phi E_i - s)) + S_i
// works on stored values throughout, so the shift costs nothing per
// direction.
template <class S, int QH, class GH, class PUT = StdPut>
__device__ __forceinline__ void collide_h(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                          size_t pcell, typename Store<S>::R phi, typename Store<S>::R gpx,
                                          typename Store<S>::R gpy, typename Store<S>::R gpz,
                                          const CellFlow<typename Store<S>::R>& f, GH geth, PUT put = PUT{}) {
  using R = typename Store<S>::R;
  const auto& rp = RP<R>(P);
  const R ux = f.ux, uy = f.uy, uz = f.uz, uu = f.uu;
  const R g2 = gpx * gpx + gpy * gpy + gpz * gpz;
  const R nrm = (R)1 / (sqrt(g2) + (R)rp.eps_n);
  const R th = derived<R>(P).four_over_xi * phi * ((R)1 - phi) * nrm;   // 4 phi (1 - phi) / xi / |grad phi|
  const R fpx = th * gpx, fpy = th * gpy, fpz = th * gpz;
  const R om = (R)rp.omega_phi;
  const R sc = (R)1 - (R)0.5 * om;
  const R sh = (R)rp.shift_h;
  const R base = phi * ((R)1 - (R)1.5 * uu) - sh;   // phi e0 - s
  const R p45 = (R)4.5 * phi, p3 = (R)3 * phi;
  auto out = [&](auto I, R v) {
    if constexpr (std::is_same<PUT, StdPut>::value) Store<S>::st(A.hd[decltype(I)::value] + pcell, v);
    else put(I, v);
  };
  {
    constexpr R w = (R)weight<QH>(0);
    const R hs = geth(std::integral_constant<int, 0>{});
    out(std::integral_constant<int, 0>{}, hs - om * (hs - w * base));
  }
  static_for<1, QH>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (pair_first<QH>(i)) {
      constexpr int j = opp<QH>(i);
      constexpr R w = (R)weight<QH>(i);
      const R cu = cdot<cx<QH>(i), cy<QH>(i), cz<QH>(i)>(ux, uy, uz);
      const R cf = cdot<cx<QH>(i), cy<QH>(i), cz<QH>(i)>(fpx, fpy, fpz);
      const R even = w * (base + p45 * cu * cu);
      const R odd = w * (p3 * cu);
      const R src = sc * w * cf;
      const R hi = geth(I), hj = geth(std::integral_constant<int, j>{});
      out(I, hi - om * (hi - (even + odd)) + src);
      out(std::integral_constant<int, j>{}, hj - om * (hj - (even - odd)) - src);
    }
  });
}

// a9 / a9': thermal LB collision, or RK stage 1 (QF = 0).  With a
// conductivity or heat-capacity ratio the LB relaxes at the cell's own rate
// 1 / (1/2 + alpha(phi) / c_s^2), which recovers div(alpha grad T); Eq.
// temperature asks for alpha lap T + (grad kappa / C) . (grad T + G), so the
// source adds (grad kappa / C) . G and (grad kappa / C - grad alpha) . grad T
// = alpha (C' / C) grad phi . grad T (isotropic grad T).  RK stage 1 takes
// alpha(phi) lap T plus the whole (grad kappa / C) . (grad T + G), with
// grad phi from its own operator (pgx.. central differences for the 7-point
// set, the isotropic gradient otherwise).  RATIO = P.alpha_ratio, resolved by
// the caller so that the uniform-property path carries none of it.
template <class S, int QF, bool RATIO, class GF, class PUT = StdPut>
__device__ __forceinline__ void collide_f(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                          int x, int y, int z, size_t cell, size_t pcell,
                                          typename Store<S>::R phi, typename Store<S>::R Tc,
                                          const Stencil27<typename Store<S>::R>& fdv,
                                          typename Store<S>::R rgx, typename Store<S>::R rgy,
                                          typename Store<S>::R rgz, typename Store<S>::R rlap,
                                          typename Store<S>::R pgx, typename Store<S>::R pgy,
                                          typename Store<S>::R pgz,
                                          const CellFlow<typename Store<S>::R>& f, GF getf, PUT put = PUT{}) {
  using R = typename Store<S>::R;
  const auto& rp = RP<R>(P);
  const R ux = f.ux, uy = f.uy, uz = f.uz, uu = f.uu;
  const R Gx = (R)rp.grad[0], Gy = (R)rp.grad[1], Gz = (R)rp.grad[2];
  auto out = [&](auto I, R v) {
    if constexpr (std::is_same<PUT, StdPut>::value) Store<S>::st(A.fd[decltype(I)::value] + pcell, v);
    else put(I, v);
  };
  const R q = heat_source<R>(P, x, y, z);
  const R uG = ux * Gx + uy * Gy + uz * Gz;
  if constexpr (QF > 0) {
    R om = (R)rp.omega_T;
    R qs = q - uG;
    if constexpr (RATIO) {
      const ThermCoef<R> tc = therm_coef<R>(P, phi);
      om = (R)1 / ((R)0.5 + (R)3 * tc.alpha);
      qs += tc.dk_C * (fdv.gpx * Gx + fdv.gpy * Gy + fdv.gpz * Gz);
      if (P.heat_cap) qs += tc.alpha * tc.dC_C * (fdv.gpx * fdv.gtx + fdv.gpy * fdv.gty + fdv.gpz * fdv.gtz);
    }
    // stored values throughout, as in collide_h (s = shift_f)
    const R sf = (R)rp.shift_f;
    const R base = Tc * ((R)1 - (R)1.5 * uu) - sf;   // T e0 - s
    const R t45 = (R)4.5 * Tc, t3 = (R)3 * Tc;
    if constexpr (weight<QF>(0) != 0.0) {
      constexpr R w = (R)weight<QF>(0);
      const R fs = getf(std::integral_constant<int, 0>{});
      out(std::integral_constant<int, 0>{}, fs - om * (fs - w * base) + w * qs);
    } else {
      // D3Q7 (w_0 = 0): the rest population relaxes to 0
      const R fs = getf(std::integral_constant<int, 0>{});
      out(std::integral_constant<int, 0>{}, fs - om * fs);
    }
    static_for<1, QF>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (pair_first<QF>(i)) {
        constexpr int j = opp<QF>(i);
        constexpr R w = (R)weight<QF>(i);
        const R cu = cdot<cx<QF>(i), cy<QF>(i), cz<QF>(i)>(ux, uy, uz);
        const R even = w * (base + t45 * cu * cu);
        const R odd = w * (t3 * cu);
        const R wq = w * qs;
        const R fi = getf(I), fj = getf(std::integral_constant<int, j>{});
        out(I, fi - om * (fi - (even + odd)) + wq);
        out(std::integral_constant<int, j>{}, fj - om * (fj - (even - odd)) + wq);
      }
    });
  } else {
    // RK stage 1: K1 = R(T^n) with the local u of this step
    R gx_, gy_, gz_, lap;
    if (P.rk_iso) {
      gx_ = fdv.gtx; gy_ = fdv.gty; gz_ = fdv.gtz; lap = fdv.lt;
    } else {
      gx_ = rgx; gy_ = rgy; gz_ = rgz; lap = rlap;
    }
    R K1 = -(ux * (gx_ + Gx) + uy * (gy_ + Gy) + uz * (gz_ + Gz)) + (R)rp.alpha * lap + q;
    if constexpr (RATIO) {
      const ThermCoef<R> tc = therm_coef<R>(P, phi);
      K1 = -(ux * (gx_ + Gx) + uy * (gy_ + Gy) + uz * (gz_ + Gz)) + tc.alpha * lap + q;
      K1 += P.rk_iso ? tc.dk_C * (fdv.gpx * (gx_ + Gx) + fdv.gpy * (gy_ + Gy) + fdv.gpz * (gz_ + Gz))
                     : tc.dk_C * (pgx * (gx_ + Gx) + pgy * (gy_ + Gy) + pgz * (gz_ + Gz));
      A.phi_out[cell] = phi;
    }
    A.u_out[cell] = ux;
    A.u_out[P.N + cell] = uy;
    A.u_out[2 * P.N + cell] = uz;
    A.s1_out[cell] = Tc + (R)0.5 * K1;
    if (A.rk_acc) A.acc_out[cell] = K1 * (R)(1.0 / 6.0);
  }
}

// MODE_SAVE: the stencil part (phi, T and their finite differences) and the
// g-moment part of one cell's intermediates.
template <class S>
__device__ __forceinline__ void save_stencil(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                             size_t cell, typename Store<S>::R phi, typename Store<S>::R Tc,
                                             const Stencil27<typename Store<S>::R>& fdv) {
  const size_t N = (size_t)P.N;
  A.save[SAVE_PHI * N + cell] = phi;
  A.save[SAVE_T * N + cell] = Tc;
  A.save[SAVE_GPX * N + cell] = fdv.gpx;
  A.save[SAVE_GPY * N + cell] = fdv.gpy;
  A.save[SAVE_GPZ * N + cell] = fdv.gpz;
  A.save[SAVE_LP * N + cell] = fdv.lp;
  A.save[SAVE_GTX * N + cell] = fdv.gtx;
  A.save[SAVE_GTY * N + cell] = fdv.gty;
  A.save[SAVE_GTZ * N + cell] = fdv.gtz;
}

template <class S>
__device__ __forceinline__ void save_moments(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                             size_t cell, const GMoments<typename Store<S>::R>& m) {
  const size_t N = (size_t)P.N;
  A.save[SAVE_PST * N + cell] = m.pst;
  A.save[SAVE_JX * N + cell] = m.jx;
  A.save[SAVE_JY * N + cell] = m.jy;
  A.save[SAVE_JZ * N + cell] = m.jz;
  A.save[SAVE_SXX * N + cell] = m.sxx;
  A.save[SAVE_SYY * N + cell] = m.syy;
  A.save[SAVE_SZZ * N + cell] = m.szz;
  A.save[SAVE_SXY * N + cell] = m.sxy;
  A.save[SAVE_SXZ * N + cell] = m.sxz;
  A.save[SAVE_SYZ * N + cell] = m.syz;
}

// a2-a10 for one cell in sequence.  GH/GG/GF: accessors i -> pulled value
// as stored (h and f shifted by w_i s; g unshifted).
template <class S, int QH, int QF, class GH, class GG, class GF>
__device__ __forceinline__ void cell_update(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                            int x, int y, int z, size_t cell, size_t pcell, int mode,
                                            typename Store<S>::R phi, typename Store<S>::R Tc,
                                            const Stencil27<typename Store<S>::R>& fdv,
                                            typename Store<S>::R rgx, typename Store<S>::R rgy,
                                            typename Store<S>::R rgz, typename Store<S>::R rlap,
                                            typename Store<S>::R pgx, typename Store<S>::R pgy,
                                            typename Store<S>::R pgz, GH geth, GG getg, GF getf,
                                            DiagAcc<typename Store<S>::R>& dsum) {
  using R = typename Store<S>::R;
  const GMoments<R> m = g_moments<R>(getg);
  if (mode & MODE_SAVE) {
    save_stencil<S>(P, A, cell, phi, Tc, fdv);
    save_moments<S>(P, A, cell, m);
  }
  CellForce<R> F = cell_force<R>(P, x, y, z, phi, Tc, fdv.gpx, fdv.gpy, fdv.gpz, fdv.lp, fdv.gtx, fdv.gty, fdv.gtz);
  if (P.rho_ratio) density_ratio_accel<R>(P, phi, fdv.gpx, fdv.gpy, fdv.gpz, m, F);
  const CellFlow<R> f = cell_velocity<R>(F.ax, F.ay, F.az, F.rho, m.jx, m.jy, m.jz);
  cell_outputs<S>(P, A, x, y, z, cell, mode, phi, Tc, m.pst, f, dsum);
  if (!(mode & MODE_COLLIDE)) return;
  collide_g<S>(P, A, pcell, phi, m, f);
  collide_h<S, QH>(P, A, pcell, phi, fdv.gpx, fdv.gpy, fdv.gpz, f, geth);
  if (P.alpha_ratio) collide_f<S, QF, true>(P, A, x, y, z, cell, pcell, phi, Tc, fdv, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
  else collide_f<S, QF, false>(P, A, x, y, z, cell, pcell, phi, Tc, fdv, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
}

}  // namespace lbm
