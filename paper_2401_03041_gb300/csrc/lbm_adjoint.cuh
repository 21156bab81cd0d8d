// lbm_adjoint.cuh - discrete adjoint of one FP64 time step (thermal LB or
// RK2 / RK4 energy solver).
//
// The paper has no adjoint; this is the exact transpose of the linearisation
// of the FP64 step the generic and bulk kernels compute (Sec. 2.2-2.3, Alg. 1
// sweep order), used for gradients of objectives of the final state with
// respect to the heater-patch intensities.
//
// Notation: s^n = post-collision PDFs of level n (what the arrays store), the
// step s^{n+1} = Phi(s^n; I).  Given lam' = dJ/ds^{n+1} the adjoint step forms
// lam = (dPhi/ds^n)^T lam' in three passes:
//   A  (adj_point_kernel)  per cell x: from the intermediates the forward step
//      saved for x (phi, T, their finite differences, moments of the pulled g;
//      MODE_SAVE of the replayed step), reverse the f, h and g collisions, u,
//      F, F^phi, mu and sigma(T).
//      Writes the direct adjoints of the pulled PDFs (lam*_i(x), without the
//      phi / T terms), the local adjoints of phi and T, and the adjoints of
//      grad phi, lap phi and grad T at x (9 fields).
//   B1 (adj_fields_kernel) per cell y: the transposes of the isotropic D3Q27
//      gradient and Laplacian (wall ghosts: phi mirrored, T = 2 T_w - T),
//      giving the total adjoints of phi(y) and T(y).
//   B2 (adj_pull_kernel)   per cell y and direction j: the transpose of the
//      pull: lam_j(y) = A_j(y + c_j) if y + c_j is a fluid cell, else the
//      bounce-back partner A_jbar(y) (negated for the thermal anti-bounce-back),
//      where A_i(x) = lam*_i(x) + lam_phi(x) (h), lam*_i(x) (g),
//      lam*_i(x) + lam_T(x) (f).
// Adjoint arrays are dense [direction][z][y][x] FP64 (N values per direction,
// h | g | f directions in one block; with an RK energy solver the T field
// takes the place of f, one slot of N values).
//
// RK2 / RK4 (Eq. rk2, Eq. rk4): the energy update T' = T + sum_k b_k K_k with
// K_k = R(psi_k), psi_1 = T, psi_k = T + c_k K_{k-1}, is affine in T given u:
// R(psi) = L_u psi + r_u with L_u psi = -u . D psi + alpha Lap psi (D, Lap the
// 7-point / central or the isotropic operators, wall ghosts 2 T_w - psi).
// Backwards over the stages (adj_rk): lam_K_k = b_k lam_T' + c_{k+1} L^T
// lam_K_{k+1}; the adjoint of T^n is lam_T' + sum_k L^T lam_K_k, of u(x) is
// -sum_k lam_K_k(x) (D psi_k(x) + G), of q_T(x) is sum_k lam_K_k(x).  The stage
// inputs psi_k are recomputed from the saved T^n and u; the u adjoint enters
// pass A, the T adjoint is added in pass B2.
//
// Reverse-mode identities used for the central-moment collision (per axis, a
// unit central moment of order e maps to the 1D basis b_e(c; u) of the
// closed-form collision in lbm_cell.cuh): d b_0 / du = b_1, d b_1 / du = 2 b_2,
// d b_2 / du = 0.
#pragma once

#include "lbm_aux.cuh"

namespace lbm {

enum : int {
  ADJ_PHI = 0, ADJ_T = 1, ADJ_GPX = 2, ADJ_GPY = 3, ADJ_GPZ = 4, ADJ_LP = 5,
  ADJ_GTX = 6, ADJ_GTY = 7, ADJ_GTZ = 8, ADJ_NFIELDS = 9
};

// 1D central-moment basis b_e(c; u), e = 0, 1, 2, c in {0, +1, -1}
__device__ __forceinline__ double bas(int e, int c, double u) {
  if (e == 0) return c == 0 ? 1.0 - u * u : (c > 0 ? 0.5 * (u * u + u) : 0.5 * (u * u - u));
  if (e == 1) return c == 0 ? -2.0 * u : (c > 0 ? u + 0.5 : u - 0.5);
  return c == 0 ? -1.0 : 0.5;
}

// Weighted moments of per-direction adjoints L_i over stencil Q:
// m0 = sum w L, m1 = sum w L c, m2 = sum w L c c (symmetric), summed per
// opposite pair.  The accessor is called once per direction.
struct WMoments {
  double m0, m1[3], xx, yy, zz, xy, xz, yz;
  __device__ __forceinline__ void m2_times(const double* v, double* out) const {
    out[0] = xx * v[0] + xy * v[1] + xz * v[2];
    out[1] = xy * v[0] + yy * v[1] + yz * v[2];
    out[2] = xz * v[0] + yz * v[1] + zz * v[2];
  }
};

template <int Q, class LF>
__device__ __forceinline__ WMoments wmoments(LF lam) {
  WMoments M;
  M.m0 = weight<Q>(0) * lam(std::integral_constant<int, 0>{});
  M.m1[0] = M.m1[1] = M.m1[2] = M.xx = M.yy = M.zz = M.xy = M.xz = M.yz = 0.0;
  static_for<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (pair_first<Q>(i)) {
      constexpr int ex = cx<Q>(i), ey = cy<Q>(i), ez = cz<Q>(i);
      constexpr double w = weight<Q>(i);
      const double a = lam(I), b = lam(std::integral_constant<int, opp<Q>(i)>{});
      const double s = w * (a + b), d = w * (a - b);
      M.m0 += s;
      if constexpr (ex != 0) { M.m1[0] += ex * d; M.xx += s; }
      if constexpr (ey != 0) { M.m1[1] += ey * d; M.yy += s; }
      if constexpr (ez != 0) { M.m1[2] += ez * d; M.zz += s; }
      if constexpr (ex * ey != 0) M.xy += (ex * ey) * s;
      if constexpr (ex * ez != 0) M.xz += (ex * ez) * s;
      if constexpr (ey * ez != 0) M.yz += (ey * ez) * s;
    }
  });
  return M;
}

// Pass A for one cell, from the intermediates the forward step saved for it
// (MODE_SAVE: phi, T, their finite differences and the moments of the pulled
// g, exactly as the step used them).
__device__ __forceinline__ void cell_adjoint_inputs(const DevParams& P, const double* __restrict__ sv,
                                                    size_t cell, double& phi, double& Tc,
                                                    Stencil27<double>& fdv, GMoments<double>& m) {
  const size_t N = (size_t)P.N;
  phi = sv[SAVE_PHI * N + cell];
  Tc = sv[SAVE_T * N + cell];
  fdv.gpx = sv[SAVE_GPX * N + cell];
  fdv.gpy = sv[SAVE_GPY * N + cell];
  fdv.gpz = sv[SAVE_GPZ * N + cell];
  fdv.lp = sv[SAVE_LP * N + cell];
  fdv.gtx = sv[SAVE_GTX * N + cell];
  fdv.gty = sv[SAVE_GTY * N + cell];
  fdv.gtz = sv[SAVE_GTZ * N + cell];
  m.pst = sv[SAVE_PST * N + cell];
  m.jx = sv[SAVE_JX * N + cell];
  m.jy = sv[SAVE_JY * N + cell];
  m.jz = sv[SAVE_JZ * N + cell];
  m.sxx = sv[SAVE_SXX * N + cell];
  m.syy = sv[SAVE_SYY * N + cell];
  m.szz = sv[SAVE_SZZ * N + cell];
  m.sxy = sv[SAVE_SXY * N + cell];
  m.sxz = sv[SAVE_SXZ * N + cell];
  m.syz = sv[SAVE_SYZ * N + cell];
}

// Forward force and velocity of a cell from its saved intermediates (the
// FP64 arithmetic of cell_force / cell_velocity for equal densities).
struct AdjFlow {
  double gTx, gTy, gTz, sigma, beta, kap, dw, mu, g2, tdp, cm, rho, ax, ay, az, ux, uy, uz;
};

__device__ __forceinline__ AdjFlow adj_flow(const DevParams& P, int x, int y, int z, double phi, double Tc,
                                            const Stencil27<double>& fdv, const GMoments<double>& gm) {
  const auto& rp = P.pd;
  AdjFlow w;
  const double gpx = fdv.gpx, gpy = fdv.gpy, gpz = fdv.gpz, lp = fdv.lp;
  const double Gx = rp.grad[0], Gy = rp.grad[1], Gz = rp.grad[2];
  const double Ttot = Tc + Gx * (x + 0.5 - rp.origin[0]) + Gy * (y + 0.5 - rp.origin[1]) +
                      Gz * (z + 0.5 - rp.origin[2]);
  w.gTx = fdv.gtx + Gx; w.gTy = fdv.gty + Gy; w.gTz = fdv.gtz + Gz;
  const double xi = rp.xi;
  w.sigma = rp.sigma_ref + rp.sigma_T * (Ttot - rp.T_ref);
  w.beta = 12.0 * w.sigma / xi;
  w.kap = 1.5 * w.sigma * xi;
  w.dw = phi * (phi - 1.0) * (phi - 0.5);
  w.mu = 4.0 * w.beta * w.dw - w.kap * lp;
  w.g2 = gpx * gpx + gpy * gpy + gpz * gpz;
  w.tdp = w.gTx * gpx + w.gTy * gpy + w.gTz * gpz;
  w.cm = 1.5 * xi * rp.sigma_T;
  w.rho = rp.rho_L + phi * (rp.rho_H - rp.rho_L);
  const double Fx = w.mu * gpx + w.cm * (w.g2 * w.gTx - w.tdp * gpx) + w.rho * rp.gravity[0];
  const double Fy = w.mu * gpy + w.cm * (w.g2 * w.gTy - w.tdp * gpy) + w.rho * rp.gravity[1];
  const double Fz = w.mu * gpz + w.cm * (w.g2 * w.gTz - w.tdp * gpz) + w.rho * rp.gravity[2];
  w.ax = Fx / w.rho; w.ay = Fy / w.rho; w.az = Fz / w.rho;
  w.ux = gm.jx + 0.5 * w.ax; w.uy = gm.jy + 0.5 * w.ay; w.uz = gm.jz + 0.5 * w.az;
  return w;
}

template <int QH, int QF>
__device__ __forceinline__ void cell_adjoint(const DevParams& P, const AdjPtrs& A, int x, int y, int z,
                                             size_t cell, double phi, double Tc,
                                             const Stencil27<double>& fdv, const GMoments<double>& gm,
                                             const double* __restrict__ rk_lu) {
  const auto& rp = P.pd;
  const size_t N = (size_t)P.N;
  constexpr int OG = QH, OF = QH + 27;
  // ---------------- forward quantities (as cell_flow / collide_*, FP64)
  const double gpx = fdv.gpx, gpy = fdv.gpy, gpz = fdv.gpz, lp = fdv.lp;
  const double Gx = rp.grad[0], Gy = rp.grad[1], Gz = rp.grad[2];
  const AdjFlow fw = adj_flow(P, x, y, z, phi, Tc, fdv, gm);
  const double gTx = fw.gTx, gTy = fw.gTy, gTz = fw.gTz;
  const double pst = gm.pst;
  const double sxx = gm.sxx, syy = gm.syy, szz = gm.szz, sxy = gm.sxy, sxz = gm.sxz, syz = gm.syz;
  const double xi = rp.xi;
  const double beta = fw.beta, kap = fw.kap, dw = fw.dw, mu = fw.mu, g2 = fw.g2, tdp = fw.tdp, cm = fw.cm;
  const double rho = fw.rho;
  const double ax = fw.ax, ay = fw.ay, az = fw.az;
  const double ux = fw.ux, uy = fw.uy, uz = fw.uz;
  const double uu = ux * ux + uy * uy + uz * uz;
  const double omg = 1.0 / (rp.tau_L + phi * (rp.tau_H - rp.tau_L));
  const double k1 = 1.0 - omg;
  const double p3 = pst / 3.0;
  const double Bxx = sxx - p3 - ux * ux + ux * ax, Byy = syy - p3 - uy * uy + uy * ay,
               Bzz = szz - p3 - uz * uz + uz * az;
  const double Bxy = sxy - ux * uy + 0.5 * (ux * ay + ax * uy);
  const double Bxz = sxz - ux * uz + 0.5 * (ux * az + ax * uz);
  const double Byz = syz - uy * uz + 0.5 * (uy * az + ay * uz);
  const double Pxx = k1 * Bxx, Pyy = k1 * Byy, Pzz = k1 * Bzz, Pxy = k1 * Bxy, Pxz = k1 * Bxz,
               Pyz = k1 * Byz;
  const double s_n = sqrt(g2);
  const double nrm = 1.0 / (s_n + rp.eps_n);
  const double cphi = 4.0 * phi * (1.0 - phi) / xi;

  // ---------------- reverse
  // Sums over the directions enter only through low moments of the weighted
  // adjoints w_i L_i (M0, M1, M2 below) and, for the central-moment part,
  // through the contractions T(a, b, c) = sum_i L_i X_a(cx) Y_b(cy) Z_c(cz).
  double l_ux = 0, l_uy = 0, l_uz = 0, l_ax = 0, l_ay = 0, l_az = 0;
  double l_phi = 0, l_T = 0, l_pst = 0;
  const double u_[3] = {ux, uy, uz}, a_[3] = {ax, ay, az};
  // f collision: f' = f* - omT (f* - w Tc E) + w (q - u.G), E = 1 - 1.5 uu + 4.5 cu^2 + 3 cu
  if constexpr (QF > 0) {
    const double omT = rp.omega_T;
    const WMoments M = wmoments<QF>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const double L = A.lam_in[(size_t)(OF + i) * N + cell];
      A.lstar[(size_t)(OF + i) * N + cell] = (1.0 - omT) * L;
      return L;
    });
    double Mu[3];
    M.m2_times(u_, Mu);
    l_T += omT * ((1.0 - 1.5 * uu) * M.m0 + 4.5 * (Mu[0] * ux + Mu[1] * uy + Mu[2] * uz) +
                  3.0 * (M.m1[0] * ux + M.m1[1] * uy + M.m1[2] * uz));
    const double k = omT * Tc;
    l_ux += k * (-3.0 * ux * M.m0 + 9.0 * Mu[0] + 3.0 * M.m1[0]) - M.m0 * Gx;
    l_uy += k * (-3.0 * uy * M.m0 + 9.0 * Mu[1] + 3.0 * M.m1[1]) - M.m0 * Gy;
    l_uz += k * (-3.0 * uz * M.m0 + 9.0 * Mu[2] + 3.0 * M.m1[2]) - M.m0 * Gz;
  }
  if constexpr (QF == 0) {
    // RK energy solver: u enters every stage slope K_k (adj_rk)
    l_ux += rk_lu[cell];
    l_uy += rk_lu[N + cell];
    l_uz += rk_lu[2 * N + cell];
  }
  // h collision: h' = h* - om (h* - w phi E) + sc w c.Fphi
  double l_Fpx, l_Fpy, l_Fpz;
  {
    const double om = rp.omega_phi, sc = 1.0 - 0.5 * om;
    const WMoments M = wmoments<QH>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const double L = A.lam_in[(size_t)i * N + cell];
      A.lstar[(size_t)i * N + cell] = (1.0 - om) * L;
      return L;
    });
    double Mu[3];
    M.m2_times(u_, Mu);
    l_phi += om * ((1.0 - 1.5 * uu) * M.m0 + 4.5 * (Mu[0] * ux + Mu[1] * uy + Mu[2] * uz) +
                   3.0 * (M.m1[0] * ux + M.m1[1] * uy + M.m1[2] * uz));
    const double k = om * phi;
    l_ux += k * (-3.0 * ux * M.m0 + 9.0 * Mu[0] + 3.0 * M.m1[0]);
    l_uy += k * (-3.0 * uy * M.m0 + 9.0 * Mu[1] + 3.0 * M.m1[1]);
    l_uz += k * (-3.0 * uz * M.m0 + 9.0 * Mu[2] + 3.0 * M.m1[2]);
    l_Fpx = sc * M.m1[0]; l_Fpy = sc * M.m1[1]; l_Fpz = sc * M.m1[2];
  }
  // g collision: g' = w [p* - 1.5 (uu + ua) + 3 cu + 1.5 ca + 4.5 cu^2 + 4.5 cu ca] + sum_m P_m B_m(c; u)
  double Lg[3][3][3];  // [iz][iy][ix], axis index 0 / 1 / 2 for c = 0 / +1 / -1
  {
    const WMoments M = wmoments<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int ix = cx<27>(i) == 0 ? 0 : (cx<27>(i) > 0 ? 1 : 2);
      constexpr int iy = cy<27>(i) == 0 ? 0 : (cy<27>(i) > 0 ? 1 : 2);
      constexpr int iz = cz<27>(i) == 0 ? 0 : (cz<27>(i) > 0 ? 1 : 2);
      const double L = A.lam_in[(size_t)(OG + i) * N + cell];
      Lg[iz][iy][ix] = L;
      return L;
    });
    double Mu[3], Ma[3];
    M.m2_times(u_, Mu);
    M.m2_times(a_, Ma);
    l_pst += M.m0;
    l_ux += -1.5 * (2.0 * ux + ax) * M.m0 + 3.0 * M.m1[0] + 9.0 * Mu[0] + 4.5 * Ma[0];
    l_uy += -1.5 * (2.0 * uy + ay) * M.m0 + 3.0 * M.m1[1] + 9.0 * Mu[1] + 4.5 * Ma[1];
    l_uz += -1.5 * (2.0 * uz + az) * M.m0 + 3.0 * M.m1[2] + 9.0 * Mu[2] + 4.5 * Ma[2];
    l_ax += -1.5 * ux * M.m0 + 1.5 * M.m1[0] + 4.5 * Mu[0];
    l_ay += -1.5 * uy * M.m0 + 1.5 * M.m1[1] + 4.5 * Mu[1];
    l_az += -1.5 * uz * M.m0 + 1.5 * M.m1[2] + 4.5 * Mu[2];
  }
  // T(a, b, c) by three 1D contractions
  double Xb[3][3], Yb[3][3], Zb[3][3];  // [order][axis index]
#pragma unroll
  for (int e = 0; e < 3; ++e) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int cv = c == 0 ? 0 : (c == 1 ? 1 : -1);
      Xb[e][c] = bas(e, cv, ux);
      Yb[e][c] = bas(e, cv, uy);
      Zb[e][c] = bas(e, cv, uz);
    }
  }
  double Tx[3][3][3];  // [a][iz][iy]
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int iz = 0; iz < 3; ++iz)
#pragma unroll
      for (int iy = 0; iy < 3; ++iy)
        Tx[a][iz][iy] = Lg[iz][iy][0] * Xb[a][0] + Lg[iz][iy][1] * Xb[a][1] + Lg[iz][iy][2] * Xb[a][2];
  double Txy[3][3][3];  // [a][b][iz]
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
      for (int iz = 0; iz < 3; ++iz)
        Txy[a][bb][iz] = Tx[a][iz][0] * Yb[bb][0] + Tx[a][iz][1] * Yb[bb][1] + Tx[a][iz][2] * Yb[bb][2];
  auto T3 = [&](int a, int bb, int c) {
    return Txy[a][bb][0] * Zb[c][0] + Txy[a][bb][1] * Zb[c][1] + Txy[a][bb][2] * Zb[c][2];
  };
  const double lPxx = T3(2, 0, 0), lPyy = T3(0, 2, 0), lPzz = T3(0, 0, 2);
  const double lPxy = T3(1, 1, 0), lPxz = T3(1, 0, 1), lPyz = T3(0, 1, 1);
  const double T120 = T3(1, 2, 0), T102 = T3(1, 0, 2), T210 = T3(2, 1, 0), T201 = T3(2, 0, 1);
  const double T111 = T3(1, 1, 1), T012 = T3(0, 1, 2), T021 = T3(0, 2, 1);
  // d/du of the bases raises the order: d b_0 = b_1, d b_1 = 2 b_2
  l_ux += Pyy * T120 + Pzz * T102 + 2.0 * Pxy * T210 + 2.0 * Pxz * T201 + Pyz * T111;
  l_uy += Pxx * T210 + Pzz * T012 + 2.0 * Pxy * T120 + Pxz * T111 + 2.0 * Pyz * T021;
  l_uz += Pxx * T201 + Pyy * T021 + Pxy * T111 + 2.0 * Pxz * T102 + 2.0 * Pyz * T012;
  // P_m = k1 B_m(s, p*, u, a)
  const double l_k1 = lPxx * Bxx + lPyy * Byy + lPzz * Bzz + lPxy * Bxy + lPxz * Bxz + lPyz * Byz;
  const double l_sxx = k1 * lPxx, l_syy = k1 * lPyy, l_szz = k1 * lPzz;
  const double l_sxy = k1 * lPxy, l_sxz = k1 * lPxz, l_syz = k1 * lPyz;
  l_pst -= (l_sxx + l_syy + l_szz) / 3.0;
  l_ux += l_sxx * (-2.0 * ux + ax) + l_sxy * (-uy + 0.5 * ay) + l_sxz * (-uz + 0.5 * az);
  l_uy += l_syy * (-2.0 * uy + ay) + l_sxy * (-ux + 0.5 * ax) + l_syz * (-uz + 0.5 * az);
  l_uz += l_szz * (-2.0 * uz + az) + l_sxz * (-ux + 0.5 * ax) + l_syz * (-uy + 0.5 * ay);
  l_ax += l_sxx * ux + 0.5 * (l_sxy * uy + l_sxz * uz);
  l_ay += l_syy * uy + 0.5 * (l_sxy * ux + l_syz * uz);
  l_az += l_szz * uz + 0.5 * (l_sxz * ux + l_syz * uy);
  l_phi += l_k1 * omg * omg * (rp.tau_H - rp.tau_L);   // k1 = 1 - 1 / tau(phi)
  // u = j + a / 2
  const double l_jx = l_ux, l_jy = l_uy, l_jz = l_uz;
  l_ax += 0.5 * l_ux; l_ay += 0.5 * l_uy; l_az += 0.5 * l_uz;
  // a = F / rho (rho does not depend on phi: equal densities)
  const double l_Fx = l_ax / rho, l_Fy = l_ay / rho, l_Fz = l_az / rho;
  // F = mu gp + cm (g2 gT - tdp gp)
  const double l_mu = l_Fx * gpx + l_Fy * gpy + l_Fz * gpz;
  const double gTl = gTx * l_Fx + gTy * l_Fy + gTz * l_Fz;
  const double gpl = gpx * l_Fx + gpy * l_Fy + gpz * l_Fz;
  double l_gpx = mu * l_Fx + cm * (2.0 * gpx * gTl - tdp * l_Fx - gTx * gpl);
  double l_gpy = mu * l_Fy + cm * (2.0 * gpy * gTl - tdp * l_Fy - gTy * gpl);
  double l_gpz = mu * l_Fz + cm * (2.0 * gpz * gTl - tdp * l_Fz - gTz * gpl);
  const double l_gTx = cm * (g2 * l_Fx - gpx * gpl);
  const double l_gTy = cm * (g2 * l_Fy - gpy * gpl);
  const double l_gTz = cm * (g2 * l_Fz - gpz * gpl);
  // Fphi = cphi(phi) n, n = gp / (|gp| + eps).  With ncap > 0 the normal is
  // differentiated only where |cphi| <= ncap |gp| (on the equilibrium tanh
  // profile cphi = |gp|): at extrema and saddles of phi and in the far-field
  // tails n is undefined or set by round-off, its exact derivative ~ cphi/|gp|
  // is unbounded, and over long horizons the linearised step grows without
  // bound there while the step itself does not (|n| <= 1).  In those cells n
  // is then held fixed.  ncap <= 0: the exact derivative everywhere.
  const double gpF = gpx * l_Fpx + gpy * l_Fpy + gpz * l_Fpz;
  l_phi += 4.0 * (1.0 - 2.0 * phi) / xi * nrm * gpF;
  if (s_n > 0.0 && (A.ncap <= 0.0 || fabs(cphi) <= A.ncap * s_n)) {
    const double k = cphi * gpF * nrm * nrm / s_n;
    l_gpx += cphi * nrm * l_Fpx - k * gpx;
    l_gpy += cphi * nrm * l_Fpy - k * gpy;
    l_gpz += cphi * nrm * l_Fpz - k * gpz;
  }
  // mu = 4 beta dw(phi) - kappa lap phi, beta and kappa linear in sigma(T)
  l_phi += l_mu * 4.0 * beta * (3.0 * phi * phi - 3.0 * phi + 0.5);
  const double l_lp = -kap * l_mu;
  const double l_sigma = l_mu * (48.0 / xi * dw - 1.5 * xi * lp);
  l_T += rp.sigma_T * l_sigma;
  // moments of g*
  static_for<0, 27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ex = cx<27>(i), ey = cy<27>(i), ez = cz<27>(i);
    A.lstar[(size_t)(OG + i) * N + cell] =
        l_pst + ex * l_jx + ey * l_jy + ez * l_jz + ex * ex * l_sxx + ey * ey * l_syy + ez * ez * l_szz +
        ex * ey * l_sxy + ex * ez * l_sxz + ey * ez * l_syz;
  });
  A.fld[(size_t)ADJ_PHI * N + cell] = l_phi;
  A.fld[(size_t)ADJ_T * N + cell] = l_T;
  A.fld[(size_t)ADJ_GPX * N + cell] = l_gpx;
  A.fld[(size_t)ADJ_GPY * N + cell] = l_gpy;
  A.fld[(size_t)ADJ_GPZ * N + cell] = l_gpz;
  A.fld[(size_t)ADJ_LP * N + cell] = l_lp;
  A.fld[(size_t)ADJ_GTX * N + cell] = l_gTx;
  A.fld[(size_t)ADJ_GTY * N + cell] = l_gTy;
  A.fld[(size_t)ADJ_GTZ * N + cell] = l_gTz;
}

// Pass A: pointwise, from the saved intermediates of the step.  Grid: x over
// the cells of one plane (32-bit index), y = z.
template <int QH, int QF>
__global__ void adj_point_kernel(const DevParams P, const AdjPtrs A, const double* __restrict__ rk_lu) {
  const unsigned plane = (unsigned)P.nx * (unsigned)P.ny;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= plane) return;
  const int y = (int)(r / (unsigned)P.nx), x = (int)(r - (unsigned)y * (unsigned)P.nx);
  const int z = blockIdx.y;
  const size_t cell = (size_t)z * plane + r;
  double phi, Tc;
  Stencil27<double> fd;
  GMoments<double> m;
  cell_adjoint_inputs(P, A.save, cell, phi, Tc, fd, m);
  cell_adjoint<QH, QF>(P, A, x, y, z, cell, phi, Tc, fd, m, rk_lu);
}

// Pass B1: total adjoints of phi and T (stencil transposes).  Grid: x over
// the cells of one plane (32-bit index), y = z.
__global__ void adj_fields_kernel(const DevParams P, const AdjPtrs A) {
  const size_t N = (size_t)P.N;
  const unsigned plane = (unsigned)P.nx * (unsigned)P.ny;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= plane) return;
  const int y = (int)(r / (unsigned)P.nx), x = (int)(r - (unsigned)y * (unsigned)P.nx);
  const int z = blockIdx.y;
  const size_t cell = (size_t)z * plane + r;
  const double* F = A.fld;
  double lphi = F[(size_t)ADJ_PHI * N + cell];
  double lT = F[(size_t)ADJ_T * N + cell];
  // central term of the Laplacian: lap(x) = 6 sum_k w_k (v(x + c_k) - v(x))
  lphi -= 6.0 * (1.0 - weight<27>(0)) * F[(size_t)ADJ_LP * N + cell];
  // x reads v at x + c_k: every (x, k) whose read resolves to this cell
  auto add_from = [&](size_t c, double w, int ex, int ey, int ez, double sgn_T) {
    double gphi = 0.0, gT = 0.0;
    if (ex) { gphi += ex * F[(size_t)ADJ_GPX * N + c]; gT += ex * F[(size_t)ADJ_GTX * N + c]; }
    if (ey) { gphi += ey * F[(size_t)ADJ_GPY * N + c]; gT += ey * F[(size_t)ADJ_GTY * N + c]; }
    if (ez) { gphi += ez * F[(size_t)ADJ_GPZ * N + c]; gT += ez * F[(size_t)ADJ_GTZ * N + c]; }
    lphi += 3.0 * w * gphi + 6.0 * w * F[(size_t)ADJ_LP * N + c];
    lT += sgn_T * 3.0 * w * gT;
  };
  static_for<1, 27>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
    constexpr double w = weight<27>(k);
    const int xs = wrap(x - ex, P.nx), ys = wrap(y - ey, P.ny);
    const int zs = z - ez;
    if (P.walls) {
      if (zs >= 0 && zs < P.nz) add_from(cell_index(P, xs, ys, zs), w, ex, ey, ez, 1.0);
      // wall ghosts: a cell of the boundary layer reading across the wall
      // reads this (same-layer) cell: phi mirrored, T as 2 T_w - T
      if constexpr (ez == -1) {
        if (z == 0) add_from(cell_index(P, xs, ys, 0), w, ex, ey, ez, -1.0);
      }
      if constexpr (ez == 1) {
        if (z == P.nz - 1) add_from(cell_index(P, xs, ys, P.nz - 1), w, ex, ey, ez, -1.0);
      }
    } else {
      add_from(cell_index(P, xs, ys, wrap(zs, P.nz)), w, ex, ey, ez, 1.0);
    }
  });
  A.tot[cell] = lphi;
  A.tot[N + cell] = lT;
}

// Pass B2: transpose of the pull (with bounce-back / anti-bounce-back), one
// thread per cell for all directions.  Grid: x over the cells of one plane
// (32-bit index), y = z.
template <int QH, int QF>
__global__ void adj_pull_kernel(const DevParams P, const AdjPtrs A, const double* __restrict__ rk_lT) {
  const size_t N = (size_t)P.N;
  const unsigned plane = (unsigned)P.nx * (unsigned)P.ny;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= plane) return;
  const int y = (int)(r / (unsigned)P.nx), x = (int)(r - (unsigned)y * (unsigned)P.nx);
  const int z = blockIdx.y;
  const size_t cell = (size_t)z * plane + r;
  const double tphi = A.tot[cell], tT = A.tot[N + cell];
  // set 0: h (+ phi), 1: g, 2: f (+ T, anti-bounce-back)
  auto one = [&](auto SET, auto J) {
    constexpr int set = decltype(SET)::value, j = decltype(J)::value;
    constexpr int Q = set == 0 ? QH : (set == 1 ? 27 : QF);
    constexpr int off = set == 0 ? 0 : (set == 1 ? QH : QH + 27);
    constexpr int ex = cx<Q>(j), ey = cy<Q>(j), ez = cz<Q>(j);
    constexpr int jb = opp<Q>(j);
    int zt = z + ez;
    bool inside = true;
    if (P.walls) inside = zt >= 0 && zt < P.nz;
    else zt = wrap(zt, P.nz);
    double v;
    if (inside) {
      const size_t c = cell_index(P, wrap(x + ex, P.nx), wrap(y + ey, P.ny), zt);
      v = A.lstar[(size_t)(off + j) * N + c];
      if constexpr (set == 0) v += A.tot[c];
      if constexpr (set == 2) v += A.tot[N + c];
    } else {
      v = A.lstar[(size_t)(off + jb) * N + cell];
      if constexpr (set == 0) v += tphi;
      if constexpr (set == 2) v = -(v + tT);
    }
    A.lam_out[(size_t)(off + j) * N + cell] = v;
  };
  static_for<0, QH>([&](auto J) { one(std::integral_constant<int, 0>{}, J); });
  static_for<0, 27>([&](auto J) { one(std::integral_constant<int, 1>{}, J); });
  if constexpr (QF > 0) static_for<0, QF>([&](auto J) { one(std::integral_constant<int, 2>{}, J); });
  else A.lam_out[(size_t)(QH + 27) * N + cell] = tT + rk_lT[cell];   // RK: the T field
}

// Seed lam^N for J(phi^N): dJ/dphi given per cell (dense, N values) -> the
// adjoint of the stored h (pull transpose with bounce-back); g, f (or T): 0.
template <int QH, int QF>
__global__ void adj_seed_kernel(const DevParams P, const double* __restrict__ dJdphi, double* lam) {
  const size_t N = (size_t)P.N;
  constexpr int NQ = QH + 27 + (QF > 0 ? QF : 1);   // RK: one T slot
  const size_t total = (size_t)NQ * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(k / N);
    const size_t cell = k - (size_t)d * N;
    if (d >= QH) {
      lam[k] = 0.0;
      continue;
    }
    const int x = (int)(cell % P.nx);
    const int y = (int)((cell / P.nx) % P.ny);
    const int z = (int)(cell / ((size_t)P.nx * P.ny));
    int zt = z + cz<QH>(d);
    bool inside = true;
    if (P.walls) inside = zt >= 0 && zt < P.nz;
    else zt = wrap(zt, P.nz);
    lam[k] = inside ? dJdphi[cell_index(P, wrap(x + cx<QH>(d), P.nx), wrap(y + cy<QH>(d), P.ny), zt)]
                    : dJdphi[cell];
  }
}

// dJ/dphi(x) of J = |c - t|^2, c = sum phi X / sum phi (cell centres X).
__global__ void adj_centroid_seed_kernel(const DevParams P, double mass, double c0, double c1, double c2,
                                         double t0, double t1, double t2, double* __restrict__ out) {
  const size_t N = (size_t)P.N;
  for (size_t cell = blockIdx.x * (size_t)blockDim.x + threadIdx.x; cell < N;
       cell += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(cell % P.nx);
    const int y = (int)((cell / P.nx) % P.ny);
    const int z = (int)(cell / ((size_t)P.nx * P.ny));
    out[cell] = 2.0 / mass * ((c0 - t0) * (x + 0.5 - c0) + (c1 - t1) * (y + 0.5 - c1) + (c2 - t2) * (z + 0.5 - c2));
  }
}

// dJ/dI_k += sum over the cells of patch k of sum_i w_i lam^{n+1}_{f,i}
// (the intensity enters every f'_i of a patch cell as w_i I_k), or with an
// RK energy solver (QF = 0) of lam_q, the adjoint of q_T over the stages.
// One block per patch, fixed summation order.
template <int QH, int QF>
__global__ void adj_patch_grad_kernel(const DevParams P, const double* __restrict__ lam, double* dJdI) {
  __shared__ double red[256];
  const size_t N = (size_t)P.N;
  const int k = blockIdx.x;
  const int ncell = P.patch_sx * P.patch_sy;
  double s = 0.0;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int x = P.px0[k] + c % P.patch_sx, y = P.py0[k] + c / P.patch_sx;
    if (x < 0 || x >= P.nx || y < 0 || y >= P.ny) continue;
    const size_t cell = cell_index(P, x, y, P.patch_z);
    if constexpr (QF > 0) {
      static_for<0, QF>([&](auto I) {
        constexpr int i = decltype(I)::value;
        s += weight<QF>(i) * lam[(size_t)(QH + 27 + i) * N + cell];
      });
    } else {
      s += lam[cell];
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) dJdI[k] += red[0];
}


// ---------------------------------------------------------------- RK part
// Cell (x, y, z) of a plane-indexed launch (x over nx * ny, y = z); false
// past the plane's end.
__device__ __forceinline__ bool adj_plane_cell(const DevParams& P, int& x, int& y, int& z, size_t& cell) {
  const unsigned plane = (unsigned)P.nx * (unsigned)P.ny;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= plane) return false;
  y = (int)(r / (unsigned)P.nx);
  x = (int)(r - (unsigned)y * (unsigned)P.nx);
  z = blockIdx.y;
  cell = (size_t)z * plane + r;
  return true;
}

// u of every cell from the saved intermediates of the step ([3][N]).
__global__ void adj_rk_velocity_kernel(const DevParams P, const double* __restrict__ save, double* __restrict__ u) {
  int x, y, z;
  size_t cell;
  if (!adj_plane_cell(P, x, y, z, cell)) return;
  double phi, Tc;
  Stencil27<double> fd;
  GMoments<double> m;
  cell_adjoint_inputs(P, save, cell, phi, Tc, fd, m);
  const AdjFlow w = adj_flow(P, x, y, z, phi, Tc, fd, m);
  const size_t N = (size_t)P.N;
  u[cell] = w.ux;
  u[N + cell] = w.uy;
  u[2 * N + cell] = w.uz;
}

// Forward replay of one stage input: out = T + c R(psi) (rk_rhs, no
// conductivity or heat-capacity ratio).
__global__ void adj_rk_replay_kernel(const DevParams P, const double* __restrict__ psi, const double* __restrict__ T,
                                     const double* __restrict__ u, double c, double* __restrict__ out) {
  int x, y, z;
  size_t cell;
  if (!adj_plane_cell(P, x, y, z, cell)) return;
  out[cell] = T[cell] + c * rk_rhs<double>(P, psi, u, nullptr, x, y, z, cell);
}

// Gradient of the stage input at (x, y, z) with R's operator: the central
// difference of the 7-point set, or the isotropic D3Q27 gradient (wall ghosts
// 2 T_w - psi as in rk_rhs).
__device__ __forceinline__ void rk_grad(const DevParams& P, const double* __restrict__ psi, int x, int y, int z,
                                        double& gx, double& gy, double& gz) {
  if (P.rk_iso) {
    gx = gy = gz = 0.0;
    static_for<1, 27>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
      if constexpr (ex > 0 || (ex == 0 && (ey > 0 || (ey == 0 && ez > 0)))) {
        constexpr double w = weight<27>(k);
        const double d = stage_at(P, psi, x, y, z, ex, ey, ez) - stage_at(P, psi, x, y, z, -ex, -ey, -ez);
        if constexpr (ex != 0) gx += ex * w * d;
        if constexpr (ey != 0) gy += ey * w * d;
        if constexpr (ez != 0) gz += ez * w * d;
      }
    });
    gx *= 3.0; gy *= 3.0; gz *= 3.0;
  } else {
    gx = 0.5 * (stage_at(P, psi, x, y, z, 1, 0, 0) - stage_at(P, psi, x, y, z, -1, 0, 0));
    gy = 0.5 * (stage_at(P, psi, x, y, z, 0, 1, 0) - stage_at(P, psi, x, y, z, 0, -1, 0));
    gz = 0.5 * (stage_at(P, psi, x, y, z, 0, 0, 1) - stage_at(P, psi, x, y, z, 0, 0, -1));
  }
}

// One stage of the RK reverse, stages last .. first.  lamK(x) = sK srcK(x) is
// the adjoint of the slope K_k = R(psi_k).  With mu = L^T lamK:
//   next(y) = b_prev lamT'(y) + c_k mu(y)    (adjoint of K_{k-1}; next != null)
//   lT(y) = lamT'(y) + mu(y) on the last stage, lT(y) += mu(y) after it
//   lu(y) (+)= -lamK(y) (D psi_k(y) + G),  lq(y) (+)= lamK(y).
// (L psi)(x) = sum_c a_c(x) psi~(x + c) - alpha l_0 psi(x), a_c(x) = -u(x) . d_c
// + alpha l_c, with psi~ the ghost-resolved read: across a wall the read of
// x + c returns 2 T_w - psi at the same-layer cell, so that cell collects
// -a_c(x).  7-point set: c = +-e, d_c = +-e / 2, l_c = 1, l_0 = 6; isotropic:
// d_c = 3 w_c c, l_c = 6 w_c, l_0 = 6 (1 - w_0).
__global__ void adj_rk_stage_kernel(const DevParams P, const double* __restrict__ srcK, double sK,
                                    const double* __restrict__ psi, const double* __restrict__ u,
                                    const double* __restrict__ lamT, double b_prev, double c_k,
                                    double* __restrict__ next, double* __restrict__ lT, double* __restrict__ lu,
                                    double* __restrict__ lq, int last) {
  int x, y, z;
  size_t cell;
  if (!adj_plane_cell(P, x, y, z, cell)) return;
  const size_t N = (size_t)P.N;
  const double alpha = P.pd.alpha;
  double mu = 0.0;
  // contribution of reader xs at offset (ex, ey, ez) with direction weights
  auto add = [&](size_t xs, double dx_, double dy_, double dz_, double lc, double sgn) {
    const double a = -(u[xs] * dx_ + u[N + xs] * dy_ + u[2 * N + xs] * dz_) + alpha * lc;
    mu += sgn * a * (sK * srcK[xs]);
  };
  auto offset = [&](int ex, int ey, int ez, double dx_, double dy_, double dz_, double lc) {
    const int xs = wrap(x - ex, P.nx), ys = wrap(y - ey, P.ny);
    if (P.walls) {
      const int zs = z - ez;
      if (zs >= 0 && zs < P.nz) add(cell_index(P, xs, ys, zs), dx_, dy_, dz_, lc, 1.0);
      if (ez == -1 && z == 0) add(cell_index(P, xs, ys, 0), dx_, dy_, dz_, lc, -1.0);
      if (ez == 1 && z == P.nz - 1) add(cell_index(P, xs, ys, P.nz - 1), dx_, dy_, dz_, lc, -1.0);
    } else {
      add(cell_index(P, xs, ys, wrap(z - ez, P.nz)), dx_, dy_, dz_, lc, 1.0);
    }
  };
  double l0;
  if (P.rk_iso) {
    static_for<1, 27>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
      constexpr double w = weight<27>(k);
      offset(ex, ey, ez, 3.0 * w * ex, 3.0 * w * ey, 3.0 * w * ez, 6.0 * w);
    });
    l0 = 6.0 * (1.0 - weight<27>(0));
  } else {
    offset(1, 0, 0, 0.5, 0.0, 0.0, 1.0);
    offset(-1, 0, 0, -0.5, 0.0, 0.0, 1.0);
    offset(0, 1, 0, 0.0, 0.5, 0.0, 1.0);
    offset(0, -1, 0, 0.0, -0.5, 0.0, 1.0);
    offset(0, 0, 1, 0.0, 0.0, 0.5, 1.0);
    offset(0, 0, -1, 0.0, 0.0, -0.5, 1.0);
    l0 = 6.0;
  }
  const double lk = sK * srcK[cell];
  mu -= alpha * l0 * lk;
  const double lt = lamT[cell];
  if (next) next[cell] = b_prev * lt + c_k * mu;
  double gx, gy, gz;
  rk_grad(P, psi, x, y, z, gx, gy, gz);
  const auto& rp = P.pd;
  const double dux = -lk * (gx + rp.grad[0]), duy = -lk * (gy + rp.grad[1]), duz = -lk * (gz + rp.grad[2]);
  if (last) {
    lT[cell] = lt + mu;
    lu[cell] = dux;
    lu[N + cell] = duy;
    lu[2 * N + cell] = duz;
    lq[cell] = lk;
  } else {
    lT[cell] += mu;
    lu[cell] += dux;
    lu[N + cell] += duy;
    lu[2 * N + cell] += duz;
    lq[cell] += lk;
  }
}

}  // namespace lbm
