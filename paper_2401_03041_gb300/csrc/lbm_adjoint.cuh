// lbm_adjoint.cuh - discrete adjoint of one FP64 time step (LB thermal).
//
// The paper has no adjoint; this is the exact transpose of the linearisation
// of the FP64 step the generic and bulk kernels compute (Sec. 2.2-2.3, Alg. 1
// sweep order), used for gradients of objectives of the final state with
// respect to the heater-patch intensities.
//
// Notation: s^n = post-collision PDFs of level n (what the arrays store), the
// step s^{n+1} = Phi(s^n; I).  Given lam' = dJ/ds^{n+1} the adjoint step forms
// lam = (dPhi/ds^n)^T lam' in three passes:
//   A  (adj_cell_kernel)   per cell x: recompute the forward quantities of x
//      from s^n (pulled PDFs, phi and T on the halo, finite differences), then
//      reverse the f, h and g collisions, u, F, F^phi, mu and sigma(T).
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
// h | g | f directions in one block); the forward state is a padded PDF set.
//
// Reverse-mode identities used for the central-moment collision (per axis, a
// unit central moment of order e maps to the 1D basis b_e(c; u) of the
// closed-form collision in lbm_cell.cuh): d b_0 / du = b_1, d b_1 / du = 2 b_2,
// d b_2 / du = 0.
#pragma once

#include "lbm_step.cuh"

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

// Pass A for one cell.  h*, g*, f* accessors return pulled FP64 values.
template <int QH, int QF, class GG>
__device__ __forceinline__ void cell_adjoint(const DevParams& P, const AdjPtrs& A, int x, int y, int z,
                                             size_t cell, double phi, double Tc,
                                             const Stencil27<double>& fdv, GG getg) {
  const auto& rp = P.pd;
  const size_t N = (size_t)P.N;
  constexpr int OG = QH, OF = QH + 27;
  // ---------------- forward recomputation (as cell_update, FP64)
  const double gpx = fdv.gpx, gpy = fdv.gpy, gpz = fdv.gpz, lp = fdv.lp;
  const double Gx = rp.grad[0], Gy = rp.grad[1], Gz = rp.grad[2];
  const double Ttot = Tc + Gx * (x + 0.5 - rp.origin[0]) + Gy * (y + 0.5 - rp.origin[1]) +
                      Gz * (z + 0.5 - rp.origin[2]);
  const double gTx = fdv.gtx + Gx, gTy = fdv.gty + Gy, gTz = fdv.gtz + Gz;
  double pst = 0, jx = 0, jy = 0, jz = 0, sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
  static_for<0, 27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ex = cx<27>(i), ey = cy<27>(i), ez = cz<27>(i);
    const double v = getg(I);
    pst += v;
    jx += ex * v; jy += ey * v; jz += ez * v;
    sxx += ex * ex * v; syy += ey * ey * v; szz += ez * ez * v;
    sxy += ex * ey * v; sxz += ex * ez * v; syz += ey * ez * v;
  });
  const double xi = rp.xi;
  const double sigma = rp.sigma_ref + rp.sigma_T * (Ttot - rp.T_ref);
  const double beta = 12.0 * sigma / xi, kap = 1.5 * sigma * xi;
  const double dw = phi * (phi - 1.0) * (phi - 0.5);
  const double mu = 4.0 * beta * dw - kap * lp;
  const double g2 = gpx * gpx + gpy * gpy + gpz * gpz;
  const double tdp = gTx * gpx + gTy * gpy + gTz * gpz;
  const double cm = 1.5 * xi * rp.sigma_T;
  const double rho = rp.rho_L + phi * (rp.rho_H - rp.rho_L);
  const double Fx = mu * gpx + cm * (g2 * gTx - tdp * gpx) + rho * rp.gravity[0];
  const double Fy = mu * gpy + cm * (g2 * gTy - tdp * gpy) + rho * rp.gravity[1];
  const double Fz = mu * gpz + cm * (g2 * gTz - tdp * gpz) + rho * rp.gravity[2];
  const double ax = Fx / rho, ay = Fy / rho, az = Fz / rho;
  const double ux = jx + 0.5 * ax, uy = jy + 0.5 * ay, uz = jz + 0.5 * az;
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
  double l_ux = 0, l_uy = 0, l_uz = 0, l_ax = 0, l_ay = 0, l_az = 0;
  double l_phi = 0, l_T = 0, l_pst = 0;
  // f collision: f' = f* - omT (f* - w Tc E) + w (q - u.G)
  if constexpr (QF > 0) {
    const double omT = rp.omega_T;
    double sw = 0;
    static_for<0, QF>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr double w = weight<QF>(i);
      constexpr int ex = cx<QF>(i), ey = cy<QF>(i), ez = cz<QF>(i);
      const double L = A.lam_in[(size_t)(OF + i) * N + cell];
      const double cu = ex * ux + ey * uy + ez * uz;
      A.lstar[(size_t)(OF + i) * N + cell] = (1.0 - omT) * L;
      l_T += omT * L * w * (1.0 - 1.5 * uu + 4.5 * cu * cu + 3.0 * cu);
      const double k = omT * L * w * Tc;
      l_ux += k * (-3.0 * ux + 9.0 * cu * ex + 3.0 * ex);
      l_uy += k * (-3.0 * uy + 9.0 * cu * ey + 3.0 * ey);
      l_uz += k * (-3.0 * uz + 9.0 * cu * ez + 3.0 * ez);
      sw += L * w;
    });
    l_ux -= sw * Gx; l_uy -= sw * Gy; l_uz -= sw * Gz;
  }
  // h collision: h' = h* - om (h* - w phi E) + sc w c.Fphi
  double l_Fpx = 0, l_Fpy = 0, l_Fpz = 0;
  {
    const double om = rp.omega_phi, sc = 1.0 - 0.5 * om;
    static_for<0, QH>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr double w = weight<QH>(i);
      constexpr int ex = cx<QH>(i), ey = cy<QH>(i), ez = cz<QH>(i);
      const double L = A.lam_in[(size_t)i * N + cell];
      const double cu = ex * ux + ey * uy + ez * uz;
      A.lstar[(size_t)i * N + cell] = (1.0 - om) * L;
      l_phi += om * L * w * (1.0 - 1.5 * uu + 4.5 * cu * cu + 3.0 * cu);
      const double k = om * L * w * phi;
      l_ux += k * (-3.0 * ux + 9.0 * cu * ex + 3.0 * ex);
      l_uy += k * (-3.0 * uy + 9.0 * cu * ey + 3.0 * ey);
      l_uz += k * (-3.0 * uz + 9.0 * cu * ez + 3.0 * ez);
      l_Fpx += sc * L * w * ex; l_Fpy += sc * L * w * ey; l_Fpz += sc * L * w * ez;
    });
  }
  // g collision: g' = w [p* - 1.5 (uu + ua) + 3 cu + 1.5 ca + 4.5 cu^2 + 4.5 cu ca] + sum_m P_m B_m(c; u)
  double lPxx = 0, lPyy = 0, lPzz = 0, lPxy = 0, lPxz = 0, lPyz = 0;
  static_for<0, 27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr double w = weight<27>(i);
    constexpr int ex = cx<27>(i), ey = cy<27>(i), ez = cz<27>(i);
    const double L = A.lam_in[(size_t)(OG + i) * N + cell];
    const double cu = ex * ux + ey * uy + ez * uz, ca = ex * ax + ey * ay + ez * az;
    const double wl = w * L;
    l_pst += wl;
    l_ux += wl * (-1.5 * (2.0 * ux + ax) + 3.0 * ex + 9.0 * cu * ex + 4.5 * ca * ex);
    l_uy += wl * (-1.5 * (2.0 * uy + ay) + 3.0 * ey + 9.0 * cu * ey + 4.5 * ca * ey);
    l_uz += wl * (-1.5 * (2.0 * uz + az) + 3.0 * ez + 9.0 * cu * ez + 4.5 * ca * ez);
    l_ax += wl * (-1.5 * ux + 1.5 * ex + 4.5 * cu * ex);
    l_ay += wl * (-1.5 * uy + 1.5 * ey + 4.5 * cu * ey);
    l_az += wl * (-1.5 * uz + 1.5 * ez + 4.5 * cu * ez);
    const double X0 = bas(0, ex, ux), X1 = bas(1, ex, ux), X2 = bas(2, ex, ux);
    const double Y0 = bas(0, ey, uy), Y1 = bas(1, ey, uy), Y2 = bas(2, ey, uy);
    const double Z0 = bas(0, ez, uz), Z1 = bas(1, ez, uz), Z2 = bas(2, ez, uz);
    lPxx += L * X2 * Y0 * Z0; lPyy += L * X0 * Y2 * Z0; lPzz += L * X0 * Y0 * Z2;
    lPxy += L * X1 * Y1 * Z0; lPxz += L * X1 * Y0 * Z1; lPyz += L * X0 * Y1 * Z1;
    l_ux += L * (Pyy * X1 * Y2 * Z0 + Pzz * X1 * Y0 * Z2 + 2.0 * Pxy * X2 * Y1 * Z0 + 2.0 * Pxz * X2 * Y0 * Z1 +
                 Pyz * X1 * Y1 * Z1);
    l_uy += L * (Pxx * X2 * Y1 * Z0 + Pzz * X0 * Y1 * Z2 + 2.0 * Pxy * X1 * Y2 * Z0 + Pxz * X1 * Y1 * Z1 +
                 2.0 * Pyz * X0 * Y2 * Z1);
    l_uz += L * (Pxx * X2 * Y0 * Z1 + Pyy * X0 * Y2 * Z1 + Pxy * X1 * Y1 * Z1 + 2.0 * Pxz * X1 * Y0 * Z2 +
                 2.0 * Pyz * X0 * Y1 * Z2);
  });
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

// Pass A: the generic kernel's z-march (phi / T halo planes from the pulled
// state s^n in shared memory), then cell_adjoint per cell.
template <int QH, int QF>
__global__ void __launch_bounds__(NTHREADS) adj_cell_kernel(const DevParams P, const AdjPtrs A, int zchunk) {
  __shared__ double s_phi[3][HP];
  __shared__ double s_T[3][HP];
  const auto& rp = P.pd;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, P.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < P.nx) && (y < P.ny);
  auto fill = [&](int zp, int slot) {
    for (int k = tid; k < HP; k += NTHREADS) {
      const int gx = wrap_any(x0 + (k % HX) - 1, P.nx);
      const int gy = wrap_any(y0 + (k / HX) - 1, P.ny);
      int zz = zp;
      bool ghost = false;
      if (P.walls) {
        if (zp < 0) { zz = 0; ghost = true; }
        else if (zp >= P.nz) { zz = P.nz - 1; ghost = true; }
      } else {
        zz = wrap(zp, P.nz);
      }
      const double phi = pulled_sum<QH, false>(P, A.s_h, gx, gy, zz, 0.0);
      double T = pulled_sum<QF, true>(P, A.s_f, gx, gy, zz, 0.0);
      if (ghost) T = 2.0 * (zp < 0 ? rp.T_bottom : rp.T_top) - T;
      s_phi[slot][k] = phi;
      s_T[slot][k] = T;
    }
  };
  int sm = 0, sc = 1, sp = 2;
  if (z0 < z1) {
    fill(z0 - 1, sm);
    fill(z0, sc);
  }
  for (int z = z0; z < z1; ++z) {
    fill(z + 1, sp);
    __syncthreads();
    if (active) {
      const int c0 = (ty + 1) * HX + (tx + 1);
      Stencil27<double> fd;
      fd.template eval<HX>(s_phi[sm], s_phi[sc], s_phi[sp], s_T[sm], s_T[sc], s_T[sp], c0);
      auto getg = [&](auto I) { return pull<27, false, decltype(I)::value>(P, A.s_g, x, y, z, 0.0); };
      cell_adjoint<QH, QF>(P, A, x, y, z, cell_index(P, x, y, z), s_phi[sc][c0], s_T[sc][c0], fd, getg);
    }
    __syncthreads();
    const int t = sm;
    sm = sc;
    sc = sp;
    sp = t;
  }
}

// Pass B1: total adjoints of phi and T (stencil transposes).  Grid: x over
// the cells of one plane (32-bit index), y = z.
__global__ void adj_fields_kernel(const DevParams P, const AdjPtrs A) {
  const size_t N = (size_t)P.N;
  const unsigned plane = (unsigned)P.nx * (unsigned)P.ny;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < plane) {
    const int y = (int)(r / (unsigned)P.nx), x = (int)(r - (unsigned)y * (unsigned)P.nx);
    const int z = blockIdx.y;
    const size_t cell = (size_t)z * plane + r;
    double lphi = A.fld[(size_t)ADJ_PHI * N + cell];
    double lT = A.fld[(size_t)ADJ_T * N + cell];
    // central term of the Laplacian: lap(x) = 6 sum_k w_k (v(x + c_k) - v(x))
    lphi -= 6.0 * (1.0 - weight<27>(0)) * A.fld[(size_t)ADJ_LP * N + cell];
    // x reads v at x + c_k: every (x, k) whose read resolves to this cell
    auto add_from = [&](int xs, int ys, int zs, int k, double sgn_T) {
      const size_t c = cell_index(P, xs, ys, zs);
      const double w = weight<27>(k);
      const int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
      lphi += 3.0 * w * (ex * A.fld[(size_t)ADJ_GPX * N + c] + ey * A.fld[(size_t)ADJ_GPY * N + c] +
                         ez * A.fld[(size_t)ADJ_GPZ * N + c]) +
              6.0 * w * A.fld[(size_t)ADJ_LP * N + c];
      lT += sgn_T * 3.0 * w * (ex * A.fld[(size_t)ADJ_GTX * N + c] + ey * A.fld[(size_t)ADJ_GTY * N + c] +
                               ez * A.fld[(size_t)ADJ_GTZ * N + c]);
    };
    for (int k = 1; k < 27; ++k) {
      const int ex = q27_cx(k), ey = q27_cy(k), ez = q27_cz(k);
      const int xs = wrap(x - ex, P.nx), ys = wrap(y - ey, P.ny);
      int zs = z - ez;
      if (P.walls) {
        if (zs >= 0 && zs < P.nz) add_from(xs, ys, zs, k, 1.0);
        // wall ghosts: a cell of the boundary layer reading across the wall
        // reads this (same-layer) cell: phi mirrored, T as 2 T_w - T
        if (z == 0 && ez == -1) add_from(xs, ys, 0, k, -1.0);
        if (z == P.nz - 1 && ez == 1) add_from(xs, ys, P.nz - 1, k, -1.0);
      } else {
        add_from(xs, ys, wrap(zs, P.nz), k, 1.0);
      }
    }
    A.tot[cell] = lphi;
    A.tot[N + cell] = lT;
  }
}

// Pass B2: transpose of the pull (with bounce-back / anti-bounce-back).
// Grid: x over the cells of one plane (32-bit index), y = z, z = direction.
template <int QH, int QF>
__global__ void adj_pull_kernel(const DevParams P, const AdjPtrs A) {
  const size_t N = (size_t)P.N;
  const unsigned plane = (unsigned)P.nx * (unsigned)P.ny;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < plane) {
    const int y = (int)(r / (unsigned)P.nx), x = (int)(r - (unsigned)y * (unsigned)P.nx);
    const int z = blockIdx.y, d = blockIdx.z;
    const size_t cell = (size_t)z * plane + r;
    const size_t k = (size_t)d * N + cell;
    int set, j, ex, ey, ez, jb;
    if (d < QH) {
      set = 0; j = d; ex = cx<QH>(j); ey = cy<QH>(j); ez = cz<QH>(j);
      jb = opp<QH>(j);
    } else if (d < QH + 27) {
      set = 1; j = d - QH; ex = cx<27>(j); ey = cy<27>(j); ez = cz<27>(j);
      jb = QH + opp<27>(j);
    } else {
      set = 2; j = d - QH - 27; ex = cx<QF>(j); ey = cy<QF>(j); ez = cz<QF>(j);
      jb = QH + 27 + opp<QF>(j);
    }
    int zt = z + ez;
    bool inside = true;
    if (P.walls) inside = zt >= 0 && zt < P.nz;
    else zt = wrap(zt, P.nz);
    double v;
    if (inside) {
      const size_t c = cell_index(P, wrap(x + ex, P.nx), wrap(y + ey, P.ny), zt);
      v = A.lstar[(size_t)d * N + c];
      if (set == 0) v += A.tot[c];
      else if (set == 2) v += A.tot[N + c];
    } else {
      v = A.lstar[(size_t)jb * N + cell];
      if (set == 0) v += A.tot[cell];
      else if (set == 2) v = -(v + A.tot[N + cell]);
    }
    A.lam_out[k] = v;
  }
}

// Seed lam^N for J(phi^N): dJ/dphi given per cell (dense, N values) -> the
// adjoint of the stored h (pull transpose with bounce-back); g, f: 0.
template <int QH, int QF>
__global__ void adj_seed_kernel(const DevParams P, const double* __restrict__ dJdphi, double* lam) {
  const size_t N = (size_t)P.N;
  constexpr int NQ = QH + 27 + QF;
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
// (the intensity enters every f'_i of a patch cell as w_i I_k).  One block
// per patch, fixed summation order.
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
    static_for<0, QF>([&](auto I) {
      constexpr int i = decltype(I)::value;
      s += weight<QF>(i) * lam[(size_t)(QH + 27 + i) * N + cell];
    });
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) dJdI[k] += red[0];
}

}  // namespace lbm
