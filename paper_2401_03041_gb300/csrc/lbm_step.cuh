// lbm_step.cuh - the fused time-step kernel and its helpers.
//
// One launch performs one full time step of the thermocapillary phase-field
// LBM (Sec. 2.2-2.3; sweep order of Alg. 1 / Alg. 2) for every cell:
//   a1 pull-stream h, g, f (half-way bounce-back / anti-bounce-back at walls)
//   a2 phi = sum h*, p* = sum g*, T = sum f* (or the stored T for RK)
//   a3 grad phi, lap phi, grad T with the isotropic D3Q27 operators
//   a4-a6 n, F^phi, sigma(T), mu_phi, F_s (+ rho g), u = sum c g* + F/(2 rho)
//   a7 h collision (single rate + Guo source of Eq. phasefieldforce)
//   a8 g collision in central-moment space (second-order moments at 1/tau(phi),
//      higher orders at rate 1, Guo forcing in moment space)
//   a9 f collision (single rate + w_i q_T)   or   a9' RK stage 1 (K1 = R(T))
//
// Blocking: a CTA owns a TX x TY column of cells and marches along z over a
// chunk of planes.  phi and T are needed on a one-cell halo for the finite
// differences; they are zeroth moments of *pulled* PDFs, so the CTA
// recomputes them for every (TX+2) x (TY+2) plane it meets and keeps three
// planes (z-1, z, z+1) in shared memory.  HBM then sees each PDF read once and
// written once per step; the halo re-reads of h and f hit L1/L2.
//
// Central-moment collision, evaluated in closed form.  With y = g* - g^eq +
// S/2 (S the Guo source), the relaxation of every central moment kappa_k at
// rate w_k gives g' = g^eq + S/2 + K(u)^-1 [(1 - w_k) kappa_k(y)].  The zeroth
// and first central moments of y vanish identically (p* = sum g*,
// u = sum c g* + a/2), and moments of order >= 3 have w_k = 1, so only the six
// second-order central moments Pi of y survive, all relaxed with w = 1/tau(phi):
//   Pi_ab = sum g* c_a c_b - p* c_s^2 d_ab - u_a u_b + (u_a a_b + a_a u_b)/2.
// K(u)^-1 is the tensor product of the 1D inverse shifts; a unit central
// moment of order e along one axis maps to the populations
//   P0(c) = {1 - u^2, (u^2 + u)/2, (u^2 - u)/2},  P1(c) = {-2u, u + 1/2, u - 1/2},
//   P2(c) = {-1, 1/2, 1/2}   for c = {0, +1, -1},
// so (K^-1 Pi)_i = sum over the six moments of products P_ex(cx) P_ey(cy) P_ez(cz).
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int HX = TX + 2;
constexpr int HY = TY + 2;
constexpr int HP = HX * HY;
constexpr int NTHREADS = TX * TY;

__device__ __forceinline__ int wrap(int v, int n) {
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// v mod n for any v (tile halos of lattices narrower than a tile span
// several periods).
__device__ __forceinline__ int wrap_any(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ size_t cell_index(const DevParams& P, int x, int y, int z) {
  return ((size_t)z * P.ny + y) * P.nx + x;
}

// Value of direction i pulled into cell (x, y, z): p_i(x - c_i), with
// half-way bounce-back (ABB=false) or anti-bounce-back (ABB=true, wall
// temperature Tw) when the source lies beyond a z wall.
template <int Q, bool ABB, class S>
__device__ __forceinline__ typename Store<S>::R pull(const DevParams& P, const S* __restrict__ base,
                                                     int i, int x, int y, int z, double shift) {
  using R = typename Store<S>::R;
  const int zs = z - cz<Q>(i);
  const R wsh = (R)(weight<Q>(i) * shift);
  if (P.walls && (zs < 0 || zs >= P.nz)) {
    const R v = Store<S>::ld(base + (size_t)opp<Q>(i) * P.N + cell_index(P, x, y, z)) + wsh;
    if (ABB) {
      const R Tw = (R)(zs < 0 ? P.T_bottom : P.T_top);
      return -v + (R)(2.0 * weight<Q>(i)) * Tw;
    }
    return v;
  }
  const int xs = wrap(x - cx<Q>(i), P.nx);
  const int ys = wrap(y - cy<Q>(i), P.ny);
  const int zz = P.walls ? zs : wrap(zs, P.nz);
  return Store<S>::ld(base + (size_t)i * P.N + cell_index(P, xs, ys, zz)) + wsh;
}

// Zeroth moment of the pulled PDFs of one stencil.
template <int Q, bool ABB, class S>
__device__ __forceinline__ typename Store<S>::R pulled_sum(const DevParams& P, const S* __restrict__ base,
                                                           int x, int y, int z, double shift) {
  using R = typename Store<S>::R;
  R s = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) s += pull<Q, ABB>(P, base, i, x, y, z, shift);
  return s;
}

// Heat source density q_T at cell (x, y, z) (centre (x+1/2, y+1/2, z+1/2)):
// Gaussian sources (Eq. HeatSource, r <= d) plus heater patches (by index).
__device__ __forceinline__ double heat_source(const DevParams& P, int x, int y, int z) {
  double q = 0.0;
  for (int k = 0; k < P.nsrc; ++k) {
    const double dx = x + 0.5 - P.src[k][0], dy = y + 0.5 - P.src[k][1], dz = z + 0.5 - P.src[k][2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double w = P.src[k][4];
    if (P.src[k][5] < 0.0 || r2 <= P.src[k][5]) q += P.src[k][3] * exp(-2.0 * r2 / (w * w));
  }
  if (P.npatch > 0 && z == P.patch_z) {
    for (int k = 0; k < P.npatch; ++k) {
      if (x >= P.px0[k] && x < P.px0[k] + P.patch_sx && y >= P.py0[k] && y < P.py0[k] + P.patch_sy)
        q += P.pI[k];
    }
  }
  return q;
}

template <class R>
__device__ __forceinline__ void inv_basis(R u, R& p0z, R& p0p, R& p0m, R& p1z, R& p1p, R& p1m) {
  // P0 and P1 of the 1D inverse shift at c = 0, +1, -1 (P2 = {-1, 1/2, 1/2})
  const R uu = u * u;
  p0z = (R)1 - uu;
  p0p = (R)0.5 * (uu + u);
  p0m = (R)0.5 * (uu - u);
  p1z = (R)-2 * u;
  p1p = u + (R)0.5;
  p1m = u - (R)0.5;
}

template <class R>
__device__ __forceinline__ R basis_pick(int c, R z, R p, R m) { return c == 0 ? z : (c > 0 ? p : m); }

// QF = 0: RK thermal (T stored as a field); QF in {7, 15, 19, 27}: LB thermal.
template <class S, int QH, int QF>
__global__ void __launch_bounds__(NTHREADS)
step_kernel(const DevParams P, const StepPtrs<S, typename Store<S>::R> A, int zchunk, int mode) {
  using R = typename Store<S>::R;
  __shared__ R s_phi[3][HP];
  __shared__ R s_T[3][HP];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, P.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < P.nx) && (y < P.ny);

  // phi and T on the (TX+2) x (TY+2) plane zp -> slot
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
      const R phi = pulled_sum<QH, false>(P, A.h_src, gx, gy, zz, P.shift_h);
      R T;
      if constexpr (QF > 0) T = pulled_sum<QF, true>(P, A.f_src, gx, gy, zz, P.shift_f);
      else T = A.T[cell_index(P, gx, gy, zz)];
      if (ghost) T = (R)(2.0 * (zp < 0 ? P.T_bottom : P.T_top)) - T;  // mirror for phi
      s_phi[slot][k] = phi;
      s_T[slot][k] = T;
    }
  };

  double dsum[kDiagVals];
#pragma unroll
  for (int k = 0; k < kDiagVals; ++k) dsum[k] = 0.0;

  int sm = 0, sc = 1, sp = 2;
  if (z0 < z1) {
    fill(z0 - 1, sm);
    fill(z0, sc);
  }
  for (int z = z0; z < z1; ++z) {
    fill(z + 1, sp);
    __syncthreads();
    if (active) {
      // ---------------------------------------------------- a3 stencils
      const int c0 = (ty + 1) * HX + (tx + 1);
      const R phi = s_phi[sc][c0];
      const R Tc = s_T[sc][c0];
      // Gradients as sums over the 13 opposite pairs of differences
      // psi(x + c) - psi(x - c): exactly zero on uniform fields (with FMA
      // contraction a sum of +w psi and -w psi terms is not).
      R gpx = 0, gpy = 0, gpz = 0, lp = 0, gtx = 0, gty = 0, gtz = 0, lt = 0;
#pragma unroll
      for (int k = 1; k < 27; ++k) {
        const int sl = q27_cz(k) == 0 ? sc : (q27_cz(k) > 0 ? sp : sm);
        const int o = c0 + q27_cy(k) * HX + q27_cx(k);
        const R vp = s_phi[sl][o];
        const R vt = s_T[sl][o];
        const R w = (R)weight<27>(k);
        lp += w * (vp - phi);
        lt += w * (vt - Tc);
        // the first direction of each pair: first non-zero component positive
        const bool first = q27_cx(k) > 0 || (q27_cx(k) == 0 && (q27_cy(k) > 0 || (q27_cy(k) == 0 && q27_cz(k) > 0)));
        if (first) {
          const int slm = q27_cz(k) == 0 ? sc : (q27_cz(k) > 0 ? sm : sp);
          const int om_ = c0 - q27_cy(k) * HX - q27_cx(k);
          const R dp = vp - s_phi[slm][om_];
          const R dt = vt - s_T[slm][om_];
          if (q27_cx(k)) { gpx += (R)q27_cx(k) * w * dp; gtx += (R)q27_cx(k) * w * dt; }
          if (q27_cy(k)) { gpy += (R)q27_cy(k) * w * dp; gty += (R)q27_cy(k) * w * dt; }
          if (q27_cz(k)) { gpz += (R)q27_cz(k) * w * dp; gtz += (R)q27_cz(k) * w * dt; }
        }
      }
      gpx *= (R)3; gpy *= (R)3; gpz *= (R)3; lp *= (R)6;
      gtx *= (R)3; gty *= (R)3; gtz *= (R)3; lt *= (R)6;
      // background gradient: T_total = T + G.(x - x0)
      const R Gx = (R)P.grad[0], Gy = (R)P.grad[1], Gz = (R)P.grad[2];
      const R Ttot = Tc + (R)(P.grad[0] * (x + 0.5 - P.origin[0]) + P.grad[1] * (y + 0.5 - P.origin[1]) +
                              P.grad[2] * (z + 0.5 - P.origin[2]));
      const R gTx = gtx + Gx, gTy = gty + Gy, gTz = gtz + Gz;

      // ---------------------------------------------------- a1/a2 hydro pull
      R gs[27];
#pragma unroll
      for (int i = 0; i < 27; ++i) gs[i] = pull<27, false>(P, A.g_src, i, x, y, z, 0.0);
      R pst = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
      for (int i = 0; i < 27; ++i) {
        pst += gs[i];
        if (cx<27>(i)) jx += (R)cx<27>(i) * gs[i];
        if (cy<27>(i)) jy += (R)cy<27>(i) * gs[i];
        if (cz<27>(i)) jz += (R)cz<27>(i) * gs[i];
      }

      // ---------------------------------------------------- a4/a5 forces
      const R sigma = (R)P.sigma_ref + (R)P.sigma_T * (Ttot - (R)P.T_ref);
      const R xi = (R)P.xi;
      const R beta = (R)12 * sigma / xi;
      const R kap = (R)1.5 * sigma * xi;
      const R mu = (R)4 * beta * phi * (phi - (R)1) * (phi - (R)0.5) - kap * lp;
      const R g2 = gpx * gpx + gpy * gpy + gpz * gpz;
      const R tdp = gTx * gpx + gTy * gpy + gTz * gpz;
      const R cm = (R)1.5 * xi * (R)P.sigma_T;
      const R rho = (R)P.rho_L + phi * (R)(P.rho_H - P.rho_L);
      const R Fx = mu * gpx + cm * (g2 * gTx - tdp * gpx) + rho * (R)P.gravity[0];
      const R Fy = mu * gpy + cm * (g2 * gTy - tdp * gpy) + rho * (R)P.gravity[1];
      const R Fz = mu * gpz + cm * (g2 * gTz - tdp * gpz) + rho * (R)P.gravity[2];
      const R irho = (R)1 / rho;
      const R ax = Fx * irho, ay = Fy * irho, az = Fz * irho;
      // ---------------------------------------------------- a6 velocity
      const R ux = jx + (R)0.5 * ax, uy = jy + (R)0.5 * ay, uz = jz + (R)0.5 * az;
      const R uu = ux * ux + uy * uy + uz * uz;

      if (mode & MODE_DIAG) {
        const double dphi = (double)phi;
        dsum[0] += dphi;
        dsum[1] += (double)Tc;
        dsum[2] += 0.5 * (double)rho * (double)uu;
        dsum[3] += dphi * (x + 0.5);
        dsum[4] += dphi * (y + 0.5);
        dsum[5] += dphi * (z + 0.5);
        if (!isfinite(dphi) || !isfinite((double)Tc) || !isfinite((double)uu)) dsum[6] += 1.0;
      }
      const size_t cell = cell_index(P, x, y, z);
      if (mode & MODE_MACRO) {
        const double vals[6] = {(double)phi, (double)ux, (double)uy, (double)uz, (double)pst, (double)Tc};
        const unsigned cnt[4] = {1u, 3u, 1u, 1u};
        int slot = 0, v = 0;
        for (int f = 0; f < 4; ++f) {
          if (A.macro_mask & (1u << f)) {
            for (unsigned c = 0; c < cnt[f]; ++c) {
              const size_t at = (size_t)(slot + c) * P.N + cell;
              if (A.macro_dtype == 0) ((double*)A.macro_out)[at] = vals[v + c];
              else ((float*)A.macro_out)[at] = (float)vals[v + c];
            }
            slot += cnt[f];
          }
          v += cnt[f];
        }
      }

      if (mode & MODE_COLLIDE) {
        // ---------------------------------------------------- a8 g collision
        {
          R sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
#pragma unroll
          for (int i = 0; i < 27; ++i) {
            if (cx<27>(i)) sxx += gs[i];
            if (cy<27>(i)) syy += gs[i];
            if (cz<27>(i)) szz += gs[i];
            if (cx<27>(i) * cy<27>(i)) sxy += (R)(cx<27>(i) * cy<27>(i)) * gs[i];
            if (cx<27>(i) * cz<27>(i)) sxz += (R)(cx<27>(i) * cz<27>(i)) * gs[i];
            if (cy<27>(i) * cz<27>(i)) syz += (R)(cy<27>(i) * cz<27>(i)) * gs[i];
          }
          const R tau = (R)P.tau_L + phi * (R)(P.tau_H - P.tau_L);
          const R om = (R)1 / tau;
          const R k1 = (R)1 - om;
          const R p3 = pst * (R)(1.0 / 3.0);
          const R Pxx = k1 * (sxx - p3 - ux * ux + ux * ax);
          const R Pyy = k1 * (syy - p3 - uy * uy + uy * ay);
          const R Pzz = k1 * (szz - p3 - uz * uz + uz * az);
          const R Pxy = k1 * (sxy - ux * uy + (R)0.5 * (ux * ay + ax * uy));
          const R Pxz = k1 * (sxz - ux * uz + (R)0.5 * (ux * az + ax * uz));
          const R Pyz = k1 * (syz - uy * uz + (R)0.5 * (uy * az + ay * uz));
          R X0z, X0p, X0m, X1z, X1p, X1m, Y0z, Y0p, Y0m, Y1z, Y1p, Y1m, Z0z, Z0p, Z0m, Z1z, Z1p, Z1m;
          inv_basis(ux, X0z, X0p, X0m, X1z, X1p, X1m);
          inv_basis(uy, Y0z, Y0p, Y0m, Y1z, Y1p, Y1m);
          inv_basis(uz, Z0z, Z0p, Z0m, Z1z, Z1p, Z1m);
          // z pass: A[(a,b)](cz) for the six moments
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
          S* dst = A.g_dst;
#pragma unroll
          for (int i = 0; i < 27; ++i) {
            const int ex = cx<27>(i), ey = cy<27>(i), ez = cz<27>(i);
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
            const R neq = r0 * B0 + r1 * B1 + r2 * B2;
            const R w = (R)weight<27>(i);
            const R cu = (R)ex * ux + (R)ey * uy + (R)ez * uz;
            const R ca = (R)ex * ax + (R)ey * ay + (R)ez * az;
            const R ua = ux * ax + uy * ay + uz * az;
            const R geq = w * (pst + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu);
            const R src = w * ((R)3 * (ca - ua) + (R)9 * cu * ca);
            Store<S>::st(dst + (size_t)i * P.N + cell, geq + (R)0.5 * src + neq);
          }
        }
        // ---------------------------------------------------- a7 h collision
        {
          const R nrm = (R)1 / (sqrt(g2) + (R)P.eps_n);
          const R th = (R)4 * phi * ((R)1 - phi) / xi * nrm;
          const R fpx = th * gpx, fpy = th * gpy, fpz = th * gpz;
          const R om = (R)P.omega_phi;
          const R sc_ = (R)1 - (R)0.5 * om;
#pragma unroll
          for (int i = 0; i < QH; ++i) {
            const R hs = pull<QH, false>(P, A.h_src, i, x, y, z, P.shift_h);
            const R w = (R)weight<QH>(i);
            const R cu = (R)cx<QH>(i) * ux + (R)cy<QH>(i) * uy + (R)cz<QH>(i) * uz;
            const R cf = (R)cx<QH>(i) * fpx + (R)cy<QH>(i) * fpy + (R)cz<QH>(i) * fpz;
            const R heq = w * phi * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu);
            const R hn = hs - om * (hs - heq) + sc_ * w * cf;
            Store<S>::st(A.h_dst + (size_t)i * P.N + cell, hn - (R)(weight<QH>(i) * P.shift_h));
          }
        }
        // ---------------------------------------------------- a9 / a9' thermal
        const R q = (R)heat_source(P, x, y, z);
        const R uG = ux * Gx + uy * Gy + uz * Gz;
        if constexpr (QF > 0) {
          const R om = (R)P.omega_T;
#pragma unroll
          for (int i = 0; i < QF; ++i) {
            const R fs = pull<QF, true>(P, A.f_src, i, x, y, z, P.shift_f);
            const R w = (R)weight<QF>(i);
            const R cu = (R)cx<QF>(i) * ux + (R)cy<QF>(i) * uy + (R)cz<QF>(i) * uz;
            const R feq = w * Tc * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu);
            const R fn = fs - om * (fs - feq) + w * (q - uG);
            Store<S>::st(A.f_dst + (size_t)i * P.N + cell, fn - (R)(weight<QF>(i) * P.shift_f));
          }
        } else {
          // RK stage 1: K1 = R(T^n) with the local u of this step
          R gx_, gy_, gz_, lap;
          if (P.rk_iso) {
            gx_ = gtx; gy_ = gty; gz_ = gtz; lap = lt;
          } else {
            const R* pl = s_T[sc];
            gx_ = (R)0.5 * (pl[c0 + 1] - pl[c0 - 1]);
            gy_ = (R)0.5 * (pl[c0 + HX] - pl[c0 - HX]);
            gz_ = (R)0.5 * (s_T[sp][c0] - s_T[sm][c0]);
            lap = pl[c0 + 1] + pl[c0 - 1] + pl[c0 + HX] + pl[c0 - HX] + s_T[sp][c0] + s_T[sm][c0] -
                  (R)6 * Tc;
          }
          const R K1 = -(ux * (gx_ + Gx) + uy * (gy_ + Gy) + uz * (gz_ + Gz)) + (R)P.alpha * lap + q;
          A.u_out[cell] = ux;
          A.u_out[P.N + cell] = uy;
          A.u_out[2 * P.N + cell] = uz;
          A.s1_out[cell] = Tc + (R)0.5 * K1;
          if (A.rk_acc) A.acc_out[cell] = K1 * (R)(1.0 / 6.0);
        }
      }
    }
    __syncthreads();
    const int t = sm;
    sm = sc;
    sc = sp;
    sp = t;
  }

  if (mode & MODE_DIAG) {
    // warp shuffle + shared-memory block reduction in FP64
    __shared__ double s_red[NTHREADS / 32][kDiagVals];
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) {
      double v = dsum[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((tid & 31) == 0) s_red[tid >> 5][k] = v;
    }
    __syncthreads();
    if (tid < kDiagVals) {
      double v = 0.0;
      for (int w = 0; w < NTHREADS / 32; ++w) v += s_red[w][tid];
      const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      A.diag_partials[b * kDiagVals + tid] = v;
    }
  }
}

}  // namespace lbm
