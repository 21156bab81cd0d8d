// lbm_aux.cuh - the non-fused kernels: RK stages 2..4, initialisation,
// PDF <-> FP64 conversion and the deterministic diagnostics reduction.
#pragma once

#include "lbm_step.cuh"

namespace lbm {

// Value of the stage field psi at (x+dx, y+dy, z+dz): periodic in x, y (and z
// without walls); beyond a wall the Dirichlet ghost 2 T_w - psi(first cell).
template <class RF>
__device__ __forceinline__ RF stage_at(const DevParams& P, const RF* __restrict__ psi, int x, int y,
                                       int z, int dx, int dy, int dz) {
  const auto& rp = RP<RF>(P);
  const int xx = wrap(x + dx, P.nx), yy = wrap(y + dy, P.ny);
  int zz = z + dz;
  if (P.walls) {
    if (zz < 0) return (RF)2 * wall_T<RF>(P, xx, true) - psi[cell_index(P, xx, yy, 0)];
    if (zz >= P.nz) return (RF)2 * rp.T_top - psi[cell_index(P, xx, yy, P.nz - 1)];
  } else {
    zz = wrap(zz, P.nz);
  }
  return psi[cell_index(P, xx, yy, zz)];
}

// phi at (x+dx, y+dy, z+dz): periodic in x, y (and z without walls); beyond a
// wall the mirror ghost phi(first cell), or the contact-angle ghost.
template <class RF>
__device__ __forceinline__ RF phi_at(const DevParams& P, const RF* __restrict__ phi, int x, int y, int z,
                                     int dx, int dy, int dz) {
  const int xx = wrap(x + dx, P.nx), yy = wrap(y + dy, P.ny);
  int zz = z + dz;
  if (P.walls) {
    if (zz < 0 || zz >= P.nz) {
      const int top = zz >= P.nz ? 1 : 0;
      const RF a = phi[cell_index(P, xx, yy, top ? P.nz - 1 : 0)];
      return P.wetting ? wet_ghost<RF>(a, wall_k<RF>(P, top)) : a;
    }
  } else {
    zz = wrap(zz, P.nz);
  }
  return phi[cell_index(P, xx, yy, zz)];
}

// Gradient of phi by the RK solver's operator (central differences, or the
// isotropic D3Q27 gradient summed over opposite pairs).
template <class RF>
__device__ __forceinline__ void rk_phi_grad(const DevParams& P, const RF* __restrict__ phi, int x, int y, int z,
                                            RF& gx, RF& gy, RF& gz) {
  if (P.rk_iso) {
    gx = gy = gz = 0;
#pragma unroll
    for (int k = 1; k < 27; ++k) {
      const bool first = q27_cx(k) > 0 || (q27_cx(k) == 0 && (q27_cy(k) > 0 || (q27_cy(k) == 0 && q27_cz(k) > 0)));
      if (first) {
        const RF w = (RF)weight<27>(k);
        const RF d = phi_at(P, phi, x, y, z, q27_cx(k), q27_cy(k), q27_cz(k)) -
                     phi_at(P, phi, x, y, z, -q27_cx(k), -q27_cy(k), -q27_cz(k));
        if (q27_cx(k)) gx += (RF)q27_cx(k) * w * d;
        if (q27_cy(k)) gy += (RF)q27_cy(k) * w * d;
        if (q27_cz(k)) gz += (RF)q27_cz(k) * w * d;
      }
    }
    gx *= (RF)3; gy *= (RF)3; gz *= (RF)3;
  } else {
    gx = (RF)0.5 * (phi_at(P, phi, x, y, z, 1, 0, 0) - phi_at(P, phi, x, y, z, -1, 0, 0));
    gy = (RF)0.5 * (phi_at(P, phi, x, y, z, 0, 1, 0) - phi_at(P, phi, x, y, z, 0, -1, 0));
    gz = (RF)0.5 * (phi_at(P, phi, x, y, z, 0, 0, 1) - phi_at(P, phi, x, y, z, 0, 0, -1));
  }
}

// R(psi) = -u.(grad psi + G) + alpha lap psi + q_T  (Eq. temperature, uniform
// kappa and rho c_p); 7-point / central operators or the isotropic D3Q27 ones.
// With a conductivity or heat-capacity ratio (phi != null): alpha(phi) lap psi
// plus (kappa_H - kappa_L) / C(phi) grad phi . (grad psi + G), phi of this step.
template <class RF>
__device__ __forceinline__ RF rk_rhs(const DevParams& P, const RF* __restrict__ psi, const RF* u,
                                     const RF* __restrict__ phi, int x, int y, int z, size_t cell) {
  const auto& rp = RP<RF>(P);
  const RF c = psi[cell];
  RF gx, gy, gz, lap;
  if (P.rk_iso) {
    gx = gy = gz = lap = 0;
#pragma unroll
    for (int k = 1; k < 27; ++k) {
      const RF v = stage_at(P, psi, x, y, z, q27_cx(k), q27_cy(k), q27_cz(k));
      const RF w = (RF)weight<27>(k);
      lap += w * (v - c);
      // opposite-pair differences (exact zero on uniform fields)
      const bool first = q27_cx(k) > 0 || (q27_cx(k) == 0 && (q27_cy(k) > 0 || (q27_cy(k) == 0 && q27_cz(k) > 0)));
      if (first) {
        const RF d = v - stage_at(P, psi, x, y, z, -q27_cx(k), -q27_cy(k), -q27_cz(k));
        if (q27_cx(k)) gx += (RF)q27_cx(k) * w * d;
        if (q27_cy(k)) gy += (RF)q27_cy(k) * w * d;
        if (q27_cz(k)) gz += (RF)q27_cz(k) * w * d;
      }
    }
    gx *= (RF)3; gy *= (RF)3; gz *= (RF)3; lap *= (RF)6;
  } else {
    const RF xp = stage_at(P, psi, x, y, z, 1, 0, 0), xm = stage_at(P, psi, x, y, z, -1, 0, 0);
    const RF yp = stage_at(P, psi, x, y, z, 0, 1, 0), ym = stage_at(P, psi, x, y, z, 0, -1, 0);
    const RF zp = stage_at(P, psi, x, y, z, 0, 0, 1), zm = stage_at(P, psi, x, y, z, 0, 0, -1);
    gx = (RF)0.5 * (xp - xm);
    gy = (RF)0.5 * (yp - ym);
    gz = (RF)0.5 * (zp - zm);
    lap = xp + xm + yp + ym + zp + zm - (RF)6 * c;
  }
  const RF ux = u[cell], uy = u[P.N + cell], uz = u[2 * P.N + cell];
  if (phi) {
    RF pgx, pgy, pgz;
    rk_phi_grad(P, phi, x, y, z, pgx, pgy, pgz);
    const ThermCoef<RF> tc = therm_coef<RF>(P, phi[cell]);
    const RF Gx = (RF)rp.grad[0], Gy = (RF)rp.grad[1], Gz = (RF)rp.grad[2];
    return -(ux * (gx + Gx) + uy * (gy + Gy) + uz * (gz + Gz)) + tc.alpha * lap + heat_source<RF>(P, x, y, z) +
           tc.dk_C * (pgx * (gx + Gx) + pgy * (gy + Gy) + pgz * (gz + Gz));
  }
  return -(ux * (gx + (RF)rp.grad[0]) + uy * (gy + (RF)rp.grad[1]) + uz * (gz + (RF)rp.grad[2])) +
         (RF)rp.alpha * lap + heat_source<RF>(P, x, y, z);
}

enum : int { RK2_FINAL = 0, RK4_STAGE2 = 1, RK4_STAGE3 = 2, RK4_FINAL = 3 };

// Later RK stages (Eq. rk2 midpoint rule; Eq. rk4), one thread per cell:
//   RK2_FINAL : T <- T + R(S1)
//   RK4_STAGE2: K2 = R(S1);  out = T + K2/2;  acc += K2/3
//   RK4_STAGE3: K3 = R(S2);  out = T + K3;    acc += K3/3
//   RK4_FINAL : K4 = R(S3);  T <- T + acc + K4/6
// T is only read and written at the thread's own cell, so the final stages
// update it in place; the stencil reads go to psi, a different buffer.
template <class RF>
__global__ void rk_stage_kernel(const DevParams P, const RF* __restrict__ psi, RF* T, const RF* u,
                                const RF* __restrict__ phi, RF* acc, RF* out, int kind) {
  const size_t n = (size_t)P.N;
  for (size_t cell = blockIdx.x * (size_t)blockDim.x + threadIdx.x; cell < n;
       cell += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(cell % P.nx);
    const int y = (int)((cell / P.nx) % P.ny);
    const int z = (int)(cell / ((size_t)P.nx * P.ny));
    const RF K = rk_rhs(P, psi, u, phi, x, y, z, cell);
    const RF Tc = T[cell];
    if (kind == RK2_FINAL) {
      T[cell] = Tc + K;
    } else if (kind == RK4_STAGE2) {
      out[cell] = Tc + (RF)0.5 * K;
      acc[cell] = acc[cell] + K * (RF)(1.0 / 3.0);
    } else if (kind == RK4_STAGE3) {
      out[cell] = Tc + K;
      acc[cell] = acc[cell] + K * (RF)(1.0 / 3.0);
    } else {
      T[cell] = Tc + (acc[cell] + K * (RF)(1.0 / 6.0));
    }
  }
}

// Initial state: tanh droplets (periodic minimum image), u = sum phi_k v_k,
// conduction profile between walls; profiles and equilibria of Sec. 2.2 in
// the compute type of the storage (FP64 in FP64 mode; FP32 otherwise, with
// the offsets to the droplet centres formed in FP64).
//
// A block covers a 32 x 4 x 2 tile of cells.  Before the per-cell loop it
// culls the droplet table against the tile's bounding box: droplet k matters
// to a cell only where 2 (r - R_k) / xi <= 40 (beyond that tanh rounds to -1
// in FP64 and the droplet's term is exactly zero; it is taken as zero).  The
// box test uses a lower bound on r with one lattice unit of margin, so it
// never drops a droplet the per-cell test would keep.  Surviving droplets are
// kept as bit masks, 1024 droplets per pass, and visited in ascending order.
constexpr int kInitTX = 32, kInitTY = 4, kInitTZ = 2;

__device__ __forceinline__ double min_image(double d, int n) { return d - n * rint(d / n); }
__device__ __forceinline__ float min_image(float d, int n) { return d - (float)n * rintf(d / (float)n); }

template <class S, int QH, int QF>
__global__ void __launch_bounds__(kInitTX * kInitTY * kInitTZ)
init_kernel(const DevParams P, const double* __restrict__ drops, int nd, S* h, S* g, S* f,
            typename Store<S>::R* Tfield) {
  using R = typename Store<S>::R;
  constexpr int NT = kInitTX * kInitTY * kInitTZ;
  const auto& rp = P.pd;  // droplet profiles and velocities in FP64 in every mode
  __shared__ uint32_t mask[32];
  const int tid = threadIdx.x;
  const int x = blockIdx.x * kInitTX + (tid % kInitTX);
  const int y = blockIdx.y * kInitTY + (tid / kInitTX) % kInitTY;
  const int z = blockIdx.z * kInitTZ + tid / (kInitTX * kInitTY);
  const bool inside = x < P.nx && y < P.ny && z < P.nz;
  // tile bounding box of cell centres: centre and half extent per axis
  const int bx0 = blockIdx.x * kInitTX, bx1 = min(bx0 + kInitTX, P.nx);
  const int by0 = blockIdx.y * kInitTY, by1 = min(by0 + kInitTY, P.ny);
  const int bz0 = blockIdx.z * kInitTZ, bz1 = min(bz0 + kInitTZ, P.nz);
  const double bcx = 0.5 * (bx0 + bx1), bhx = 0.5 * (bx1 - bx0 - 1);
  const double bcy = 0.5 * (by0 + by1), bhy = 0.5 * (by1 - by0 - 1);
  const double bcz = 0.5 * (bz0 + bz1), bhz = 0.5 * (bz1 - bz0 - 1);
  const double reach = 20.0 * rp.xi + 1.0;

  // droplet profiles in the compute type of the storage: FP64 in FP64 mode;
  // with FP32 / FP16 storage the offsets to the centre are formed in FP64
  // and the profile evaluated in FP32 (the FP64 pipe is a small fraction of
  // the FP32 rate on this GPU and would dominate the initialisation)
  using PR = R;
  PR phi = 0, ux = 0, uy = 0, uz = 0;
  for (int k0 = 0; k0 < nd; k0 += 1024) {
    for (int j = tid; j < 1024; j += NT) {   // every warp takes whole 32-droplet words
      const int k = k0 + j;
      bool near = false;
      if (k < nd && P.sub) {
        near = true;   // sub-domain: no culling (the tile box is in local columns)
      } else if (k < nd) {
        const double* d = drops + 7 * k;
        double dx = bcx - d[0], dy = bcy - d[1], dz = bcz - d[2];
        dx = min_image(dx, P.nx);
        dy = min_image(dy, P.ny);
        if (!P.walls) dz = min_image(dz, P.nz);
        dx = fmax(fabs(dx) - bhx, 0.0);
        dy = fmax(fabs(dy) - bhy, 0.0);
        dz = fmax(fabs(dz) - bhz, 0.0);
        const double lim = d[3] + reach;
        near = dx * dx + dy * dy + dz * dz <= lim * lim;
      }
      const unsigned bits = __ballot_sync(0xffffffffu, near);
      if ((j & 31) == 0) mask[j >> 5] = bits;
    }
    __syncthreads();
    if (inside) {
      for (int wd = 0; wd < 32; ++wd) {
        for (uint32_t m = mask[wd]; m; m &= m - 1) {
          const int k = k0 + wd * 32 + __ffs(m) - 1;
          const double* d = drops + 7 * k;
          PR dx = (PR)(global_x(P, x) + 0.5 - d[0]), dy = (PR)(y + 0.5 - d[1]), dz = (PR)(z + 0.5 - d[2]);
          dx = min_image(dx, P.sub ? P.gnx : P.nx);
          dy = min_image(dy, P.ny);
          if (!P.walls) dz = min_image(dz, P.nz);
          const PR r = sqrt(dx * dx + dy * dy + dz * dz);
          const PR a = (PR)2 * ((PR)d[3] - r) / (PR)rp.xi;
          if (a < (PR)-40) continue;
          const PR pk = (PR)0.5 * ((PR)1 + tanh(a));
          phi = fmax(phi, pk);
          ux += pk * (PR)d[4];
          uy += pk * (PR)d[5];
          uz += pk * (PR)d[6];
        }
      }
    }
    __syncthreads();
  }
  if (!inside) return;
  const size_t cell = ((size_t)z * P.ny + y) * P.nx + x;
  const double Tb = wall_T<double>(P, x, true);
  const double T0 = P.walls ? Tb + (rp.T_top - Tb) * (z + 0.5) / P.nz : 0.0;
  const size_t pc = pdf_index(P, x, y, z);
  const size_t np = (size_t)P.Np;
  // equilibria in the compute type of the storage (FP64 in FP64 mode)
  const auto& rq = RP<R>(P);
  const R phR = (R)phi, TR = (R)T0, uxR = (R)ux, uyR = (R)uy, uzR = (R)uz;
  const R uu = uxR * uxR + uyR * uyR + uzR * uzR;
#pragma unroll
  for (int i = 0; i < QH; ++i) {
    const R cu = (R)cx<QH>(i) * uxR + (R)cy<QH>(i) * uyR + (R)cz<QH>(i) * uzR;
    const R w = (R)weight<QH>(i);
    const R e = w * phR * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu);
    Store<S>::st(h + (size_t)i * np + pc, e - w * (R)rq.shift_h);
  }
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const R cu = (R)cx<27>(i) * uxR + (R)cy<27>(i) * uyR + (R)cz<27>(i) * uzR;
    const R e = (R)weight<27>(i) * ((R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu);
    Store<S>::st(g + (size_t)i * np + pc, e);
  }
  if constexpr (QF > 0) {
#pragma unroll
    for (int i = 0; i < QF; ++i) {
      const R cu = (R)cx<QF>(i) * uxR + (R)cy<QF>(i) * uyR + (R)cz<QF>(i) * uzR;
      const R w = (R)weight<QF>(i);
      const R e = w * TR * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu);
      Store<S>::st(f + (size_t)i * np + pc, e - w * (R)rq.shift_f);
    }
  } else {
    Tfield[cell] = (R)T0;
  }
}

// Stored (shifted) PDFs in the padded layout <-> dense FP64 values [Q][N].
template <class S, int Q>
__global__ void pdf_to_f64_kernel(const DevParams P, const S* __restrict__ src, double* __restrict__ dst,
                                  double shift) {
  const size_t N = (size_t)P.N, total = (size_t)Q * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(k / N);
    const size_t c = k - (size_t)i * N;
    const int x = (int)(c % P.nx), y = (int)((c / P.nx) % P.ny), z = (int)(c / ((size_t)P.nx * P.ny));
    double w = 0.0;
#pragma unroll
    for (int j = 0; j < Q; ++j)
      if (j == i) w = weight<Q>(j);
    dst[k] = (double)Store<S>::ld(src + (size_t)i * P.Np + pdf_index(P, x, y, z)) + w * shift;
  }
}

template <class S, int Q>
__global__ void f64_to_pdf_kernel(const DevParams P, const double* __restrict__ src, S* __restrict__ dst,
                                  double shift) {
  using R = typename Store<S>::R;
  const size_t N = (size_t)P.N, total = (size_t)Q * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(k / N);
    const size_t c = k - (size_t)i * N;
    const int x = (int)(c % P.nx), y = (int)((c / P.nx) % P.ny), z = (int)(c / ((size_t)P.nx * P.ny));
    double w = 0.0;
#pragma unroll
    for (int j = 0; j < Q; ++j)
      if (j == i) w = weight<Q>(j);
    Store<S>::st(dst + (size_t)i * P.Np + pdf_index(P, x, y, z), (R)(src[k] - w * shift));
  }
}

// Which ghost sides of each array of a PDF set a ghost fill writes (bits:
// 1 the columns x < 0, 2 the columns x >= nx, 4 the rows y < 0, 8 the rows y
// >= ny; a corner where its column and row sides both apply; 16 / 32 every
// side on plane 0 / nz - 1 when the lattice has z walls).  All bits: the
// whole periodic extension.
constexpr int kMaxSetArrays = 27 + 27 + 27;
struct GhostSides {
  unsigned char m[kMaxSetArrays];
};

// Periodic ghost cells of one padded PDF buffer of nq directions: every
// ghost position (x, y) outside [0, nx) x [0, ny) on a side that sides.m[q]
// selects receives the value of cell (x mod nx, y mod ny) of the same plane
// and direction (the single-GPU form of a ghost-layer exchange).  Grid: x
// over the items of one plane, y = z, z = direction.  Items [0, NYP): the
// ghost columns of padded row y (ghost rows included, sources taken from row
// y mod ny); items [NYP, NYP + 2 GY nvec): one 16-byte vector of interior
// columns of a ghost row.  With nx a multiple of V = 16 / sizeof(S) (GX = V) a
// row's two ghost blocks are 16-byte vectors; with nx a multiple of 2V each is
// written together with the interior half of its 32-byte sector (the same
// values that half holds), so that no sector is written partially.
template <class S>
__global__ void __launch_bounds__(128) ghost_fill_kernel(const DevParams P, S* __restrict__ buf,
                                                         const __grid_constant__ GhostSides sides) {
  constexpr int V = 16 / (int)sizeof(S);
  const int GX = P.GX, GY = P.GY, nx = P.nx, ny = P.ny;
  const int z = blockIdx.y, q = blockIdx.z;
  unsigned m = sides.m[q];
  if (P.walls && (((m & 16) && z == 0) || ((m & 32) && z == P.nz - 1))) m |= 15;
  if ((m & 15) == 0) return;
  const bool left = m & 1, right = m & 2, low = m & 4, high = m & 8;
  S* plane = buf + (size_t)q * P.Np + (size_t)z * P.NYP * P.NXP;
  const int nvec = (nx + V - 1) / V;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  auto wrap_y = [&](int y) { int ys = y % ny; return ys < 0 ? ys + ny : ys; };
  if (r < P.NYP) {
    const int y = r - GY;
    if ((y < 0 && !low) || (y >= ny && !high)) return;
    S* row = plane + (size_t)r * P.NXP;                        // element x at row[x + GX]
    const S* src = plane + (size_t)(wrap_y(y) + GY) * P.NXP;
    if (nx % V == 0) {
      if (nx % (2 * V) == 0) {
        // sectors [x -V .. V-1] and [x nx-V .. nx+V-1] both become (b, a)
        const uint4 a = *reinterpret_cast<const uint4*>(src + GX);           // x = 0 .. V-1
        const uint4 b = *reinterpret_cast<const uint4*>(src + GX + nx - V);  // x = nx-V .. nx-1
        if (left) {
          uint4* s0 = reinterpret_cast<uint4*>(row);
          s0[0] = b; s0[1] = a;
        }
        if (right) {
          uint4* s1 = reinterpret_cast<uint4*>(row + GX + nx - V);
          s1[0] = b; s1[1] = a;
        }
      } else {
        if (left) *reinterpret_cast<uint4*>(row) = *reinterpret_cast<const uint4*>(src + GX + nx - V);
        if (right) *reinterpret_cast<uint4*>(row + GX + nx) = *reinterpret_cast<const uint4*>(src + GX);
      }
    } else {
      for (int j = 0; j < GX; ++j) {
        int xl = (j - GX) % nx; if (xl < 0) xl += nx;               // ghost x = j - GX
        if (left) row[j] = src[GX + xl];
        if (right) row[GX + nx + j] = src[GX + (j % nx)];            // ghost x = nx + j
      }
    }
  } else {
    const int k = r - P.NYP;
    if (k >= 2 * GY * nvec) return;
    const int which = k / nvec, j = k - which * nvec;
    if ((which < GY && !low) || (which >= GY && !high)) return;
    const int y = which < GY ? which - GY : ny + (which - GY);      // ghost row
    S* dst = plane + (size_t)(y + GY) * P.NXP + GX + j * V;
    const S* src = plane + (size_t)(wrap_y(y) + GY) * P.NXP + GX + j * V;
    if (j * V + V <= nx) {
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
    } else {
      for (int e = 0; e < nx - j * V; ++e) dst[e] = src[e];
    }
  }
}

// Fixed-order (deterministic) sum of the per-CTA diagnostics partials.
static __global__ void diag_finalize_kernel(const double* __restrict__ partials, int nblocks,
                                     double* __restrict__ out) {
  __shared__ double s[256];
  for (int k = 0; k < kDiagVals; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(size_t)b * kDiagVals + k];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
      if (threadIdx.x < off) s[threadIdx.x] += s[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = s[0];
    __syncthreads();
  }
}

// Halo exchange of an x-slab decomposition: columns [x0, x0 + w) of every
// row, for the nq directions of one padded PDF set (stride Np, stored
// values) and, if T is given, of the dense RK temperature field, to / from
// a contiguous buffer [direction][z][y][w] followed (16-byte aligned) by
// T [z][y][w].
template <class S>
__global__ void halo_x_kernel(const DevParams P, S* __restrict__ set, int nq, typename Store<S>::R* __restrict__ T,
                              int x0, int w, unsigned char* __restrict__ buf, size_t t_off, int to_buf) {
  using R = typename Store<S>::R;
  const size_t plane = (size_t)P.nz * P.ny * w;
  const size_t npdf = (size_t)nq * plane;
  const size_t total = npdf + (T ? plane : 0);
  S* pb = reinterpret_cast<S*>(buf);
  R* tb = reinterpret_cast<R*>(buf + t_off);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const size_t r = k < npdf ? k % plane : k - npdf;
    const int xx = (int)(r % w), y = (int)((r / w) % P.ny), z = (int)(r / ((size_t)w * P.ny));
    const int x = x0 + xx;
    if (k < npdf) {
      const int i = (int)(k / plane);
      S* at = set + (size_t)i * P.Np + pdf_index(P, x, y, z);
      if (to_buf) pb[k] = *at;
      else *at = pb[k];
    } else {
      R* at = T + ((size_t)z * P.ny + y) * P.nx + x;
      if (to_buf) tb[r] = *at;
      else *at = tb[r];
    }
  }
}

}  // namespace lbm
