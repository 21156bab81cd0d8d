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
    if (zz < 0) return (RF)2 * rp.T_bottom - psi[cell_index(P, xx, yy, 0)];
    if (zz >= P.nz) return (RF)2 * rp.T_top - psi[cell_index(P, xx, yy, P.nz - 1)];
  } else {
    zz = wrap(zz, P.nz);
  }
  return psi[cell_index(P, xx, yy, zz)];
}

// R(psi) = -u.(grad psi + G) + alpha lap psi + q_T  (Eq. temperature, uniform
// kappa and rho c_p); 7-point / central operators or the isotropic D3Q27 ones.
template <class RF>
__device__ __forceinline__ RF rk_rhs(const DevParams& P, const RF* __restrict__ psi, const RF* u,
                                     int x, int y, int z, size_t cell) {
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
                                RF* acc, RF* out, int kind) {
  const size_t n = (size_t)P.N;
  for (size_t cell = blockIdx.x * (size_t)blockDim.x + threadIdx.x; cell < n;
       cell += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(cell % P.nx);
    const int y = (int)((cell / P.nx) % P.ny);
    const int z = (int)(cell / ((size_t)P.nx * P.ny));
    const RF K = rk_rhs(P, psi, u, x, y, z, cell);
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
// conduction profile between walls; equilibria of Sec. 2.2 evaluated in FP64.
template <class S, int QH, int QF>
__global__ void init_kernel(const DevParams P, const double* __restrict__ drops, int nd, S* h, S* g,
                            S* f, typename Store<S>::R* Tfield) {
  using R = typename Store<S>::R;
  const auto& rp = P.pd;  // initialisation runs in FP64 in every mode
  const size_t n = (size_t)P.N;
  for (size_t cell = blockIdx.x * (size_t)blockDim.x + threadIdx.x; cell < n;
       cell += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(cell % P.nx);
    const int y = (int)((cell / P.nx) % P.ny);
    const int z = (int)(cell / ((size_t)P.nx * P.ny));
    double phi = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
    for (int k = 0; k < nd; ++k) {
      const double* d = drops + 7 * k;
      double dx = x + 0.5 - d[0], dy = y + 0.5 - d[1], dz = z + 0.5 - d[2];
      dx -= P.nx * rint(dx / P.nx);
      dy -= P.ny * rint(dy / P.ny);
      if (!P.walls) dz -= P.nz * rint(dz / P.nz);
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      const double pk = 0.5 * (1.0 + tanh(2.0 * (d[3] - r) / rp.xi));
      phi = fmax(phi, pk);
      ux += pk * d[4];
      uy += pk * d[5];
      uz += pk * d[6];
    }
    const double T0 = P.walls ? rp.T_bottom + (rp.T_top - rp.T_bottom) * (z + 0.5) / P.nz : 0.0;
    const size_t pc = pdf_index(P, x, y, z);
    const size_t np = (size_t)P.Np;
    const double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < QH; ++i) {
      const double cu = cx<QH>(i) * ux + cy<QH>(i) * uy + cz<QH>(i) * uz;
      const double e = weight<QH>(i) * phi * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
      Store<S>::st(h + (size_t)i * np + pc, (R)(e - weight<QH>(i) * rp.shift_h));
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) {
      const double cu = cx<27>(i) * ux + cy<27>(i) * uy + cz<27>(i) * uz;
      const double e = weight<27>(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
      Store<S>::st(g + (size_t)i * np + pc, (R)e);
    }
    if constexpr (QF > 0) {
#pragma unroll
      for (int i = 0; i < QF; ++i) {
        const double cu = cx<QF>(i) * ux + cy<QF>(i) * uy + cz<QF>(i) * uz;
        const double e = weight<QF>(i) * T0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        Store<S>::st(f + (size_t)i * np + pc, (R)(e - weight<QF>(i) * rp.shift_f));
      }
    } else {
      Tfield[cell] = (R)T0;
    }
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

// Periodic ghost cells of one padded PDF buffer of nq directions: every
// ghost position (x, y) outside [0, nx) x [0, ny) receives the value of cell
// (x mod nx, y mod ny) of the same plane and direction (the single-GPU form
// of a ghost-layer exchange).  Ghost positions of a plane are enumerated as
// the left/right column strips of the interior rows, then the full top and
// bottom row strips.
template <class S>
__global__ void ghost_fill_kernel(const DevParams P, S* __restrict__ buf) {
  // grid: x over the ghost positions of one plane, y = z, z = direction
  const int GX = P.GX, GY = P.GY;
  const int side = 2 * GX * P.ny;            // column strips of the interior rows
  const int per_plane = side + 2 * GY * P.NXP;
  const int z = blockIdx.y, q = blockIdx.z;
  S* base = buf + (size_t)q * P.Np;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < per_plane; r += gridDim.x * blockDim.x) {
    int x, y;
    if (r < side) {
      y = r / (2 * GX);
      const int j = r - y * (2 * GX);
      x = j < GX ? j - GX : P.nx + (j - GX);
    } else {
      const int rr = r - side;
      const int j = rr / P.NXP;              // 0 .. 2 GY - 1
      x = rr - j * P.NXP - GX;
      y = j < GY ? j - GY : P.ny + (j - GY);
    }
    if (x >= P.nx + GX) continue;            // row-pitch padding: never read
    int xs = x % P.nx; if (xs < 0) xs += P.nx;
    int ys = y % P.ny; if (ys < 0) ys += P.ny;
    base[pdf_index(P, x, y, z)] = base[pdf_index(P, xs, ys, z)];
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

}  // namespace lbm
