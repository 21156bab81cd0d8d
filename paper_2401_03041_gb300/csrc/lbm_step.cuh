// lbm_step.cuh - the generic fused time-step kernel (any lattice size).
//
// One launch performs one full time step of the thermocapillary phase-field
// LBM (Sec. 2.2-2.3; sweep order of Alg. 1 / Alg. 2) for every cell.  A CTA
// owns a TX x TY column of cells and marches along z over a chunk of planes.
// phi and T are needed on a one-cell halo for the finite differences; they
// are zeroth moments of *pulled* PDFs, so the CTA recomputes them for every
// (TX+2) x (TY+2) plane it meets and keeps three planes (z-1, z, z+1) in
// shared memory.  PDFs are read straight from global memory with periodic
// wrap and wall rules.  The bulk kernel (lbm_bulk.cuh) is the fast path;
// this one serves lattices that path does not cover and is its cross-check.
#pragma once

#include "lbm_cell.cuh"

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

// Value of direction I pulled into cell (x, y, z): p_I(x - c_I) as stored
// (shifted by w_I s, s = shift), with half-way bounce-back (ABB=false) or
// anti-bounce-back (ABB=true; in stored form -p_opp + 2 w_I (T_w - s)) when
// the source lies beyond a z wall.
template <int Q, bool ABB, int I, class S>
__device__ __forceinline__ typename Store<S>::R pull(const DevParams& P, const S* __restrict__ base,
                                                     int x, int y, int z, typename Store<S>::R shift) {
  using R = typename Store<S>::R;
  const int zs = z - cz<Q>(I);
  constexpr R w = (R)weight<Q>(I);
  if (P.walls && (zs < 0 || zs >= P.nz)) {
    const R v = Store<S>::ld(base + (size_t)opp<Q>(I) * P.Np + pdf_index(P, x, y, z));
    if constexpr (ABB) {
      R Tw = wall_T<R>(P, x, zs < 0);
      if (P.moving_walls) Tw *= wall_even<Q, I, R>(P, zs >= P.nz ? 1 : 0);
      return -v + (R)2 * w * (Tw - shift);
    }
    return v;
  }
  const int xs = wrap(x - cx<Q>(I), P.nx);
  const int ys = wrap(y - cy<Q>(I), P.ny);
  const int zz = P.walls ? zs : wrap(zs, P.nz);
  return Store<S>::ld(base + (size_t)I * P.Np + pdf_index(P, xs, ys, zz));
}

// Moving-wall momentum of direction I pulled into plane z (zero unless its
// source lies beyond a moving wall); h takes it times phi.
template <int Q, int I, class R>
__device__ __forceinline__ R pull_wall_term(const DevParams& P, int z) {
  if (!P.moving_walls) return (R)0;
  const int zs = z - cz<Q>(I);
  if (zs >= 0 && zs < P.nz) return (R)0;
  return wall_momentum<Q, I, R>(P, zs >= P.nz ? 1 : 0);
}

// Zeroth moment of the pulled populations (un-shifted: the stored values plus
// sum_i w_i s = s).
template <int Q, bool ABB, class S>
__device__ __forceinline__ typename Store<S>::R pulled_sum(const DevParams& P, const S* __restrict__ base,
                                                           int x, int y, int z,
                                                           typename Store<S>::R shift) {
  using R = typename Store<S>::R;
  R s = shift;
  static_for<0, Q>([&](auto I) { s += pull<Q, ABB, decltype(I)::value>(P, base, x, y, z, shift); });
  return s;
}

// Fixed-order block reduction of the FP64 diagnostics partials, through
// red[NT / 32][kDiagVals] doubles of shared memory.
template <int NT>
__device__ __forceinline__ void diag_block_reduce_in(const double* dsum, double* out_partials, double* red) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
#pragma unroll
  for (int k = 0; k < kDiagVals; ++k) {
    double v = dsum[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) red[(tid >> 5) * kDiagVals + k] = v;
  }
  __syncthreads();
  if (tid < kDiagVals) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v += red[w * kDiagVals + tid];
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    out_partials[b * kDiagVals + tid] = v;
  }
}

template <int NT>
__device__ __forceinline__ void diag_block_reduce(const double* dsum, double* out_partials) {
  __shared__ double s_red[NT / 32 * kDiagVals];
  diag_block_reduce_in<NT>(dsum, out_partials, s_red);
}

// QF = 0: RK thermal (T stored as a field); QF in {7, 15, 19, 27}: LB thermal.
template <class S, int QH, int QF>
__global__ void __launch_bounds__(NTHREADS)
step_kernel(const DevParams P, const StepPtrs<S, typename Store<S>::R> A, int zchunk, int mode) {
  using R = typename Store<S>::R;
  const auto& rp = RP<R>(P);
  __shared__ R s_phi[3][HP];
  __shared__ R s_T[3][HP];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, P.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < P.nx) && (y < P.ny);
  const R shh = (R)rp.shift_h, shf = (R)rp.shift_f;

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
      const R phi = pulled_sum<QH, false>(P, A.h_src, gx, gy, zz, shh);
      R T;
      if constexpr (QF > 0) T = pulled_sum<QF, true>(P, A.f_src, gx, gy, zz, shf);
      else T = A.T[cell_index(P, gx, gy, zz)];
      if (ghost) T = (R)2 * wall_T<R>(P, gx, zp < 0) - T;
      // phi beyond a wall: the mirror, or the contact-angle ghost
      const R phig = (ghost && P.wetting) ? wet_ghost<R>(phi, wall_k<R>(P, zp < 0 ? 0 : 1)) : phi;
      s_phi[slot][k] = phig;
      s_T[slot][k] = T;
    }
  };

  DiagAcc<R> dsum;   // per-thread FP64 diagnostics

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
      Stencil27<R> fd;
      fd.template eval<HX>(s_phi[sm], s_phi[sc], s_phi[sp], s_T[sm], s_T[sc], s_T[sp], c0);
      R rgx = 0, rgy = 0, rgz = 0, rlap = 0;
      R pgx = 0, pgy = 0, pgz = 0, plap;
      if constexpr (QF == 0) {
        rk_std<R, HX>(s_T[sm], s_T[sc], s_T[sp], c0, rgx, rgy, rgz, rlap);
        if (P.alpha_ratio && !P.rk_iso) rk_std<R, HX>(s_phi[sm], s_phi[sc], s_phi[sp], c0, pgx, pgy, pgz, plap);
      }
      const size_t cell = cell_index(P, x, y, z);
      const R phic = s_phi[sc][(ty + 1) * HX + (tx + 1)];
      auto geth = [&](auto I) {
        constexpr int i = decltype(I)::value;
        return pull<QH, false, i>(P, A.h_src, x, y, z, shh) + phic * pull_wall_term<QH, i, R>(P, z);
      };
      auto getg = [&](auto I) {
        constexpr int i = decltype(I)::value;
        return pull<27, false, i>(P, A.g_src, x, y, z, (R)0) + pull_wall_term<27, i, R>(P, z);
      };
      auto getf = [&](auto I) {
        if constexpr (QF > 0) return pull<QF, true, decltype(I)::value>(P, A.f_src, x, y, z, shf);
        else return (R)0;
      };
      cell_update<S, QH, QF>(P, A, x, y, z, cell, pdf_index(P, x, y, z), mode, s_phi[sc][c0], s_T[sc][c0], fd, rgx, rgy,
                             rgz, rlap, pgx, pgy, pgz, geth, getg, getf, dsum);
    }
    __syncthreads();
    const int t = sm;
    sm = sc;
    sc = sp;
    sp = t;
  }

  if (mode & MODE_DIAG) {
    double ds[kDiagVals];
    dsum.flush(ds);
    diag_block_reduce<NTHREADS>(ds, A.diag_partials);
  }
}

}  // namespace lbm
