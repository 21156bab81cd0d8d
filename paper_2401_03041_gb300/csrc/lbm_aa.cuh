// lbm_aa.cuh - the in-place (AA-pattern) time step: one PDF set per field.
//
// The two-grid pull scheme of the other kernels reads one PDF set and writes
// the other.  Here a single set F is read and overwritten in place, in two
// alternating phases (Bailey et al.'s AA pattern), with stored populations
// p_i(x) (post-collision, before streaming) held as
//   even time level:  F[opp(i)](x) = p_i(x);
//   odd time level:   F[i](x + c_i) = p_i(x)   (F[opp(i)](x) where x + c_i
//                                                lies beyond a z wall).
// A step from an even level gathers the pulled population f*_i(x) =
// p_i(x - c_i) = F[opp(i)](x - c_i) and scatters the new p_i(x) to
// F[i](x + c_i); a step from an odd level gathers f*_i(x) = F[i](x) and
// scatters to F[opp(i)](x).  Either way a cell reads and writes the same set
// of slots, and no other cell touches them, so the update is race-free.
// Sources beyond a z wall take the wall rules of the two-grid kernels
// (bounce-back with the moving-wall term, thermal anti-bounce-back) applied
// to F[i](x), the slot the previous phase left the reflected population in.
//
// The finite differences need phi and T of level n at the neighbours, which
// an in-place update overwrites; so each step first writes the (phi, T) pairs
// of every cell (zeroth moments of the gathered populations, summed in the
// same order as the two-grid kernels' halo sums: aa_moments_kernel here, or
// aa_moments_tiled_kernel in lbm_skew.cuh on the tiled path), and the step
// kernel takes its stencil values from that field.
// In FP64 the result equals the generic two-grid kernel's to rounding (the
// two are compiled separately and contract their products into FMAs
// differently).
#pragma once

#include "lbm_step.cuh"

namespace lbm {

// Population of direction I gathered into cell (x, y, z), as stored (shifted
// by w_I s): nb = true for a step from an even level (from the neighbour),
// false from an odd level (local).  ABB: thermal anti-bounce-back at walls.
template <int Q, bool ABB, int I, class S>
__device__ __forceinline__ typename Store<S>::R aa_get(const DevParams& P, const S* __restrict__ base, int x,
                                                       int y, int z, bool nb, typename Store<S>::R shift) {
  using R = typename Store<S>::R;
  const int zs = z - cz<Q>(I);
  if (P.walls && (zs < 0 || zs >= P.nz)) {
    const R v = Store<S>::ld(base + (size_t)I * P.Np + pdf_index(P, x, y, z));
    if constexpr (ABB) {
      constexpr R w = (R)weight<Q>(I);
      R Tw = wall_T<R>(P, x, zs < 0);
      if (P.moving_walls) Tw *= wall_even<Q, I, R>(P, zs >= P.nz ? 1 : 0);
      return -v + (R)2 * w * (Tw - shift);
    }
    return v;
  }
  if (!nb) return Store<S>::ld(base + (size_t)I * P.Np + pdf_index(P, x, y, z));
  const int xs = wrap(x - cx<Q>(I), P.nx);
  const int ys = wrap(y - cy<Q>(I), P.ny);
  const int zz = P.walls ? zs : wrap(zs, P.nz);
  return Store<S>::ld(base + (size_t)opp<Q>(I) * P.Np + pdf_index(P, xs, ys, zz));
}

// Destination of the new population of direction I of cell (x, y, z).
template <int Q, int I>
__device__ __forceinline__ size_t aa_put_index(const DevParams& P, int x, int y, int z, bool nb) {
  if (!nb) return (size_t)opp<Q>(I) * P.Np + pdf_index(P, x, y, z);
  const int zd = z + cz<Q>(I);
  if (P.walls && (zd < 0 || zd >= P.nz)) return (size_t)opp<Q>(I) * P.Np + pdf_index(P, x, y, z);
  const int xd = wrap(x + cx<Q>(I), P.nx);
  const int yd = wrap(y + cy<Q>(I), P.ny);
  const int zz = P.walls ? zd : wrap(zd, P.nz);
  return (size_t)I * P.Np + pdf_index(P, xd, yd, zz);
}

// (phi, T) of every cell at the current level, from the gathered
// populations: phi = s_h + sum_i h*_i, T = s_f + sum_i f*_i (LB) or the
// stored field (RK), summed in direction order like the two-grid kernels.
// Grid: x = row blocks of kAaRowBlock cells times the ny rows, y = planes;
// 32-bit index arithmetic.  (Gathering through refreshed periodic ghosts
// instead of wrapping x and y was measured slower: 6.4 against 5.1 ms at
// 512^3 FP32.)
constexpr int kAaRowBlock = 128;

template <class S, int QH, int QF>
__global__ void __launch_bounds__(kAaRowBlock)
aa_moments_kernel(const DevParams P, const S* __restrict__ h, const S* __restrict__ f,
                  const typename Store<S>::R* __restrict__ Tfield, int nb,
                  typename PairOf<typename Store<S>::R>::type* __restrict__ phiT) {
  using R = typename Store<S>::R;
  const auto& rp = RP<R>(P);
  const R shh = (R)rp.shift_h, shf = (R)rp.shift_f;
  const int bx = (P.nx + kAaRowBlock - 1) / kAaRowBlock;
  const int y = (int)(blockIdx.x / (unsigned)bx);
  const int x = (int)(blockIdx.x - (unsigned)y * (unsigned)bx) * kAaRowBlock + (int)threadIdx.x;
  const int z = (int)blockIdx.y;
  if (x >= P.nx) return;
  const size_t c = cell_index(P, x, y, z);
  auto body = [&](auto nbtag) {
    constexpr bool NB = decltype(nbtag)::value;
    R phi = shh;
    static_for<0, QH>([&](auto I) { phi += aa_get<QH, false, decltype(I)::value>(P, h, x, y, z, NB, shh); });
    R T;
    if constexpr (QF > 0) {
      T = shf;
      static_for<0, QF>([&](auto I) { T += aa_get<QF, true, decltype(I)::value>(P, f, x, y, z, NB, shf); });
    } else {
      T = Tfield[c];
    }
    typename PairOf<R>::type v;
    v.x = phi;
    v.y = T;
    phiT[c] = v;
  };
  if (nb) body(std::true_type{});
  else body(std::false_type{});
}

// One in-place step of every cell (the generic kernel's tiles and z-march),
// with the stencil tiles read from the (phi, T) field of aa_moments_kernel.
template <class S, int QH, int QF>
__global__ void __launch_bounds__(NTHREADS)
aa_step_kernel(const DevParams P, const StepPtrs<S, typename Store<S>::R> A,
               const typename PairOf<typename Store<S>::R>::type* __restrict__ phiT, int nb, int zchunk,
               int mode) {
  using R = typename Store<S>::R;
  __shared__ R s_phi[3][HP];
  __shared__ R s_T[3][HP];
  S* const hb = const_cast<S*>(A.h_src);
  S* const gbase = const_cast<S*>(A.g_src);
  S* const fb = const_cast<S*>(A.f_src);
  const bool NB = nb != 0;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, P.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < P.nx) && (y < P.ny);
  const R shh = (R)RP<R>(P).shift_h, shf = (R)RP<R>(P).shift_f;

  // phi and T on the (TX+2) x (TY+2) plane zp -> slot, from the field
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
      const auto v = phiT[cell_index(P, gx, gy, zz)];
      R phi = v.x, T = v.y;
      if (ghost) {
        T = (R)2 * wall_T<R>(P, gx, zp < 0) - T;
        if (P.wetting) phi = wet_ghost<R>(phi, wall_k<R>(P, zp < 0 ? 0 : 1));
      }
      s_phi[slot][k] = phi;
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
      const R phi = s_phi[sc][c0], Tc = s_T[sc][c0];
      auto geth = [&](auto I) {
        constexpr int i = decltype(I)::value;
        return aa_get<QH, false, i>(P, hb, x, y, z, NB, shh) + phi * pull_wall_term<QH, i, R>(P, z);
      };
      auto getg = [&](auto I) {
        constexpr int i = decltype(I)::value;
        return aa_get<27, false, i>(P, gbase, x, y, z, NB, (R)0) + pull_wall_term<27, i, R>(P, z);
      };
      auto getf = [&](auto I) {
        if constexpr (QF > 0) return aa_get<QF, true, decltype(I)::value>(P, fb, x, y, z, NB, shf);
        else return (R)0;
      };
      auto puth = [&](auto I, R v) { Store<S>::st(hb + aa_put_index<QH, decltype(I)::value>(P, x, y, z, NB), v); };
      auto putg = [&](auto I, R v) { Store<S>::st(gbase + aa_put_index<27, decltype(I)::value>(P, x, y, z, NB), v); };
      auto putf = [&](auto I, R v) {
        if constexpr (QF > 0) Store<S>::st(fb + aa_put_index<QF, decltype(I)::value>(P, x, y, z, NB), v);
      };
      // a2-a10 as in cell_update, with the in-place destinations
      const GMoments<R> m = g_moments<R>(getg);
      if (mode & MODE_SAVE) {
        save_stencil<S>(P, A, cell, phi, Tc, fd);
        save_moments<S>(P, A, cell, m);
      }
      CellForce<R> F = cell_force<R>(P, x, y, z, phi, Tc, fd.gpx, fd.gpy, fd.gpz, fd.lp, fd.gtx, fd.gty, fd.gtz);
      if (P.rho_ratio) density_ratio_accel<R>(P, phi, fd.gpx, fd.gpy, fd.gpz, m, F);
      const CellFlow<R> fl = cell_velocity<R>(F.ax, F.ay, F.az, F.rho, m.jx, m.jy, m.jz);
      cell_outputs<S>(P, A, x, y, z, cell, mode, phi, Tc, m.pst, fl, dsum);
      if (mode & MODE_COLLIDE) {
        const size_t pcell = pdf_index(P, x, y, z);
        collide_g<S>(P, A, pcell, phi, m, fl, putg);
        collide_h<S, QH>(P, A, pcell, phi, fd.gpx, fd.gpy, fd.gpz, fl, geth, puth);
        if (P.alpha_ratio)
          collide_f<S, QF, true>(P, A, x, y, z, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, fl,
                                 getf, putf);
        else
          collide_f<S, QF, false>(P, A, x, y, z, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, fl,
                                  getf, putf);
      }
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

// In-place swap of the opposite slots of every cell: turns populations stored
// p_i(x) at slot i (two-grid layout) into the even-level AA layout
// F[opp(i)](x) = p_i(x), and back.
template <class S, int Q>
__global__ void aa_swap_kernel(const DevParams P, S* __restrict__ base) {
  const size_t N = (size_t)P.N;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % P.nx), y = (int)((c / P.nx) % P.ny), z = (int)(c / ((size_t)P.nx * P.ny));
    const size_t pc = pdf_index(P, x, y, z);
    static_for<1, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (pair_first<Q>(i)) {
        constexpr int j = opp<Q>(i);
        S* a = base + (size_t)i * P.Np + pc;
        S* b = base + (size_t)j * P.Np + pc;
        const S t = *a;
        *a = *b;
        *b = t;
      }
    });
  }
}

// AA layout of the current level <-> dense FP64 p_i(x) [Q][N] (un-shifted).
template <class S, int Q>
__global__ void aa_to_f64_kernel(const DevParams P, const S* __restrict__ base, double* __restrict__ dst,
                                 double shift, int odd_level) {
  const size_t N = (size_t)P.N;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % P.nx), y = (int)((c / P.nx) % P.ny), z = (int)(c / ((size_t)P.nx * P.ny));
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      // where p_i(x) lives: the destination of direction i's last scatter
      const size_t at = aa_put_index<Q, i>(P, x, y, z, odd_level != 0);
      dst[(size_t)i * N + c] = (double)Store<S>::ld(base + at) + weight<Q>(i) * shift;
    });
  }
}

template <class S, int Q>
__global__ void f64_to_aa_kernel(const DevParams P, const double* __restrict__ src, S* __restrict__ base,
                                 double shift, int odd_level) {
  using R = typename Store<S>::R;
  const size_t N = (size_t)P.N;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % P.nx), y = (int)((c / P.nx) % P.ny), z = (int)(c / ((size_t)P.nx * P.ny));
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const size_t at = aa_put_index<Q, i>(P, x, y, z, odd_level != 0);
      Store<S>::st(base + at, (R)(src[(size_t)i * N + c] - weight<Q>(i) * shift));
    });
  }
}


}  // namespace lbm
