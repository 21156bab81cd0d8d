// inst_step.cuh - explicit instantiations of the step-kernel launchers for one
// storage type LBM_S and one phase-field stencil LBM_QH (set by the including
// translation unit), for the energy solvers of part LBM_QF_PART (QF = 0: RK;
// 7/15/19/27: LB).
#pragma once

#include "launchers.h"
#include "lbm_aux.cuh"
#include "lbm_aa.cuh"
#include "lbm_skew.cuh"

namespace lbm {

template <class S, int QH, int QF>
void launch_step(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A, const TMaps& maps,
                 dim3 grid, int zchunk, const BulkSched& sched, int mode, int use_bulk, cudaStream_t st) {
  constexpr size_t bytes = BulkSmem<S, QH, QF>::bytes;
  if constexpr (bytes <= kMaxDynSmem) {
    const dim3 bgrid((unsigned)bulk_sched_blocks(sched));
    if constexpr (skew_fits<S, QH, QF>()) {
      // the skewed kernel, except with a density ratio (its forces need the
      // moments and the stencils of one plane together)
      if (use_bulk == 2 && !P.rho_ratio) {
        constexpr size_t sbytes = SkewSmem<S, QH, QF>::bytes;
        static bool sattr_set = false;
        if (!sattr_set) {
          cudaFuncSetAttribute(step_skew_kernel<S, QH, QF, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sbytes);
          cudaFuncSetAttribute(step_skew_kernel<S, QH, QF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sbytes);
          sattr_set = true;
        }
        if (P.alpha_ratio || P.tw_waves || P.wall_ext || P.sub)
          step_skew_kernel<S, QH, QF, true><<<bgrid, SkewSmem<S, QH, QF>::G::NTHR, sbytes, st>>>(
              P, A, maps.h, maps.g, maps.f, sched, mode, nullptr);
        else
          step_skew_kernel<S, QH, QF, false><<<bgrid, SkewSmem<S, QH, QF>::G::NTHR, sbytes, st>>>(
              P, A, maps.h, maps.g, maps.f, sched, mode, nullptr);
        return;
      }
    }
    if (use_bulk) {
      static bool attr_set = false;
      if (!attr_set) {
        cudaFuncSetAttribute(step_bulk_kernel<S, QH, QF, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
        cudaFuncSetAttribute(step_bulk_kernel<S, QH, QF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
        attr_set = true;
      }
      if (P.alpha_ratio || P.tw_waves || P.rho_ratio || P.wall_ext || P.sub)
        step_bulk_kernel<S, QH, QF, true><<<bgrid, BulkSmem<S, QH, QF>::G::NTHR, bytes, st>>>(
            P, A, maps.h, maps.g, maps.f, sched, mode);
      else
        step_bulk_kernel<S, QH, QF, false><<<bgrid, BulkSmem<S, QH, QF>::G::NTHR, bytes, st>>>(
            P, A, maps.h, maps.g, maps.f, sched, mode);
      return;
    }
  }
  step_kernel<S, QH, QF><<<grid, dim3(TX, TY), 0, st>>>(P, A, zchunk, mode);
}

template <class S, int QH, int QF>
void launch_aa_step(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A, void* phiT, int nb,
                    dim3 grid, int zchunk, int mode, cudaStream_t st) {
  using R = typename Store<S>::R;
  using P2 = typename PairOf<R>::type;
  const dim3 mgrid((unsigned)(((P.nx + kAaRowBlock - 1) / kAaRowBlock) * P.ny), (unsigned)P.nz);
  aa_moments_kernel<S, QH, QF><<<mgrid, kAaRowBlock, 0, st>>>(P, A.h_src, A.f_src, A.T, nb, (P2*)phiT);
  aa_step_kernel<S, QH, QF><<<grid, dim3(TX, TY), 0, st>>>(P, A, (const P2*)phiT, nb, zchunk, mode);
}

template <class S, int QH, int QF>
void launch_aa_tiled(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A, const TMaps& maps,
                     void* phiT, int nb, const BulkSched& sched, int mode, cudaStream_t st) {
  using R = typename Store<S>::R;
  using P2 = typename PairOf<R>::type;
  if constexpr (skew_fits<S, QH, QF, 1>()) {
    constexpr size_t sbytes = SkewSmem<S, QH, QF, 1>::bytes;
    constexpr int nthr = SkewSmem<S, QH, QF, 1>::G::NTHR;
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(step_skew_kernel<S, QH, QF, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sbytes);
      cudaFuncSetAttribute(step_skew_kernel<S, QH, QF, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sbytes);
      cudaFuncSetAttribute(step_skew_kernel<S, QH, QF, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sbytes);
      cudaFuncSetAttribute(step_skew_kernel<S, QH, QF, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sbytes);
      attr_set = true;
    }
    S* set = const_cast<S*>(A.h_src);
    // destination pointers of the level: F[i] shifted by c_i's x and y
    // (even) or F[opp(i)] (odd); the kernel adds the cell and, for even
    // levels, the z offset of the destination plane
    StepPtrs<S, R> B = A;
    const long long np = P.Np, nxp = P.NXP;
    auto point = [&](auto qtag, const S* base, S** out) {
      constexpr int Q = decltype(qtag)::value;
      S* b = const_cast<S*>(base);
      for (int i = 0; i < Q; ++i)
        out[i] = nb ? b + (long long)i * np + cx<Q>(i) + (long long)cy<Q>(i) * nxp : b + (long long)opp<Q>(i) * np;
    };
    point(std::integral_constant<int, QH>{}, A.h_src, B.hd);
    point(std::integral_constant<int, 27>{}, A.g_src, B.gd);
    if constexpr (QF > 0) point(std::integral_constant<int, QF>{}, A.f_src, B.fd);
    const dim3 bgrid((unsigned)bulk_sched_blocks(sched));
    // (phi, T) of the level from TMA-staged boxes (as plain loads the gathers
    // of an even level, shifted rows of three planes, ran at half the copy rate)
    constexpr size_t mbytes = AaMomSmem<S, QH, QF>::bytes;
    constexpr int mthr = AaMomSmem<S, QH, QF>::G::NT;
    static bool mattr_set = false;
    if (!mattr_set) {
      cudaFuncSetAttribute(aa_moments_tiled_kernel<S, QH, QF, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mbytes);
      cudaFuncSetAttribute(aa_moments_tiled_kernel<S, QH, QF, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mbytes);
      cudaFuncSetAttribute(aa_moments_tiled_kernel<S, QH, QF, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mbytes);
      cudaFuncSetAttribute(aa_moments_tiled_kernel<S, QH, QF, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mbytes);
      mattr_set = true;
    }
    // model extensions (conductivity / heat-capacity ratio, modulated wall,
    // moving walls, wetting) in their own instantiation, as on two grids
    auto go = [&](auto ext_tag) {
      constexpr bool EXT = decltype(ext_tag)::value;
      if (nb) {
        launch_ghost_fill<S>(P, set, QH + 27 + QF, st);
        aa_moments_tiled_kernel<S, QH, QF, 2, EXT><<<bgrid, mthr, mbytes, st>>>(P, maps.h, maps.f, sched, A.T,
                                                                                (P2*)phiT, A.error_flag);
        step_skew_kernel<S, QH, QF, EXT, 2><<<bgrid, nthr, sbytes, st>>>(P, B, maps.h, maps.g, maps.f, sched, mode,
                                                                          (const P2*)phiT);
        aa_fold_kernel<S, QH, QF><<<dim3((P.nx + P.ny + 127) / 128, P.nz, QH + 27 + QF), 128, 0, st>>>(P, set);
      } else {
        aa_moments_tiled_kernel<S, QH, QF, 1, EXT><<<bgrid, mthr, mbytes, st>>>(P, maps.h, maps.f, sched, A.T,
                                                                                (P2*)phiT, A.error_flag);
        step_skew_kernel<S, QH, QF, EXT, 1><<<bgrid, nthr, sbytes, st>>>(P, B, maps.h, maps.g, maps.f, sched, mode,
                                                                          (const P2*)phiT);
      }
    };
    if (P.alpha_ratio || P.tw_waves || P.wall_ext) go(std::true_type{});
    else go(std::false_type{});
  }
}

template <class S, int QH, int QF>
void launch_init(const DevParams& P, const double* drops, int nd, S* h, S* g, S* f,
                 typename Store<S>::R* T, cudaStream_t st) {
  const dim3 grid((P.nx + kInitTX - 1) / kInitTX, (P.ny + kInitTY - 1) / kInitTY,
                  (P.nz + kInitTZ - 1) / kInitTZ);
  init_kernel<S, QH, QF><<<grid, kInitTX * kInitTY * kInitTZ, 0, st>>>(P, drops, nd, h, g, f, T);
}

#define LBM_INST(QF)                                                                          \
  template void launch_step<LBM_S, LBM_QH, QF>(const DevParams&,                              \
                                               const StepPtrs<LBM_S, Store<LBM_S>::R>&,       \
                                               const TMaps&, dim3, int, const BulkSched&, int, int, \
                                               cudaStream_t);                                 \
  template void launch_aa_step<LBM_S, LBM_QH, QF>(const DevParams&,                           \
                                                  const StepPtrs<LBM_S, Store<LBM_S>::R>&,    \
                                                  void*, int, dim3, int, int, cudaStream_t);  \
  template void launch_aa_tiled<LBM_S, LBM_QH, QF>(const DevParams&,                          \
                                                   const StepPtrs<LBM_S, Store<LBM_S>::R>&,   \
                                                   const TMaps&, void*, int, const BulkSched&, \
                                                   int, cudaStream_t);                        \
  template void launch_init<LBM_S, LBM_QH, QF>(const DevParams&, const double*, int, LBM_S*,  \
                                               LBM_S*, LBM_S*, Store<LBM_S>::R*, cudaStream_t);
// LBM_QF_PART (set by the including unit) splits the energy solvers over two
// translation units so that they compile in parallel: 0 = RK, D3Q7, D3Q15;
// 1 = D3Q19, D3Q27.
#if LBM_QF_PART == 0
LBM_INST(0)
LBM_INST(7)
LBM_INST(15)
#else
LBM_INST(19)
LBM_INST(27)
#endif
#undef LBM_INST

}  // namespace lbm
