// launchers.h - host-side launch entry points of the device kernels.  The
// kernel templates are instantiated in the inst_*.cu translation units (one
// per storage precision) so that they compile in parallel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// use_bulk: the bulk kernel (tensor-TMA staging; tiles of BulkSmem<S, QH, QF>::G) if
// its shared memory fits, else the generic kernel (TX x TY tiles).
// Tensor maps of the current source PDF buffers (bulk kernel only).
struct TMaps {
  CUtensorMap h, g, f;
};

// use_bulk: 0 generic kernel, 1 bulk kernel, 2 skewed kernel where its layout
// fits (lbm_skew.cuh; the bulk kernel otherwise and with a density ratio).
// grid / zchunk: the generic kernel's launch (TX x TY tiles, z-chunks);
// sched: the bulk kernels' work assignment (one-dimensional grid).
template <class S, int QH, int QF>
void launch_step(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A, const TMaps& maps,
                 dim3 grid, int zchunk, const BulkSched& sched, int mode, int use_bulk, cudaStream_t st);

// Refresh the periodic ghost cells of nq consecutive padded directions at buf:
// the sides that sides[q] selects for array q (bits of GhostSides in
// lbm_aux.cuh; null: every side, the whole periodic extension).
template <class S>
void launch_ghost_fill(const DevParams& P, void* buf, int nq, cudaStream_t st,
                       const unsigned char* sides = nullptr);

// Dynamic shared memory of the bulk kernel for (precision, q_phase, q_f),
// and the largest a CTA may use; also its tile height.
size_t bulk_smem_bytes(int prec, int qh, int qf);
size_t skew_smem_bytes(int prec, int qh, int qf);   // 0: the skewed layout does not fit
size_t aa_skew_smem_bytes(int prec, int qh, int qf);   // the same for its in-place variant
int bulk_tile_rows(int prec, int qh, int qf);
int bulk_tile_cols(int prec);
int bulk_box_cols(int prec);   // staged row length W of the bulk kernel
constexpr size_t kMaxDynSmem = 232448;

// In-place (AA) layout: (phi, T) pass then the step, on the generic tiles;
// nb = 1 for a step from an even level.
template <class S, int QH, int QF>
void launch_aa_step(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A, void* phiT, int nb,
                    dim3 grid, int zchunk, int mode, cudaStream_t st);
// The same on the skewed kernel's tensor-TMA tiles (maps: TYB-row boxes over
// the one set): (phi, T) pass; from an even level the periodic ghosts are
// refreshed first and folded back after the step.
template <class S, int QH, int QF>
void launch_aa_tiled(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A, const TMaps& maps,
                     void* phiT, int nb, const BulkSched& sched, int mode, cudaStream_t st);
template <class S>
void launch_aa_swap(const DevParams& P, int Q, S* base, cudaStream_t st);
template <class S>
void launch_aa_convert(const DevParams& P, int Q, bool to_f64, void* pdf, double* f64, double shift,
                       int odd_level, cudaStream_t st);

// Slab halo columns <-> contiguous buffer (see halo_x_kernel).
template <class S>
void launch_halo_x(const DevParams& P, S* set, int nq, typename Store<S>::R* T, int x0, int w, void* buf,
                   size_t t_off, bool to_buf, cudaStream_t st);

template <class S, int QH, int QF>
void launch_init(const DevParams& P, const double* drops, int nd, S* h, S* g, S* f,
                 typename Store<S>::R* T, cudaStream_t st);

template <class S>
void launch_rk_stage(const DevParams& P, const typename Store<S>::R* psi, typename Store<S>::R* T,
                     const typename Store<S>::R* u, const typename Store<S>::R* phi,
                     typename Store<S>::R* acc, typename Store<S>::R* out, int kind, cudaStream_t st);

template <class S>
void launch_pdf_convert(const DevParams& P, int Q, bool to_f64, void* pdf, double* f64, double shift,
                        cudaStream_t st);

void launch_diag_finalize(const double* partials, int nblocks, double* out, cudaStream_t st);

}  // namespace lbm

#include "../../include/lbm.h"

namespace lbm {

// Adjoint step (FP64; thermal LB D3Q7/15/19/27 or RK2/RK4; inst_adjoint.cu).
// qf = 0 selects the RK energy solvers, whose state holds the T field in
// place of f (one slot of N values after h and g in the adjoint arrays).
bool adj_supported(int qh, int qf);
// rk_lu: RK only, the adjoint of u through the RK update ([3][N]), added to
// the velocity adjoint of pass A.
void adj_cell(const DevParams& P, const AdjPtrs& A, int qh, int qf, const double* rk_lu, cudaStream_t st);
void adj_fields(const DevParams& P, const AdjPtrs& A, cudaStream_t st);
// rk_lT: RK only, the adjoint of T^n through the RK update, added to the
// stencil adjoint of T in the T slot of lam_out.
void adj_pull(const DevParams& P, const AdjPtrs& A, int qh, int qf, const double* rk_lT, cudaStream_t st);
void adj_seed(const DevParams& P, const double* dJdphi, double* lam, int qh, int qf, cudaStream_t st);
void adj_centroid_seed(const DevParams& P, double mass, const double* c, const double* t, double* out,
                       cudaStream_t st);
// dJ/dI_k += sum over the cells of patch k of the intensity's adjoint:
// sum_i w_i lam_{f,i} (LB: lam = lam^{n+1}), or the per-cell adjoint of q_T
// (RK: lam = AdjRK::lq).
void adj_patch_grad(const DevParams& P, const double* lam, double* dJdI, int qh, int qf, cudaStream_t st);

// Buffers of the RK part of an adjoint step (N doubles each unless noted).
struct AdjRK {
  double* u;        // [3][N]: u of the step, from the saved intermediates
  double* psi[3];   // stage inputs psi_k = T + c_k K_{k-1}, k = 2, 3, 4 (RK2: psi[0])
  double* lk[2];    // adjoints of the stage slopes K_k (ping-pong)
  double* lT;       // adjoint of T^n through the RK update
  double* lu;       // [3][N]: adjoint of u through the RK update
  double* lq;       // adjoint of the heat-source density q_T (all stages)
};
// The RK update's adjoint for one step: from lam_T' = dJ/dT^{n+1} (lamT,
// N values) and the step's intermediates, fills R.lT, R.lu and R.lq.
void adj_rk(const DevParams& P, const double* save, const double* lamT, const AdjRK& R, bool rk4,
            cudaStream_t st);

// Set the calling thread's lbm_last_error message and return s.
lbm_status set_error(lbm_status s, const char* msg);

}  // namespace lbm
