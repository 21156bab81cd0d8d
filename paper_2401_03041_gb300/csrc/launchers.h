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

// Refresh the periodic ghost cells of nq consecutive padded directions at buf.
template <class S>
void launch_ghost_fill(const DevParams& P, void* buf, int nq, cudaStream_t st);

// Dynamic shared memory of the bulk kernel for (precision, q_phase, q_f),
// and the largest a CTA may use; also its tile height.
size_t bulk_smem_bytes(int prec, int qh, int qf);
size_t skew_smem_bytes(int prec, int qh, int qf);   // 0: the skewed layout does not fit
int bulk_tile_rows(int prec, int qh, int qf);
int bulk_tile_cols(int prec);
int bulk_box_cols(int prec);   // staged row length W of the bulk kernel
constexpr size_t kMaxDynSmem = 232448;

// In-place (AA) layout: (phi, T) pass then the step, on the generic tiles;
// nb = 1 for a step from an even level.
template <class S, int QH, int QF>
void launch_aa_step(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A, void* phiT, int nb,
                    dim3 grid, int zchunk, int mode, cudaStream_t st);
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

// Adjoint step (FP64, LB thermal; inst_adjoint.cu).
bool adj_supported(int qh, int qf);
void adj_cell(const DevParams& P, const AdjPtrs& A, int qh, int qf, cudaStream_t st);
void adj_fields(const DevParams& P, const AdjPtrs& A, cudaStream_t st);
void adj_pull(const DevParams& P, const AdjPtrs& A, int qh, int qf, cudaStream_t st);
void adj_seed(const DevParams& P, const double* dJdphi, double* lam, int qh, int qf, cudaStream_t st);
void adj_centroid_seed(const DevParams& P, double mass, const double* c, const double* t, double* out,
                       cudaStream_t st);
void adj_patch_grad(const DevParams& P, const double* lam, double* dJdI, int qh, int qf, cudaStream_t st);

// Set the calling thread's lbm_last_error message and return s.
lbm_status set_error(lbm_status s, const char* msg);

}  // namespace lbm
