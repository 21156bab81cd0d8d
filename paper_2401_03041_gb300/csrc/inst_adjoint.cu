// inst_adjoint.cu - instantiations and launchers of the adjoint-step kernels
// (FP64; h on D3Q15 or D3Q27, thermal LB D3Q7).
#include "launchers.h"
#include "lbm_adjoint.cuh"

namespace lbm {

namespace {

int grid_1d(size_t work) {
  const size_t b = (work + 255) / 256;
  return (int)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

bool adj_supported(int qh, int qf) { return (qh == 15 || qh == 27) && qf == 7; }

// plane-indexed grids: x over nx * ny (< 2^31), y = z (<= 65535)
static unsigned plane_blocks(const DevParams& P) {
  return (unsigned)(((size_t)P.nx * P.ny + 255) / 256);
}

void adj_cell(const DevParams& P, const AdjPtrs& A, int qh, int qf, cudaStream_t st) {
  (void)qf;
  const dim3 grid(plane_blocks(P), P.nz);
  if (qh == 15) adj_point_kernel<15, 7><<<grid, 256, 0, st>>>(P, A);
  else adj_point_kernel<27, 7><<<grid, 256, 0, st>>>(P, A);
}

void adj_fields(const DevParams& P, const AdjPtrs& A, cudaStream_t st) {
  adj_fields_kernel<<<dim3(plane_blocks(P), P.nz), 256, 0, st>>>(P, A);
}

void adj_pull(const DevParams& P, const AdjPtrs& A, int qh, int qf, cudaStream_t st) {
  const dim3 grid(plane_blocks(P), P.nz);
  if (qh == 15) adj_pull_kernel<15, 7><<<grid, 256, 0, st>>>(P, A);
  else adj_pull_kernel<27, 7><<<grid, 256, 0, st>>>(P, A);
}

void adj_seed(const DevParams& P, const double* dJdphi, double* lam, int qh, int qf, cudaStream_t st) {
  const size_t work = (size_t)(qh + 27 + qf) * (size_t)P.N;
  if (qh == 15) adj_seed_kernel<15, 7><<<grid_1d(work), 256, 0, st>>>(P, dJdphi, lam);
  else adj_seed_kernel<27, 7><<<grid_1d(work), 256, 0, st>>>(P, dJdphi, lam);
}

void adj_centroid_seed(const DevParams& P, double mass, const double* c, const double* t, double* out,
                       cudaStream_t st) {
  adj_centroid_seed_kernel<<<grid_1d((size_t)P.N), 256, 0, st>>>(P, mass, c[0], c[1], c[2], t[0], t[1], t[2],
                                                                  out);
}

void adj_patch_grad(const DevParams& P, const double* lam, double* dJdI, int qh, int qf, cudaStream_t st) {
  if (P.npatch < 1) return;
  if (qh == 15) adj_patch_grad_kernel<15, 7><<<P.npatch, 256, 0, st>>>(P, lam, dJdI);
  else adj_patch_grad_kernel<27, 7><<<P.npatch, 256, 0, st>>>(P, lam, dJdI);
}

}  // namespace lbm
