// Instantiations of the precision-generic auxiliary kernels (RK stages, PDF
// conversion, diagnostics reduction).
#include "launchers.h"
#include "lbm_aux.cuh"
#include "lbm_aa.cuh"
#include "lbm_skew.cuh"

namespace lbm {

template <class S>
void launch_rk_stage(const DevParams& P, const typename Store<S>::R* psi, typename Store<S>::R* T,
                     const typename Store<S>::R* u, const typename Store<S>::R* phi,
                     typename Store<S>::R* acc, typename Store<S>::R* out, int kind, cudaStream_t st) {
  const long long blocks = (P.N + 255) / 256;
  const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
  rk_stage_kernel<typename Store<S>::R><<<grid, 256, 0, st>>>(P, psi, T, u, phi, acc, out, kind);
}

template <class S, int Q>
static void convert_q(const DevParams& P, bool to_f64, void* pdf, double* f64, double shift, cudaStream_t st) {
  const long long blocks = ((long long)Q * P.N + 255) / 256;
  const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
  if (to_f64) pdf_to_f64_kernel<S, Q><<<grid, 256, 0, st>>>(P, (const S*)pdf, f64, shift);
  else f64_to_pdf_kernel<S, Q><<<grid, 256, 0, st>>>(P, f64, (S*)pdf, shift);
}

template <class S>
void launch_pdf_convert(const DevParams& P, int Q, bool to_f64, void* pdf, double* f64, double shift,
                        cudaStream_t st) {
  switch (Q) {
    case 7: convert_q<S, 7>(P, to_f64, pdf, f64, shift, st); break;
    case 15: convert_q<S, 15>(P, to_f64, pdf, f64, shift, st); break;
    case 19: convert_q<S, 19>(P, to_f64, pdf, f64, shift, st); break;
    default: convert_q<S, 27>(P, to_f64, pdf, f64, shift, st); break;
  }
}

template <class S, int Q>
static void aa_swap_q(const DevParams& P, S* base, cudaStream_t st) {
  const long long blocks = (P.N + 255) / 256;
  const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
  aa_swap_kernel<S, Q><<<grid, 256, 0, st>>>(P, base);
}

template <class S>
void launch_aa_swap(const DevParams& P, int Q, S* base, cudaStream_t st) {
  switch (Q) {
    case 7: aa_swap_q<S, 7>(P, base, st); break;
    case 15: aa_swap_q<S, 15>(P, base, st); break;
    case 19: aa_swap_q<S, 19>(P, base, st); break;
    default: aa_swap_q<S, 27>(P, base, st); break;
  }
}

template <class S, int Q>
static void aa_convert_q(const DevParams& P, bool to_f64, void* pdf, double* f64, double shift, int odd,
                         cudaStream_t st) {
  const long long blocks = (P.N + 255) / 256;
  const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
  if (to_f64) aa_to_f64_kernel<S, Q><<<grid, 256, 0, st>>>(P, (const S*)pdf, f64, shift, odd);
  else f64_to_aa_kernel<S, Q><<<grid, 256, 0, st>>>(P, f64, (S*)pdf, shift, odd);
}

template <class S>
void launch_aa_convert(const DevParams& P, int Q, bool to_f64, void* pdf, double* f64, double shift,
                       int odd_level, cudaStream_t st) {
  switch (Q) {
    case 7: aa_convert_q<S, 7>(P, to_f64, pdf, f64, shift, odd_level, st); break;
    case 15: aa_convert_q<S, 15>(P, to_f64, pdf, f64, shift, odd_level, st); break;
    case 19: aa_convert_q<S, 19>(P, to_f64, pdf, f64, shift, odd_level, st); break;
    default: aa_convert_q<S, 27>(P, to_f64, pdf, f64, shift, odd_level, st); break;
  }
}

template <class S>
void launch_halo_x(const DevParams& P, S* set, int nq, typename Store<S>::R* T, int x0, int w, void* buf,
                   size_t t_off, bool to_buf, cudaStream_t st) {
  const long long total = (long long)(nq + (T ? 1 : 0)) * P.nz * P.ny * w;
  const long long blocks = (total + 255) / 256;
  const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
  halo_x_kernel<S><<<grid, 256, 0, st>>>(P, set, nq, T, x0, w, (unsigned char*)buf, t_off, to_buf ? 1 : 0);
}

template <class S>
void launch_ghost_fill(const DevParams& P, void* buf, int nq, cudaStream_t st, const unsigned char* sides) {
  constexpr int V = 16 / (int)sizeof(S);
  const int per_plane = P.NYP + 2 * P.GY * ((P.nx + V - 1) / V);
  const int bx = (per_plane + 127) / 128;
  GhostSides g;
  for (int q = 0; q < kMaxSetArrays; ++q) g.m[q] = (sides && q < nq) ? sides[q] : (unsigned char)15;
  // grid y = z and grid z = direction; nz is bounded by 65535 in the API
  ghost_fill_kernel<S><<<dim3(bx, P.nz, nq), 128, 0, st>>>(P, (S*)buf, g);
}

template <class S, int QH>
static size_t bulk_bytes_qf(int qf) {
  switch (qf) {
    case 0: return BulkSmem<S, QH, 0>::bytes;
    case 7: return BulkSmem<S, QH, 7>::bytes;
    case 15: return BulkSmem<S, QH, 15>::bytes;
    case 19: return BulkSmem<S, QH, 19>::bytes;
    default: return BulkSmem<S, QH, 27>::bytes;
  }
}

template <class S>
static size_t bulk_bytes_s(int qh, int qf) {
  return qh == 15 ? bulk_bytes_qf<S, 15>(qf) : bulk_bytes_qf<S, 27>(qf);
}

template <class S, int QH, int QF>
static constexpr size_t skew_bytes_one() {
  return skew_fits<S, QH, QF>() ? SkewSmem<S, QH, QF>::bytes : 0;
}

template <class S, int QH>
static size_t skew_bytes_qf(int qf) {
  switch (qf) {
    case 0: return skew_bytes_one<S, QH, 0>();
    case 7: return skew_bytes_one<S, QH, 7>();
    case 15: return skew_bytes_one<S, QH, 15>();
    case 19: return skew_bytes_one<S, QH, 19>();
    default: return skew_bytes_one<S, QH, 27>();
  }
}

template <class S, int QH, int QF>
static constexpr size_t aa_skew_bytes_one() {
  return skew_fits<S, QH, QF, 1>() ? SkewSmem<S, QH, QF, 1>::bytes : 0;
}

template <class S, int QH>
static size_t aa_skew_bytes_qf(int qf) {
  switch (qf) {
    case 0: return aa_skew_bytes_one<S, QH, 0>();
    case 7: return aa_skew_bytes_one<S, QH, 7>();
    case 15: return aa_skew_bytes_one<S, QH, 15>();
    case 19: return aa_skew_bytes_one<S, QH, 19>();
    default: return aa_skew_bytes_one<S, QH, 27>();
  }
}

size_t aa_skew_smem_bytes(int prec, int qh, int qf) {
  if (prec == 0) return qh == 15 ? aa_skew_bytes_qf<double, 15>(qf) : aa_skew_bytes_qf<double, 27>(qf);
  if (prec == 1) return qh == 15 ? aa_skew_bytes_qf<float, 15>(qf) : aa_skew_bytes_qf<float, 27>(qf);
  return qh == 15 ? aa_skew_bytes_qf<__half, 15>(qf) : aa_skew_bytes_qf<__half, 27>(qf);
}

size_t skew_smem_bytes(int prec, int qh, int qf) {
  if (prec == 0) return qh == 15 ? skew_bytes_qf<double, 15>(qf) : skew_bytes_qf<double, 27>(qf);
  if (prec == 1) return qh == 15 ? skew_bytes_qf<float, 15>(qf) : skew_bytes_qf<float, 27>(qf);
  return qh == 15 ? skew_bytes_qf<__half, 15>(qf) : skew_bytes_qf<__half, 27>(qf);
}

size_t bulk_smem_bytes(int prec, int qh, int qf) {
  if (prec == 0) return bulk_bytes_s<double>(qh, qf);
  if (prec == 1) return bulk_bytes_s<float>(qh, qf);
  return bulk_bytes_s<__half>(qh, qf);
}

int bulk_tile_cols(int prec) {
  return prec == 0 ? BulkGeom<double>::TXB : (prec == 1 ? BulkGeom<float>::TXB : BulkGeom<__half>::TXB);
}

int bulk_box_cols(int prec) {
  return prec == 0 ? BulkGeom<double>::W : (prec == 1 ? BulkGeom<float>::W : BulkGeom<__half>::W);
}

template <class S, int QH>
static int bulk_rows_qf(int qf) {
  switch (qf) {
    case 0: return BulkSmem<S, QH, 0>::G::TYB;
    case 7: return BulkSmem<S, QH, 7>::G::TYB;
    case 15: return BulkSmem<S, QH, 15>::G::TYB;
    case 19: return BulkSmem<S, QH, 19>::G::TYB;
    default: return BulkSmem<S, QH, 27>::G::TYB;
  }
}

template <class S>
static int bulk_rows_s(int qh, int qf) {
  return qh == 15 ? bulk_rows_qf<S, 15>(qf) : bulk_rows_qf<S, 27>(qf);
}

int bulk_tile_rows(int prec, int qh, int qf) {
  if (prec == 0) return bulk_rows_s<double>(qh, qf);
  if (prec == 1) return bulk_rows_s<float>(qh, qf);
  return bulk_rows_s<__half>(qh, qf);
}

void launch_diag_finalize(const double* partials, int nblocks, double* out, cudaStream_t st) {
  diag_finalize_kernel<<<1, 256, 0, st>>>(partials, nblocks, out);
}

template void launch_rk_stage<double>(const DevParams&, const double*, double*, const double*,
                                      const double*, double*, double*, int, cudaStream_t);
template void launch_rk_stage<float>(const DevParams&, const float*, float*, const float*, const float*,
                                     float*, float*, int, cudaStream_t);
template void launch_rk_stage<__half>(const DevParams&, const float*, float*, const float*, const float*,
                                      float*, float*, int, cudaStream_t);
template void launch_pdf_convert<double>(const DevParams&, int, bool, void*, double*, double, cudaStream_t);
template void launch_pdf_convert<float>(const DevParams&, int, bool, void*, double*, double, cudaStream_t);
template void launch_pdf_convert<__half>(const DevParams&, int, bool, void*, double*, double, cudaStream_t);
template void launch_aa_swap<double>(const DevParams&, int, double*, cudaStream_t);
template void launch_aa_swap<float>(const DevParams&, int, float*, cudaStream_t);
template void launch_aa_swap<__half>(const DevParams&, int, __half*, cudaStream_t);
template void launch_aa_convert<double>(const DevParams&, int, bool, void*, double*, double, int, cudaStream_t);
template void launch_aa_convert<float>(const DevParams&, int, bool, void*, double*, double, int, cudaStream_t);
template void launch_aa_convert<__half>(const DevParams&, int, bool, void*, double*, double, int, cudaStream_t);
template void launch_halo_x<double>(const DevParams&, double*, int, double*, int, int, void*, size_t, bool,
                                    cudaStream_t);
template void launch_halo_x<float>(const DevParams&, float*, int, float*, int, int, void*, size_t, bool,
                                   cudaStream_t);
template void launch_halo_x<__half>(const DevParams&, __half*, int, float*, int, int, void*, size_t, bool,
                                    cudaStream_t);
template void launch_ghost_fill<double>(const DevParams&, void*, int, cudaStream_t,
                                          const unsigned char*);
template void launch_ghost_fill<float>(const DevParams&, void*, int, cudaStream_t,
                                          const unsigned char*);
template void launch_ghost_fill<__half>(const DevParams&, void*, int, cudaStream_t,
                                          const unsigned char*);

}  // namespace lbm
