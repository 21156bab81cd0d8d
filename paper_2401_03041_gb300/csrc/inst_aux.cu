// Instantiations of the precision-generic auxiliary kernels (RK stages, PDF
// conversion, diagnostics reduction).
#include "launchers.h"
#include "lbm_aux.cuh"

namespace lbm {

template <class S>
void launch_rk_stage(const DevParams& P, const typename Store<S>::R* psi, typename Store<S>::R* T,
                     const typename Store<S>::R* u, typename Store<S>::R* acc,
                     typename Store<S>::R* out, int kind, cudaStream_t st) {
  const long long blocks = (P.N + 255) / 256;
  const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
  rk_stage_kernel<typename Store<S>::R><<<grid, 256, 0, st>>>(P, psi, T, u, acc, out, kind);
}

template <class S, int Q>
static void convert_q(bool to_f64, void* pdf, double* f64, long long N, double shift, cudaStream_t st) {
  const long long blocks = ((long long)Q * N + 255) / 256;
  const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
  if (to_f64) pdf_to_f64_kernel<S, Q><<<grid, 256, 0, st>>>((const S*)pdf, f64, N, shift);
  else f64_to_pdf_kernel<S, Q><<<grid, 256, 0, st>>>(f64, (S*)pdf, N, shift);
}

template <class S>
void launch_pdf_convert(int Q, bool to_f64, void* pdf, double* f64, long long N, double shift,
                        cudaStream_t st) {
  switch (Q) {
    case 1: convert_q<S, 1>(to_f64, pdf, f64, N, shift, st); break;
    case 7: convert_q<S, 7>(to_f64, pdf, f64, N, shift, st); break;
    case 15: convert_q<S, 15>(to_f64, pdf, f64, N, shift, st); break;
    case 19: convert_q<S, 19>(to_f64, pdf, f64, N, shift, st); break;
    default: convert_q<S, 27>(to_f64, pdf, f64, N, shift, st); break;
  }
}

void launch_diag_finalize(const double* partials, int nblocks, double* out, cudaStream_t st) {
  diag_finalize_kernel<<<1, 256, 0, st>>>(partials, nblocks, out);
}

template void launch_rk_stage<double>(const DevParams&, const double*, double*, const double*,
                                      double*, double*, int, cudaStream_t);
template void launch_rk_stage<float>(const DevParams&, const float*, float*, const float*, float*,
                                     float*, int, cudaStream_t);
template void launch_rk_stage<__half>(const DevParams&, const float*, float*, const float*, float*,
                                      float*, int, cudaStream_t);
template void launch_pdf_convert<double>(int, bool, void*, double*, long long, double, cudaStream_t);
template void launch_pdf_convert<float>(int, bool, void*, double*, long long, double, cudaStream_t);
template void launch_pdf_convert<__half>(int, bool, void*, double*, long long, double, cudaStream_t);

}  // namespace lbm
