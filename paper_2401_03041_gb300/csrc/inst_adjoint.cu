// inst_adjoint.cu - instantiations and launchers of the adjoint-step kernels
// (FP64; h on D3Q15 or D3Q27; thermal LB D3Q7, D3Q15, D3Q19 or D3Q27, or the
// RK2 / RK4 energy solvers, QF = 0).
#include "launchers.h"
#include "lbm_adjoint.cuh"

namespace lbm {

namespace {

int grid_1d(size_t work) {
  const size_t b = (work + 255) / 256;
  return (int)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

bool adj_supported(int qh, int qf) {
  return (qh == 15 || qh == 27) && (qf == 0 || qf == 7 || qf == 15 || qf == 19 || qf == 27);
}

// Calls fn(integral_constant<QH>, integral_constant<QF>) for a supported pair.
template <class F>
static void adj_dispatch(int qh, int qf, F fn) {
  auto with_qf = [&](auto QH) {
    switch (qf) {
      case 0: fn(QH, std::integral_constant<int, 0>{}); break;
      case 7: fn(QH, std::integral_constant<int, 7>{}); break;
      case 15: fn(QH, std::integral_constant<int, 15>{}); break;
      case 19: fn(QH, std::integral_constant<int, 19>{}); break;
      default: fn(QH, std::integral_constant<int, 27>{}); break;
    }
  };
  if (qh == 15) with_qf(std::integral_constant<int, 15>{});
  else with_qf(std::integral_constant<int, 27>{});
}

// plane-indexed grids: x over nx * ny (< 2^31), y = z (<= 65535)
static unsigned plane_blocks(const DevParams& P) {
  return (unsigned)(((size_t)P.nx * P.ny + 255) / 256);
}

void adj_cell(const DevParams& P, const AdjPtrs& A, int qh, int qf, const double* rk_lu, cudaStream_t st) {
  const dim3 grid(plane_blocks(P), P.nz);
  adj_dispatch(qh, qf, [&](auto QH, auto QF) {
    adj_point_kernel<decltype(QH)::value, decltype(QF)::value><<<grid, 256, 0, st>>>(P, A, rk_lu);
  });
}

void adj_fields(const DevParams& P, const AdjPtrs& A, cudaStream_t st) {
  adj_fields_kernel<<<dim3(plane_blocks(P), P.nz), 256, 0, st>>>(P, A);
}

void adj_pull(const DevParams& P, const AdjPtrs& A, int qh, int qf, const double* rk_lT, cudaStream_t st) {
  const dim3 grid(plane_blocks(P), P.nz);
  adj_dispatch(qh, qf, [&](auto QH, auto QF) {
    adj_pull_kernel<decltype(QH)::value, decltype(QF)::value><<<grid, 256, 0, st>>>(P, A, rk_lT);
  });
}

void adj_seed(const DevParams& P, const double* dJdphi, double* lam, int qh, int qf, cudaStream_t st) {
  const size_t work = (size_t)(qh + 27 + (qf > 0 ? qf : 1)) * (size_t)P.N;
  adj_dispatch(qh, qf, [&](auto QH, auto QF) {
    adj_seed_kernel<decltype(QH)::value, decltype(QF)::value><<<grid_1d(work), 256, 0, st>>>(P, dJdphi, lam);
  });
}

void adj_centroid_seed(const DevParams& P, double mass, const double* c, const double* t, double* out,
                       cudaStream_t st) {
  adj_centroid_seed_kernel<<<grid_1d((size_t)P.N), 256, 0, st>>>(P, mass, c[0], c[1], c[2], t[0], t[1], t[2],
                                                                  out);
}

void adj_patch_grad(const DevParams& P, const double* lam, double* dJdI, int qh, int qf, cudaStream_t st) {
  if (P.npatch < 1) return;
  adj_dispatch(qh, qf, [&](auto QH, auto QF) {
    adj_patch_grad_kernel<decltype(QH)::value, decltype(QF)::value><<<P.npatch, 256, 0, st>>>(P, lam, dJdI);
  });
}

// The RK update's adjoint (see lbm_adjoint.cuh): u from the saved
// intermediates, the stage inputs replayed forward, then the stages in
// reverse.  RK4: b = (1/6, 1/3, 1/3, 1/6), stage inputs T + K1/2, T + K2/2,
// T + K3.  RK2 (midpoint): T' = T + K2, stage input T + K1/2.
void adj_rk(const DevParams& P, const double* save, const double* lamT, const AdjRK& R, bool rk4,
            cudaStream_t st) {
  const dim3 grid(plane_blocks(P), P.nz);
  const double* T = save + (size_t)SAVE_T * (size_t)P.N;
  adj_rk_velocity_kernel<<<grid, 256, 0, st>>>(P, save, R.u);
  auto replay = [&](const double* psi, double c, double* out) {
    adj_rk_replay_kernel<<<grid, 256, 0, st>>>(P, psi, T, R.u, c, out);
  };
  auto stage = [&](const double* src, double sK, const double* psi, double b_prev, double c_k, double* next,
                   int last) {
    adj_rk_stage_kernel<<<grid, 256, 0, st>>>(P, src, sK, psi, R.u, lamT, b_prev, c_k, next, R.lT, R.lu, R.lq,
                                              last);
  };
  if (rk4) {
    replay(T, 0.5, R.psi[0]);
    replay(R.psi[0], 0.5, R.psi[1]);
    replay(R.psi[1], 1.0, R.psi[2]);
    stage(lamT, 1.0 / 6.0, R.psi[2], 1.0 / 3.0, 1.0, R.lk[0], 1);    // K4 -> adjoint of K3
    stage(R.lk[0], 1.0, R.psi[1], 1.0 / 3.0, 0.5, R.lk[1], 0);      // K3 -> K2
    stage(R.lk[1], 1.0, R.psi[0], 1.0 / 6.0, 0.5, R.lk[0], 0);      // K2 -> K1
    stage(R.lk[0], 1.0, T, 0.0, 0.0, nullptr, 0);                   // K1
  } else {
    replay(T, 0.5, R.psi[0]);
    stage(lamT, 1.0, R.psi[0], 0.0, 0.5, R.lk[0], 1);               // K2 -> adjoint of K1
    stage(R.lk[0], 1.0, T, 0.0, 0.0, nullptr, 0);                   // K1
  }
}

}  // namespace lbm
