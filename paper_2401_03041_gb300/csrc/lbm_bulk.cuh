// lbm_bulk.cuh - the fused time-step kernel with tensor-TMA staging.
//
// Same arithmetic as the generic kernel (lbm_step.cuh, via lbm_cell.cuh); the
// difference is how the pulled PDFs reach the SM.  A CTA owns a TXB x TYB
// column of cells and marches along z.  For every plane it stages, in shared
// memory, the PDF boxes the pull scheme reads, one 4D tensor-TMA box
// (x, y, z, direction) per direction:
//   HF(p): h and f over the (TYB + 2)-row halo tile of plane p, each box
//          shifted by -c_y and taken from plane p - c_z; columns
//          [x0 - GXP, x0 + TXB + GXP) with GXP = 16 / sizeof(S), so that every
//          box starts on a 16-byte boundary (the -c_x shift is applied when
//          reading shared memory);
//   G(p):  g over the TYB interior rows, same scheme.
// The PDF arrays carry periodic ghost cells (GXP columns, two rows) that a
// ghost-fill pass refreshes after every step, so no box wraps.  Boxes whose
// source lies beyond a z wall come from the opposite direction at the same
// cell (bounce-back) and are read without shift.  Boxes complete on mbarriers
// (expect_tx byte counts).  While plane z is computed, HF(z + 2) and G(z + 1)
// are in flight: HF uses a ring of three buffers (z, z + 1 for phi/T, z + 2 in
// flight), G a ring of two (or of one, issued mid-plane, where two do not fit
// in shared memory).  phi and T of the halo tile are summed from HF and
// kept for planes z - 1, z, z + 1.
//
// Every wait is bounded (about 2 s); on a timeout the CTA raises the domain's
// error flag, drains its outstanding copies (bounded too) and returns.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "lbm_step.cuh"

namespace lbm {

// ----------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Bring a tensor-map descriptor into the descriptor cache.
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// 4D tensor box (x, y, z, direction) global -> shared, completing on bar.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false after ~2 s without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 2000000000ull) return false;
  }
  return true;
}

// Runtime velocity tables (for the copy tasks, whose direction index is not
// a compile-time constant): D3Q27 order, Q15 maps through to27.
struct DirTab {
  signed char c[27][3];
  signed char opp[27];
};
__host__ __device__ constexpr DirTab make_dirtab27() {
  DirTab t{};
  for (int i = 0; i < 27; ++i) {
    t.c[i][0] = (signed char)q27_cx(i);
    t.c[i][1] = (signed char)q27_cy(i);
    t.c[i][2] = (signed char)q27_cz(i);
    t.opp[i] = (signed char)opp<27>(i);
  }
  return t;
}
static __constant__ DirTab kDir27 = make_dirtab27();

template <int Q>
__device__ __forceinline__ int rt_to27(int i) { return (Q == 15 && i >= 7) ? i + 12 : i; }
template <int Q>
__device__ __forceinline__ int rt_from27(int k) { return (Q == 15 && k >= 19) ? k - 12 : k; }

template <class S, int TYB_ = 4>
struct BulkGeom {
  static constexpr int GXP = 16 / (int)sizeof(S);       // halo columns on each side (= ghost width)
  static constexpr int TXB = sizeof(S) == 8 ? 32 : 64;  // columns per CTA
  static constexpr int W = TXB + 2 * GXP;               // staged row length (elements)
  static constexpr int TYB = TYB_;                      // rows per CTA
  static constexpr int HXB = TXB + 2;                   // phi/T plane pitch
  static constexpr int HYB = TYB + 2;
  static constexpr int HPB = HXB * HYB;
  static constexpr int NT = TXB * TYB;                  // cells per CTA
  static constexpr int NTHR = 2 * NT;                   // threads: two roles per cell
  // shared-memory pitch of one box (128-byte aligned destinations)
  static constexpr int HFB = (int)(((size_t)W * (TYB + 2) * sizeof(S) + 127) / 128 * 128 / sizeof(S));
  static constexpr int GB = (int)(((size_t)W * TYB * sizeof(S) + 127) / 128 * 128 / sizeof(S));
};

template <class S, int QH, int QF, int TYB_>
struct BulkSmemT {
  using R = typename Store<S>::R;
  using G = BulkGeom<S, TYB_>;
  static constexpr int NHF = QH + QF;
  static constexpr size_t hf_stage = (size_t)NHF * G::HFB;   // elements
  static constexpr size_t g_stage = (size_t)27 * G::GB;
  // g ring depth: two stages (G(z + 1) in flight during all of plane z) where
  // the layout fits in 227 KB, else one (G(z + 1) issued once every g-role
  // thread has taken the moments of G(z))
  static constexpr size_t fixed_bytes = 3 * hf_stage * sizeof(S) + 3 * G::HPB * 2 * sizeof(R) +
                                        8 * G::NT * sizeof(R) + 5 * sizeof(uint64_t) + 128 + 64;
  static constexpr int GR = fixed_bytes + 2 * g_stage * sizeof(S) <= 232448 ? 2 : 1;
  static constexpr size_t off_hf = 0;
  static constexpr size_t off_g = off_hf + 3 * hf_stage * sizeof(S);
  // (phi, T) of the halo tile, interleaved, for planes z - 1, z, z + 1
  static constexpr size_t off_phi = (off_g + GR * g_stage * sizeof(S) + 15) & ~size_t(15);
  static constexpr size_t off_T = off_phi + 3 * G::HPB * sizeof(R);   // end of the first half
  // per-cell exchange between the two roles: phi and the acceleration a (3)
  // from the h/f role; j (3), p* from the g role
  static constexpr int NX = 8;
  static constexpr size_t off_x = (off_T + 3 * G::HPB * sizeof(R) + 15) & ~size_t(15);
  static constexpr size_t off_bar = (off_x + (size_t)NX * G::NT * sizeof(R) + 15) & ~size_t(15);
  // + 128: the kernel aligns the start of its dynamic shared memory to 128
  // bytes at run time (tensor boxes need 128-byte aligned destinations)
  static constexpr size_t bytes = off_bar + 5 * sizeof(uint64_t) + 128;
  // bytes one stage's boxes deliver (box padding is not written)
  static constexpr uint32_t hf_tx = (uint32_t)((size_t)NHF * G::W * (G::TYB + 2) * sizeof(S));
  static constexpr uint32_t g_tx = (uint32_t)((size_t)27 * G::W * G::TYB * sizeof(S));
};

// Tiles of four rows where that layout fits in 227 KB of shared memory, else
// of two rows (large thermal stencils, h on D3Q27): half the cells per CTA.
template <class S, int QH, int QF>
using BulkSmem = BulkSmemT<S, QH, QF, (BulkSmemT<S, QH, QF, 4>::bytes <= 232448 ? 4 : 2)>;

// Issue the boxes of one stage.  Box issue is spread over the warps (lane j
// of warp w issues direction w + j * nwarps): box issues by lanes of one warp
// serialise, so a single warp issuing every box would stall the whole CTA.
//   KIND 0 (HF): rows y0 - 1 .. y0 + TYB of plane p; directions 0..QH-1 from
//                h (map mh), QH..QH+QF-1 from f (map mf).
//   KIND 1 (G):  rows y0 .. y0 + TYB - 1 of plane p; g directions (map mg).
// Tensor coordinates are those of the padded arrays: (x + GX, y + GY, z, q).
// AAM selects the in-place layout's gathers (0: two grids; 1: odd level, all
// local; 2: even level, F[opp(i)] from x - c_i); its h/f boxes hold rows
// y0 .. y0 + TYB - 1 only (maps with TYB-row boxes).
template <class S, class G, int QH, int QF, int KIND, int AAM = 0>
__device__ __forceinline__ void issue_stage(const DevParams& P, const CUtensorMap* mh,
                                            const CUtensorMap* mg, const CUtensorMap* mf,
                                            S* dst_stage, uint64_t* bar, int p, int x0, int y0,
                                            int tid, int nwarps = G::NTHR / 32) {
  constexpr int ndir = KIND == 0 ? QH + QF : 27;
  const int d = (tid >> 5) + (tid & 31) * nwarps;
  if (d >= ndir) return;
  // plane whose tile this is (walls: the ghost planes reuse the boundary plane)
  int pe = p;
  if (P.walls) pe = p < 0 ? 0 : (p >= P.nz ? P.nz - 1 : p);
  else pe = p < 0 ? p + P.nz : (p >= P.nz ? p - P.nz : p);
  int k27, q;
  const CUtensorMap* map;
  if (KIND == 1) {
    map = mg;
    k27 = d;
    q = d;
  } else if (d < QH) {
    map = mh;
    k27 = rt_to27<QH>(d);
    q = d;
  } else {
    map = mf;
    q = d - QH;
    k27 = QF == 15 ? rt_to27<15>(q) : q;   // Q7/Q19/Q27 are prefixes of the D3Q27 order
  }
  // the array of the opposite direction
  auto opp_q = [&]() {
    const int o27 = kDir27.opp[k27];
    if (KIND == 1) return o27;
    if (d < QH) return rt_from27<QH>(o27);
    return QF == 15 ? rt_from27<15>(o27) : o27;
  };
  // in place (AAM != 0) the boxes hold the tile's own rows only; the two-grid
  // h/f boxes add one halo row on each side
  const int ylo = y0 - ((KIND == 0 && AAM == 0) ? 1 : 0);
  int zz = pe - kDir27.c[k27][2], yy;
  if (AAM == 1) {
    // in place, odd level: every population is gathered from its own cell
    zz = pe;
    yy = ylo;
  } else if (P.walls && (zz < 0 || zz >= P.nz)) {
    // source beyond a wall.  Two grids: the opposite direction of the same
    // cells (bounce-back).  In place, even level: the direction's own array
    // at the same cells, where the previous step left the reflected value.
    if (AAM == 0) q = opp_q();
    zz = pe;
    yy = ylo;
  } else {
    zz = zz < 0 ? zz + P.nz : (zz >= P.nz ? zz - P.nz : zz);
    yy = ylo - kDir27.c[k27][1];
    // in place, even level: f*_i(x) = F[opp(i)](x - c_i)
    if (AAM == 2) q = opp_q();
  }
  S* dst = dst_stage + (size_t)d * ((KIND == 0 && AAM == 0) ? G::HFB : G::GB);
  tma_load_4d(dst, map, x0 - G::GXP + P.GX, yy + P.GY, zz, q, bar);
}

// Anti-bounce-back wall value of direction I of the thermal LB in stored form,
// T_w E_I - s: the wall temperature (the bottom wall's modulation in EXT
// builds), times the even part of the equilibrium at the wall's velocity for
// a moving wall (E_I = 1 at rest), minus the storage shift s.
template <class S, int QF, int I, bool EXT, bool BOUNCE>
__device__ __forceinline__ typename Store<S>::R abb_wall_value(const DevParams& P, int x,
                                                              typename Store<S>::R shf) {
  using R = typename Store<S>::R;
  const auto& rp = RP<R>(P);
  constexpr bool bottom = cz<QF>(I) > 0;
  R Tw;
  if constexpr (bottom) {
    if constexpr (EXT) Tw = wall_T<R>(P, x, true);
    else Tw = (R)rp.T_bottom;
  } else {
    Tw = (R)rp.T_top;
  }
  if constexpr (EXT && BOUNCE && cz<QF>(I) != 0)
    if (P.moving_walls) Tw *= wall_even<QF, I, R>(P, bottom ? 0 : 1);
  return Tw - shf;
}

// phi and T over the (TYB + 2) x (TXB + 2) halo tile of plane p, summed from
// the staged h / f boxes of that plane (st), into the interleaved (phi, T)
// plane pt; items k0, k0 + kstep, ... of the tile.  Ghost planes beyond a z
// wall mirror phi and take T_g = 2 T_w - T; with an RK energy solver T comes
// from the stored field (or, for the first item, from *tpre: the caller's
// value of that field cell, loaded ahead).  Planes next to a wall take the
// bounce-back variant (BOUNCE = true); all other planes run the select-free
// one.
template <class S, int QH, int QF, bool EXT, class G, bool BOUNCE>
__device__ __forceinline__ void stage_sum_plane_v(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                                  const S* st, typename PairOf<typename Store<S>::R>::type* pt,
                                                  int p, int pe, bool ghost, bool lo, bool hi, int x0, int y0,
                                                  int k0, int kstep, int kend,
                                                  const typename Store<S>::R* tpre) {
  using R = typename Store<S>::R;
  using P2 = typename PairOf<R>::type;
  const auto& rp = RP<R>(P);
  const R shh = (R)rp.shift_h, shf = (R)rp.shift_f;
  for (int k = k0; k < kend; k += kstep) {
    const int hr = k / G::HXB, hc = k % G::HXB;
    const int col = hc + G::GXP - 1;
    const S* rowb = st + (size_t)hr * G::W + col;
    R phi = 0;
    static_for<0, QH>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const bool b = BOUNCE && ((cz<QH>(i) > 0 && lo) || (cz<QH>(i) < 0 && hi));
      const S* rowp = rowb + (size_t)i * G::HFB;
      phi += Store<S>::ld_s(b ? rowp : rowp - cx<QH>(i));
    });
    phi += shh;  // sum_i w_i * shift_h
    R T;
    // wall temperature below this halo column (its x wrapped into the lattice)
    auto bottom_T = [&]() {
      int gx = x0 + hc - 1;
      gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
      return wall_T<R>(P, gx, true);
    };
    if constexpr (QF > 0) {
      // stored values (shifted by w_i s, s = shift_f; sum_i w_i = 1);
      // anti-bounce-back in stored form: -v_s + 2 w_i (T_w - s)
      T = shf;
      R Tb = 0, Tt = 0, Tbr = 0, Ttr = 0;
      if constexpr (BOUNCE) {
        if constexpr (EXT) Tb = bottom_T();
        else Tb = (R)rp.T_bottom;
        Tt = (R)rp.T_top;
        Tbr = Tb - shf;
        Ttr = Tt - shf;
      }
      static_for<0, QF>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const bool b = BOUNCE && ((cz<QF>(i) > 0 && lo) || (cz<QF>(i) < 0 && hi));
        const S* rowp = rowb + (size_t)(QH + i) * G::HFB;
        const R v = Store<S>::ld_s(b ? rowp : rowp - cx<QF>(i));
        R tw = cz<QF>(i) > 0 ? Tbr : Ttr;
        if constexpr (EXT && BOUNCE) {
          // moving wall: the even part of the equilibrium at u_w
          if (P.moving_walls)
            tw = (cz<QF>(i) > 0 ? Tb : Tt) * wall_even<QF, i, R>(P, cz<QF>(i) > 0 ? 0 : 1) - shf;
        }
        T += b ? (-v + (R)(2.0 * weight<QF>(i)) * tw) : v;
      });
    } else {
      if (tpre && k == k0) {
        T = *tpre;
      } else {
        int gx = x0 + hc - 1, gy = y0 + hr - 1;
        gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
        gy = gy < 0 ? gy + P.ny : (gy >= P.ny ? gy - P.ny : gy);
        T = A.T[cell_index(P, gx, gy, pe)];
      }
    }
    if constexpr (EXT) {
      if (ghost) T = (R)2 * (p < 0 ? bottom_T() : (R)rp.T_top) - T;
      // phi beyond a wall: the mirror, or the contact-angle ghost
      if (ghost && P.wetting) phi = wet_ghost<R>(phi, wall_k<R>(P, p < 0 ? 0 : 1));
    } else {
      if (ghost) T = (R)2 * (p < 0 ? rp.T_bottom : rp.T_top) - T;
    }
    P2 v;
    v.x = phi;
    v.y = T;
    pt[k] = v;
  }
}

template <class S, int QH, int QF, bool EXT, class G>
__device__ __forceinline__ void stage_sum_plane(const DevParams& P, const StepPtrs<S, typename Store<S>::R>& A,
                                                const S* st, typename PairOf<typename Store<S>::R>::type* pt,
                                                int p, int x0, int y0, int k0, int kstep,
                                                int kend = G::HPB, const typename Store<S>::R* tpre = nullptr) {
  int pe = p;
  bool ghost = false;
  if (P.walls) {
    if (p < 0) { pe = 0; ghost = true; }
    else if (p >= P.nz) { pe = P.nz - 1; ghost = true; }
  } else {
    pe = p < 0 ? p + P.nz : (p >= P.nz ? p - P.nz : p);  // periodic z
  }
  const bool lo = P.walls && pe == 0, hi = P.walls && pe == P.nz - 1;
  if (lo || hi)
    stage_sum_plane_v<S, QH, QF, EXT, G, true>(P, A, st, pt, p, pe, ghost, lo, hi, x0, y0, k0, kstep, kend, tpre);
  else
    stage_sum_plane_v<S, QH, QF, EXT, G, false>(P, A, st, pt, p, pe, ghost, false, false, x0, y0, k0, kstep, kend,
                                                tpre);
}

// EXT: the extensions of the uniform-property model (conductivity ratio,
// modulated bottom wall) are compiled in; lattices without them run the
// EXT = false instantiation, which carries none of their code.
template <class S, int QH, int QF, bool EXT>
__global__ void __launch_bounds__(BulkSmem<S, QH, QF>::G::NTHR, 1)
step_bulk_kernel(const DevParams P, const StepPtrs<S, typename Store<S>::R> A,
                 const __grid_constant__ CUtensorMap mh, const __grid_constant__ CUtensorMap mg,
                 const __grid_constant__ CUtensorMap mf, const BulkSched sched, int mode) {
  using R = typename Store<S>::R;
  const auto& rp = RP<R>(P);
  using L = BulkSmem<S, QH, QF>;
  using G = typename L::G;
  constexpr int NC = G::NT;       // cells per CTA
  constexpr int NT = G::NTHR;     // threads per CTA
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  S* hf = (S*)(smem + L::off_hf);
  S* gb = (S*)(smem + L::off_g);
  using P2 = typename PairOf<R>::type;
  P2* s_pt = (P2*)(smem + L::off_phi);             // [3][HPB] (phi, T)
  R* xch = (R*)(smem + L::off_x);                  // [NX][NC] role exchange
  uint64_t* bar = (uint64_t*)(smem + L::off_bar);  // [0..2] HF ring, [3..4] G ring

  // Two threads per cell: threads [0, NC) run the g part of the update (role
  // A), threads [NC, 2 NC) the phi / T stencils and the h and f parts (role
  // B).  Warp w of role A and warp w + NC/32 of role B hold the same 32 cells.
  const int tid = threadIdx.x;
  const bool role_g = tid < NC;
  const int cidx = role_g ? tid : tid - NC;
  const int tx = cidx % G::TXB, ty = cidx / G::TXB;
  int tcol, trow, z0, z1;
  bulk_unit(sched, P.nz, (int)blockIdx.x, tcol, trow, z0, z1);
  const int x0 = tcol * G::TXB, y0 = trow * G::TYB;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < P.nx) && (y < P.ny);
  const R shh = (R)rp.shift_h, shf = (R)rp.shift_f;
  constexpr uint32_t hf_bytes = L::hf_tx;
  constexpr uint32_t g_bytes = L::g_tx;

  if (tid == 0) {
    for (int k = 0; k < 5; ++k) mbar_init(&bar[k], 1);
    mbar_fence_init();
  } else if (tid == 32) {
    tma_prefetch_desc(&mh);
    tma_prefetch_desc(&mg);
    tma_prefetch_desc(&mf);
  }
  __syncthreads();

  // ring bookkeeping, relative to the chunk: HF plane p -> slot (p - z0 + 1) % 3
  // and fill index (p - z0 + 1) / 3; G plane p -> slot (p - z0) % 2, index (p - z0) / 2
  auto hf_slot = [&](int p) { return (p - z0 + 1) % 3; };
  auto hf_par = [&](int p) { return (uint32_t)(((p - z0 + 1) / 3) & 1); };
  constexpr int GR = L::GR;
  auto g_slot = [&](int p) { return (p - z0) % GR; };
  auto g_par = [&](int p) { return (uint32_t)(((p - z0) / GR) & 1); };
  auto hf_ptr = [&](int p) { return hf + (size_t)hf_slot(p) * L::hf_stage; };
  auto g_ptr = [&](int p) { return gb + (size_t)g_slot(p) * L::g_stage; };

  // phi / T of the halo tile of plane p from HF(p) -> phi/T slot (p - z0 + 1) % 3
  auto sum_plane = [&](int p) {
    stage_sum_plane<S, QH, QF, EXT, G>(P, A, hf_ptr(p), s_pt + hf_slot(p) * G::HPB, p, x0, y0, tid, NT);
  };

  DiagAcc<R> dsum;   // per-thread FP64 diagnostics

  bool ok = true;
  // pending[k]: slot k has copies in flight with parity pend_par[k]
  uint32_t pending = 0, pend_par = 0;
  auto mark = [&](int k, uint32_t par) { pending |= 1u << k; pend_par = (pend_par & ~(1u << k)) | (par << k); };
  auto wait_slot = [&](int k, uint32_t par) {
    const bool r = mbar_wait(&bar[k], par);
    if (r) pending &= ~(1u << k);
    return r;
  };

  // Copy schedule: HF(p) lands in slot (p - z0 + 1) % 3, G(p) in (p - z0) % 2.
  // At the start of iteration z both HF(z + 2) and G(z + 1) are issued into
  // the slots that iteration z - 1 has just released, so their latency is
  // hidden behind the whole of iteration z (phi/T sum and collision).  Thread
  // 0 posts the expected byte counts before the barrier that precedes the
  // copies.
  auto expect_for = [&](int z) {
    if (z + 2 <= z1) mbar_expect_tx(&bar[hf_slot(z + 2)], hf_bytes);
    if (GR == 2 && z + 1 < z1) mbar_expect_tx(&bar[3 + g_slot(z + 1)], g_bytes);
  };
  if (z0 < z1) {
    // prologue: HF(z0-1), HF(z0), HF(z0+1), G(z0) now; HF(z0+2), G(z0+1) at
    // the start of the first iteration
    if (tid == 0) {
      // (test of the timeout path: 16 bytes more than the copies deliver, so
      // the first stage never completes and its bounded wait runs out)
      for (int p = z0 - 1; p <= z0 + 1; ++p)
        mbar_expect_tx(&bar[hf_slot(p)], hf_bytes + (P.test_stall && p == z0 - 1 ? 16u : 0u));
      mbar_expect_tx(&bar[3 + g_slot(z0)], g_bytes);
    }
    __syncthreads();
    for (int p = z0 - 1; p <= z0 + 1; ++p) {
      issue_stage<S, G, QH, QF, 0>(P, &mh, &mg, &mf, hf_ptr(p), &bar[hf_slot(p)], p, x0, y0, tid);
      mark(hf_slot(p), hf_par(p));
    }
    issue_stage<S, G, QH, QF, 1>(P, &mh, &mg, &mf, g_ptr(z0), &bar[3 + g_slot(z0)], z0, x0, y0, tid);
    mark(3 + g_slot(z0), g_par(z0));
    ok = ok && wait_slot(hf_slot(z0 - 1), hf_par(z0 - 1));
    if (ok) sum_plane(z0 - 1);
    ok = ok && wait_slot(hf_slot(z0), hf_par(z0));
    if (ok) sum_plane(z0);
    // every thread has waited on HF(z0 - 1), whose slot HF(z0 + 2) reuses
    if (__syncthreads_or(!ok)) ok = false;
    if (tid == 0 && ok) expect_for(z0);
    __syncthreads();
  }

  for (int z = z0; z < z1 && ok; ++z) {
    // slots of HF(z - 1) and G(z - 1) are free: refill them
    if (z + 2 <= z1) {
      issue_stage<S, G, QH, QF, 0>(P, &mh, &mg, &mf, hf_ptr(z + 2), &bar[hf_slot(z + 2)], z + 2, x0, y0, tid);
      mark(hf_slot(z + 2), hf_par(z + 2));
    }
    if (GR == 2 && z + 1 < z1) {
      issue_stage<S, G, QH, QF, 1>(P, &mh, &mg, &mf, g_ptr(z + 1), &bar[3 + g_slot(z + 1)], z + 1, x0, y0, tid);
      mark(3 + g_slot(z + 1), g_par(z + 1));
    }
    ok = ok && wait_slot(hf_slot(z + 1), hf_par(z + 1));
    if (ok) sum_plane(z + 1);
    ok = ok && wait_slot(3 + g_slot(z), g_par(z));
    if (__syncthreads_or(!ok)) { ok = false; break; }
    {
      const bool lo = P.walls && z == 0, hi = P.walls && z == P.nz - 1;
      const int col = tx + G::GXP;
      const S* hrow = hf_ptr(z) + (size_t)(ty + 1) * G::W + col;   // direction 0, this cell
      const S* grow = g_ptr(z) + (size_t)ty * G::W + col;
      const size_t cell = cell_index(P, x, y, z);
      const size_t pcell = pdf_index(P, x, y, z);
      // pairs warp w (role A) with warp w + NC/32 (role B): named barrier 1 + w
      const int pair_id = 1 + (cidx >> 5);
      auto pair_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(pair_id) : "memory"); };
      if (role_g) {
        auto run = [&](auto btag) {
          constexpr bool BOUNCE = decltype(btag)::value;
          auto getg = [&](auto I) {
            constexpr int i = decltype(I)::value;
            const bool b = BOUNCE && ((cz<27>(i) > 0 && lo) || (cz<27>(i) < 0 && hi));
            const S* p_ = grow + (size_t)i * G::GB;
            R v = Store<S>::ld_s(b ? p_ : p_ - cx<27>(i));
            if constexpr (EXT && BOUNCE && cz<27>(i) != 0)
              if (b && P.moving_walls) v += wall_momentum<27, i, R>(P, cz<27>(i) > 0 ? 0 : 1);
            return v;
          };
          // density ratio (EXT only): the g role adds F_p and F_mu, which need
          // the moments of g, and hands u and p* back after a second pair
          // barrier; the exchange slots then carry phi, a, grad phi (h/f role)
          // and u, p* (g role)
          const bool ratio = EXT && P.rho_ratio;
          GMoments<R> m;
          if (active) {
            m = g_moments<R>(getg);
            if (mode & MODE_SAVE) save_moments<S>(P, A, cell, m);
            if (!ratio) {
              xch[4 * NC + cidx] = m.jx;
              xch[5 * NC + cidx] = m.jy;
              xch[6 * NC + cidx] = m.jz;
              xch[7 * NC + cidx] = m.pst;
            }
          }
          if constexpr (GR == 1) {
            // every g-role thread has read G(z): warp 0 of the role refills
            // the single G slot with G(z + 1)
            asm volatile("bar.sync 15, %0;" ::"r"(NC) : "memory");
            if (z + 1 < z1) {
              if (tid < 32) {
                if (tid == 0) mbar_expect_tx(&bar[3 + g_slot(z + 1)], g_bytes);
                __syncwarp();
                issue_stage<S, G, QH, QF, 1>(P, &mh, &mg, &mf, g_ptr(z + 1), &bar[3 + g_slot(z + 1)], z + 1, x0,
                                          y0, tid, 1);
              }
              mark(3 + g_slot(z + 1), g_par(z + 1));
            }
          }
          pair_sync();
          if constexpr (EXT) {
            if (ratio) {
              CellFlow<R> f;
              const R phi = active ? xch[cidx] : (R)0;
              if (active) {
                CellForce<R> F;
                F.ax = xch[NC + cidx]; F.ay = xch[2 * NC + cidx]; F.az = xch[3 * NC + cidx];
                F.rho = (R)rp.rho_L + phi * (R)(rp.rho_H - rp.rho_L);
                density_ratio_accel<R>(P, phi, xch[4 * NC + cidx], xch[5 * NC + cidx], xch[6 * NC + cidx], m, F);
                f = cell_velocity<R>(F.ax, F.ay, F.az, F.rho, m.jx, m.jy, m.jz);
                xch[cidx] = f.ux;
                xch[NC + cidx] = f.uy;
                xch[2 * NC + cidx] = f.uz;
                xch[3 * NC + cidx] = m.pst;
              }
              pair_sync();
              if (active && (mode & MODE_COLLIDE)) collide_g<S>(P, A, pcell, phi, m, f);
              return;
            }
          }
          if (active && (mode & MODE_COLLIDE)) {
            const R phi = xch[cidx];
            const CellFlow<R> f = cell_velocity<R>(xch[NC + cidx], xch[2 * NC + cidx], xch[3 * NC + cidx],
                                                   (R)1, m.jx, m.jy, m.jz);
            collide_g<S>(P, A, pcell, phi, m, f);
          }
        };
        if (lo || hi) run(std::true_type{});
        else run(std::false_type{});
      } else {
        const P2* pm = s_pt + hf_slot(z - 1) * G::HPB;
        const P2* pc = s_pt + hf_slot(z) * G::HPB;
        const P2* pp = s_pt + hf_slot(z + 1) * G::HPB;
        const int c0 = (ty + 1) * G::HXB + (tx + 1);
        Stencil27<R> fd;
        R rgx = 0, rgy = 0, rgz = 0, rlap = 0, pgx = 0, pgy = 0, pgz = 0;
        const P2 cen = pc[c0];
        CellForce<R> F;
        if (active) {
          eval_pairs<G::HXB>(fd, pm, pc, pp, c0);
          if constexpr (QF == 0) {
            rk_std_pairs<P2, R, G::HXB>(pm, pc, pp, c0, rgx, rgy, rgz, rlap);
            if constexpr (EXT)
              if (P.alpha_ratio && !P.rk_iso) central_phi_pairs<P2, R, G::HXB>(pm, pc, pp, c0, pgx, pgy, pgz);
          }
          if (mode & MODE_SAVE) save_stencil<S>(P, A, cell, cen.x, cen.y, fd);
          // a4-a5 need nothing from the g role: the force is computed here,
          // once, and only phi and a go across
          F = cell_force<R, EXT>(P, x, y, z, cen.x, cen.y, fd.gpx, fd.gpy, fd.gpz, fd.lp, fd.gtx, fd.gty, fd.gtz);
          xch[cidx] = cen.x;
          xch[NC + cidx] = F.ax;
          xch[2 * NC + cidx] = F.ay;
          xch[3 * NC + cidx] = F.az;
          if (EXT && P.rho_ratio) {
            xch[4 * NC + cidx] = fd.gpx;
            xch[5 * NC + cidx] = fd.gpy;
            xch[6 * NC + cidx] = fd.gpz;
          }
        }
        pair_sync();
        R ex_u[3] = {0, 0, 0}, ex_p = 0;
        if (EXT && P.rho_ratio) {
          // u and p* from the g role, which added F_p and F_mu
          pair_sync();
          if (active) {
            ex_u[0] = xch[cidx]; ex_u[1] = xch[NC + cidx]; ex_u[2] = xch[2 * NC + cidx];
            ex_p = xch[3 * NC + cidx];
          }
        }
        if (active) {
          const R phi = cen.x, Tc = cen.y;
          CellFlow<R> f;
          R pst;
          if (EXT && P.rho_ratio) {
            f.ux = ex_u[0]; f.uy = ex_u[1]; f.uz = ex_u[2];
            f.uu = f.ux * f.ux + f.uy * f.uy + f.uz * f.uz;
            f.rho = F.rho;
            f.ax = f.ay = f.az = (R)0;   // (not used by the h / f collisions)
            pst = ex_p;
          } else {
            f = cell_velocity<R>(F.ax, F.ay, F.az, F.rho, xch[4 * NC + cidx], xch[5 * NC + cidx],
                                 xch[6 * NC + cidx]);
            pst = xch[7 * NC + cidx];
          }
          cell_outputs<S>(P, A, x, y, z, cell, mode, phi, Tc, pst, f, dsum);
          if (mode & MODE_COLLIDE) {
            auto run = [&](auto btag) {
              constexpr bool BOUNCE = decltype(btag)::value;
              // pulled values as stored (collide_h / collide_f work on them)
              auto geth = [&](auto I) {
                constexpr int i = decltype(I)::value;
                const bool b = BOUNCE && ((cz<QH>(i) > 0 && lo) || (cz<QH>(i) < 0 && hi));
                const S* p_ = hrow + (size_t)i * G::HFB;
                R v = Store<S>::ld_s(b ? p_ : p_ - cx<QH>(i));
                if constexpr (EXT && BOUNCE && cz<QH>(i) != 0)
                  if (b && P.moving_walls) v += phi * wall_momentum<QH, i, R>(P, cz<QH>(i) > 0 ? 0 : 1);
                return v;
              };
              auto getf = [&](auto I) {
                if constexpr (QF > 0) {
                  constexpr int i = decltype(I)::value;
                  const bool b = BOUNCE && ((cz<QF>(i) > 0 && lo) || (cz<QF>(i) < 0 && hi));
                  const S* p_ = hrow + (size_t)(QH + i) * G::HFB;
                  const R v = Store<S>::ld_s(b ? p_ : p_ - cx<QF>(i));
                  // anti-bounce-back in stored form: -v_s + 2 w_i (T_w E_i - s), E_i = 1 at rest
                  return b ? (-v + (R)(2.0 * weight<QF>(i)) * abb_wall_value<S, QF, i, EXT, BOUNCE>(P, x, shf)) : v;
                } else {
                  return (R)0;
                }
              };
              collide_h<S, QH>(P, A, pcell, phi, fd.gpx, fd.gpy, fd.gpz, f, geth);
              if (EXT && P.alpha_ratio)
                collide_f<S, QF, EXT>(P, A, x, y, z, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
              else
                collide_f<S, QF, false>(P, A, x, y, z, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
            };
            if (lo || hi) run(std::true_type{});
            else run(std::false_type{});
          }
        }
      }
    }
    if (tid == 0 && ok) expect_for(z + 1);
    if (__syncthreads_or(!ok)) { ok = false; break; }
  }

  if (!ok) {
    // raise the error flag, drain outstanding copies (bounded), leave
    if (tid == 0 && A.error_flag) atomicExch(A.error_flag, 1);
    for (int k = 0; k < 5; ++k)
      if (pending & (1u << k)) mbar_wait(&bar[k], (pend_par >> k) & 1u);
    return;
  }
  // the reduction's scratch reuses the h/f ring (no copies are in flight and
  // every thread has passed the last plane's barrier), so the kernel needs
  // no static shared memory beyond its dynamic layout
  if (mode & MODE_DIAG) {
    double ds[kDiagVals];
    dsum.flush(ds);
    diag_block_reduce_in<NT>(ds, A.diag_partials, reinterpret_cast<double*>(smem + L::off_hf));
  }
}

}  // namespace lbm
