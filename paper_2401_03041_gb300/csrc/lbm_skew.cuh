// lbm_skew.cuh - the fused time-step kernel with the two roles of a cell
// skewed by one plane, so that they never wait for each other inside a plane.
//
// Same staging as the bulk kernel (lbm_bulk.cuh: tensor-TMA boxes of the
// pulled PDFs, a ring of three h/f stages, a g ring, interleaved (phi, T)
// planes) and the same per-cell arithmetic (lbm_cell.cuh).  What differs is
// the schedule of the two threads of a cell.  In the bulk kernel the g role
// needs the acceleration a(z) of the stencil role and the stencil role needs
// the first moment j(z) of the g role within the same plane, so both meet at
// a barrier between their two halves and each waits for the other's slower
// half.  Here, while the CTA marches over plane z,
//   g role (A):       collides g of plane z      (m(z), and phi(z), a(z) that
//                                                  B left in the exchange),
//                     then takes the moments m(z + 2) of the staged G(z + 2);
//   stencil role (B): sums phi / T of plane z + 2 from the staged h/f boxes,
//                     computes the stencils and the force of plane z + 1,
//                     leaves phi(z + 1), a(z + 1) for A, and collides h and f
//                     of plane z + 1 with j(z + 1), p*(z + 1) that A left
//                     there one plane earlier.
// Every value a role reads from the other was written in an earlier plane,
// so the roles meet only at the one block barrier that ends each plane (the
// exchange is double-buffered by plane parity).  The g role carries the
// moments of two planes in registers; the h/f ring still needs only three
// stages (h/f boxes of z + 1 for the collisions, z + 2 just summed, z + 3 in
// flight).
//
// The density-ratio forces need the moments of g and the stencil of the same
// plane in one place, so a lattice with rho_L != rho_H runs the bulk kernel.
//
// In-place layout (AAM != 0; lbm_aa.cuh has the AA pattern): one PDF set is
// gathered and overwritten.  The boxes then hold the tile's own rows only
// (each slot is read and written by exactly one cell within a step, and a
// halo row of another tile may already hold that tile's new values), and phi
// / T of the halo tile come from the level's (phi, T) field instead of the
// staged boxes.  AAM = 1, odd level: f*_i(x) = F[i](x), new values to
// F[opp(i)](x).  AAM = 2, even level: f*_i(x) = F[opp(i)](x - c_i), new values
// to F[i](x + c_i); x + c_i may be a periodic ghost column or row, which the
// host folds back into the interior after the step (aa_fold_kernel).  The
// host sets the per-direction destination pointers (StepPtrs hd, gd, fd) for
// the level: F[opp(i)] (odd) or F[i] shifted by c_i's x and y (even).
// Every wait is bounded (about 2 s); on a timeout the CTA raises the domain's
// error flag, drains its outstanding copies (bounded too) and returns.
#pragma once

#include "lbm_bulk.cuh"

namespace lbm {

template <class S, int QH, int QF, int TYB_, int AAM = 0>
struct SkewSmemT {
  using R = typename Store<S>::R;
  using G = BulkGeom<S, TYB_>;
  static constexpr int NHF = QH + QF;
  // h/f box pitch: halo rows included (two grids) or the tile's rows (in place)
  static constexpr int HFP = AAM ? G::GB : G::HFB;
  static constexpr size_t hf_stage = (size_t)NHF * HFP;   // elements
  static constexpr size_t g_stage = (size_t)27 * G::GB;
  // exchange slots per cell and plane parity: phi, a (3) from B; j (3), p* from A
  static constexpr int NX = 8;
  static constexpr size_t fixed_bytes = 3 * hf_stage * sizeof(S) + 3 * G::HPB * 2 * sizeof(R) +
                                        2 * NX * G::NT * sizeof(R) + 5 * sizeof(uint64_t) + 128 + 64;
  // g ring: G(z + 2) consumed while G(z + 3) is in flight where two stages
  // fit, else one stage refilled right after the moments are taken
  static constexpr int GR = fixed_bytes + 2 * g_stage * sizeof(S) <= 232448 ? 2 : 1;
  static constexpr size_t off_hf = 0;
  static constexpr size_t off_g = off_hf + 3 * hf_stage * sizeof(S);
  static constexpr size_t off_pt = (off_g + GR * g_stage * sizeof(S) + 15) & ~size_t(15);
  static constexpr size_t off_x = (off_pt + 3 * G::HPB * 2 * sizeof(R) + 15) & ~size_t(15);
  static constexpr size_t off_bar = (off_x + 2 * (size_t)NX * G::NT * sizeof(R) + 15) & ~size_t(15);
  // + 128: the start of the dynamic shared memory is aligned at run time
  static constexpr size_t bytes = off_bar + 5 * sizeof(uint64_t) + 128;
  static constexpr uint32_t hf_tx = (uint32_t)((size_t)NHF * G::W * (AAM ? G::TYB : G::TYB + 2) * sizeof(S));
  static constexpr uint32_t g_tx = (uint32_t)((size_t)27 * G::W * G::TYB * sizeof(S));
  // halo items of a plane's phi / T sum taken by the g role: the first SUM_A
  // of the tile's HPB items, as many as leave one item per stencil-role
  // thread (at most one per g-role thread); the stencil role sums the rest
  // and waits for both shares
  static constexpr int SUM_A = G::HPB - G::NT < 0 ? 0 : (G::HPB - G::NT > G::NT ? G::NT : G::HPB - G::NT);
};

// The skewed kernel uses the bulk kernel's tile (one launch geometry for
// both, so that a lattice can switch between them); it is available where its
// layout fits at that tile height.
template <class S, int QH, int QF, int AAM = 0>
using SkewSmem = SkewSmemT<S, QH, QF, BulkSmem<S, QH, QF>::G::TYB, AAM>;

template <class S, int QH, int QF, int AAM = 0>
constexpr bool skew_fits() {
  return SkewSmem<S, QH, QF, AAM>::bytes <= 232448;
}

// In-place store, even level, of the new population of direction I (stencil
// Q) of the cell at pcell: F[I](x + c_I), or F[opp(I)](x) where x + c_I lies
// beyond a z wall (lo: the cell is on plane 0, hi: on plane nz - 1).  The
// host points dst[I] at F[I] shifted by c_I's x and y components (the
// destination may be a ghost column or row); pc_m / pc_p are pcell moved to
// the plane below / above (periodic wrap included).  At an odd level the
// host points dst[I] at F[opp(I)] and the plain store dst[I] + pcell applies.
template <class S, int Q, int I, bool BOUNCE>
__device__ __forceinline__ void aa_store_even(const DevParams& P, S* const* dst, const S* base, size_t pcell,
                                              size_t pc_m, size_t pc_p, bool lo, bool hi,
                                              typename Store<S>::R v) {
  constexpr int ez = cz<Q>(I);
  if constexpr (BOUNCE && ez != 0) {
    if ((ez < 0 && lo) || (ez > 0 && hi)) {
      Store<S>::st(const_cast<S*>(base) + (size_t)opp<Q>(I) * P.Np + pcell, v);
      return;
    }
  }
  Store<S>::st(dst[I] + (ez < 0 ? pc_m : (ez > 0 ? pc_p : pcell)), v);
}

template <class S, int QH, int QF, bool EXT, int AAM = 0>
__global__ void __launch_bounds__(SkewSmem<S, QH, QF, AAM>::G::NTHR, 1)
step_skew_kernel(const DevParams P, const StepPtrs<S, typename Store<S>::R> A,
                 const __grid_constant__ CUtensorMap mh, const __grid_constant__ CUtensorMap mg,
                 const __grid_constant__ CUtensorMap mf, const BulkSched sched, int mode,
                 const typename PairOf<typename Store<S>::R>::type* __restrict__ aa_phiT) {
  using R = typename Store<S>::R;
  using L = SkewSmem<S, QH, QF, AAM>;
  using G = typename L::G;
  using P2 = typename PairOf<R>::type;
  constexpr int NC = G::NT;       // cells per CTA
  constexpr int NT = G::NTHR;     // threads per CTA
  constexpr int NX = L::NX;
  constexpr int GR = L::GR;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  S* hf = (S*)(smem + L::off_hf);
  S* gb = (S*)(smem + L::off_g);
  P2* s_pt = (P2*)(smem + L::off_pt);             // [3][HPB] (phi, T)
  R* xch = (R*)(smem + L::off_x);                 // [2][NX][NC]
  uint64_t* bar = (uint64_t*)(smem + L::off_bar);  // [0..2] HF ring, [3..4] G ring

  const int tid = threadIdx.x;
  const bool role_g = tid < NC;
  const int cidx = role_g ? tid : tid - NC;
  const int tx = cidx % G::TXB, ty = cidx / G::TXB;
  int tcol, trow, z0, z1;
  bulk_unit(sched, P.nz, (int)blockIdx.x, tcol, trow, z0, z1);
  const int x0 = tcol * G::TXB, y0 = trow * G::TYB;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < P.nx) && (y < P.ny);
  const int col = tx + G::GXP;

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
  // (fill (p - z0 + 1) / 3), G plane p -> slot (p - z0) % GR (fill (p - z0) / GR)
  auto hf_slot = [&](int p) { return (p - z0 + 1) % 3; };
  auto hf_par = [&](int p) { return (uint32_t)(((p - z0 + 1) / 3) & 1); };
  auto g_slot = [&](int p) { return (p - z0) % GR; };
  auto g_par = [&](int p) { return (uint32_t)(((p - z0) / GR) & 1); };
  auto hf_ptr = [&](int p) { return hf + (size_t)hf_slot(p) * L::hf_stage; };
  auto g_ptr = [&](int p) { return gb + (size_t)g_slot(p) * L::g_stage; };
  auto pt_ptr = [&](int p) { return s_pt + hf_slot(p) * G::HPB; };
  auto xb = [&](int p, int slot) { return xch + ((size_t)(p & 1) * NX + slot) * NC + cidx; };

  bool ok = true;
  uint32_t pending = 0, pend_par = 0;
  auto mark = [&](int k, uint32_t par) { pending |= 1u << k; pend_par = (pend_par & ~(1u << k)) | (par << k); };
  auto wait_slot = [&](int k, uint32_t par) {
    const bool r = mbar_wait(&bar[k], par);
    if (r) pending &= ~(1u << k);
    return r;
  };
  // HF(p) into its slot, boxes spread over all warps
  auto issue_hf = [&](int p, uint32_t extra) {
    if (tid == 0) mbar_expect_tx(&bar[hf_slot(p)], L::hf_tx + extra);
    issue_stage<S, G, QH, QF, 0, AAM>(P, &mh, &mg, &mf, hf_ptr(p), &bar[hf_slot(p)], p, x0, y0, tid);
    mark(hf_slot(p), hf_par(p));
  };
  // G(p) into its slot, boxes spread over the g role's warps (g role only)
  auto issue_g = [&](int p) {
    if (tid == 0) mbar_expect_tx(&bar[3 + g_slot(p)], L::g_tx);
    issue_stage<S, G, QH, QF, 1, AAM>(P, &mh, &mg, &mf, g_ptr(p), &bar[3 + g_slot(p)], p, x0, y0, cidx, NC / 32);
    mark(3 + g_slot(p), g_par(p));
  };
  auto a_barrier = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory"); };
  // in place: (phi, T) of halo-tile item k of plane p as stored in the
  // level's field (raw), and the value the plane takes (ghost planes beyond a
  // wall: phi mirrored, T_g = 2 T_w - T)
  auto field_raw = [&](int p, int k) -> P2 {
    int pe;
    if (P.walls) pe = p < 0 ? 0 : (p >= P.nz ? P.nz - 1 : p);
    else pe = p < 0 ? p + P.nz : (p >= P.nz ? p - P.nz : p);
    int gx = x0 + k % G::HXB - 1, gy = y0 + k / G::HXB - 1;
    gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
    gy = gy < 0 ? gy + P.ny : (gy >= P.ny ? gy - P.ny : gy);
    return aa_phiT[cell_index(P, gx, gy, pe)];
  };
  auto field_put = [&](int p, int k, P2 v) {
    if (P.walls && (p < 0 || p >= P.nz)) {
      if constexpr (EXT) {
        // the modulated bottom wall's value above this column; the
        // contact-angle ghost of phi
        int gx = x0 + k % G::HXB - 1;
        gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
        v.y = (R)2 * (p < 0 ? wall_T<R>(P, gx, true) : (R)RP<R>(P).T_top) - v.y;
        if (P.wetting) v.x = wet_ghost<R>(v.x, wall_k<R>(P, p < 0 ? 0 : 1));
      } else {
        v.y = (R)2 * (R)(p < 0 ? RP<R>(P).T_bottom : RP<R>(P).T_top) - v.y;
      }
    }
    pt_ptr(p)[k] = v;
  };
  // the plane's (phi, T) pairs, items k0, k0 + kstep, .. < kend (tpre: the
  // value of the first item, loaded ahead)
  auto sum_plane = [&](int p, int k0, int kstep, int kend = G::HPB, const R* tpre = nullptr,
                       const P2* fpre = nullptr) {
    if constexpr (AAM != 0) {
      for (int k = k0; k < kend; k += kstep) field_put(p, k, (fpre && k == k0) ? *fpre : field_raw(p, k));
    } else {
      stage_sum_plane<S, QH, QF, EXT, G>(P, A, hf_ptr(p), pt_ptr(p), p, x0, y0, k0, kstep, kend, tpre);
    }
  };
  // RK energy solvers: the stored T of the one plane-sum item this thread
  // takes in the main loop (g role: item cidx < SUM_A; stencil role: item
  // SUM_A + cidx), read one plane ahead so that the load's latency is
  // covered by a plane's work.  p stays within z0 - 1 .. z1, like the sums.
  const int k_me = role_g ? cidx : L::SUM_A + cidx;
  const bool t_item_valid = role_g ? cidx < L::SUM_A : L::SUM_A + cidx < G::HPB;
  auto t_item = [&](int p) -> R {
    if (!t_item_valid) return (R)0;
    int pe;
    if (P.walls) pe = p < 0 ? 0 : (p >= P.nz ? P.nz - 1 : p);
    else pe = p < 0 ? p + P.nz : (p >= P.nz ? p - P.nz : p);
    int gx = x0 + k_me % G::HXB - 1, gy = y0 + k_me / G::HXB - 1;
    gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
    gy = gy < 0 ? gy + P.ny : (gy >= P.ny ? gy - P.ny : gy);
    return A.T[cell_index(P, gx, gy, pe)];
  };
  R t_cur = 0, t_next = 0;
  P2 f_cur{}, f_next{};   // in place: the item's (phi, T), one plane ahead
  if constexpr (AAM != 0) {
    if (z0 + 2 <= z1 && t_item_valid) f_cur = field_raw(z0 + 2, k_me);
  } else if constexpr (QF == 0) {
    if (z0 + 2 <= z1) t_cur = t_item(z0 + 2);
  }
  // producer / consumer barrier of a plane's phi / T sum: the g role arrives
  // once its share is written, the stencil role waits for every share
  auto sum_arrive = [&]() { asm volatile("bar.arrive 3, %0;" ::"r"(NT) : "memory"); };
  auto sum_wait = [&]() { asm volatile("bar.sync 3, %0;" ::"r"(NT) : "memory"); };

  // moments of the pulled g of plane p (g role), as GMoments
  auto moments = [&](int p) {
    const bool lo = P.walls && p == 0, hi = P.walls && p == P.nz - 1;
    const S* grow = g_ptr(p) + (size_t)ty * G::W + col;
    auto run = [&](auto btag) {
      constexpr bool BOUNCE = decltype(btag)::value;
      auto getg = [&](auto I) {
        constexpr int i = decltype(I)::value;
        // b: the source lies beyond a wall; the read is local then, and
        // always at an odd in-place level
        const bool b = BOUNCE && ((cz<27>(i) > 0 && lo) || (cz<27>(i) < 0 && hi));
        const S* p_ = grow + (size_t)i * G::GB;
        R v = Store<S>::ld_s((AAM == 1 || b) ? p_ : p_ - cx<27>(i));
        if constexpr (EXT && BOUNCE && cz<27>(i) != 0)
          if (b && P.moving_walls) v += wall_momentum<27, i, R>(P, cz<27>(i) > 0 ? 0 : 1);
        return v;
      };
      return g_moments<R>(getg);
    };
    return (lo || hi) ? run(std::true_type{}) : run(std::false_type{});
  };
  auto publish_moments = [&](int p, const GMoments<R>& m) {
    if (mode & MODE_SAVE) save_moments<S>(P, A, cell_index(P, x, y, p), m);
    *xb(p, 4) = m.jx;
    *xb(p, 5) = m.jy;
    *xb(p, 6) = m.jz;
    *xb(p, 7) = m.pst;
  };
  // g collision of plane p from its moments and B's phi(p), a(p)
  // element offsets to the planes below / above plane p (periodic wrap)
  const long long plane_el = (long long)P.NYP * P.NXP;
  auto off_below = [&](int p) { return p == 0 ? (long long)(P.nz - 1) * plane_el : -plane_el; };
  auto off_above = [&](int p) { return p == P.nz - 1 ? -(long long)(P.nz - 1) * plane_el : plane_el; };
  auto g_collide = [&](int p, const GMoments<R>& m) {
    const R phi = *xb(p, 0);
    const CellFlow<R> f = cell_velocity<R>(*xb(p, 1), *xb(p, 2), *xb(p, 3), (R)1, m.jx, m.jy, m.jz);
    const size_t pcell = pdf_index(P, x, y, p);
    if constexpr (AAM == 2) {
      const bool lo = P.walls && p == 0, hi = P.walls && p == P.nz - 1;
      const size_t pc_m = pcell + (size_t)off_below(p), pc_p = pcell + (size_t)off_above(p);
      auto run = [&](auto btag) {
        constexpr bool BOUNCE = decltype(btag)::value;
        collide_g<S>(P, A, pcell, phi, m, f, [&](auto I, R v) {
          aa_store_even<S, 27, decltype(I)::value, BOUNCE>(P, A.gd, A.g_src, pcell, pc_m, pc_p, lo, hi, v);
        });
      };
      if (lo || hi) run(std::true_type{});
      else run(std::false_type{});
    } else {
      // two grids, or in place at an odd level (dst pointers at F[opp(i)])
      collide_g<S>(P, A, pcell, phi, m, f);
    }
  };

  DiagAcc<R> dsum;   // per-thread FP64 diagnostics

  // stencil role, plane p: stencils and force; phi(p), a(p) to the exchange;
  // then (after the plane's j and p* are in the exchange) the h and f
  // collisions and the outputs.  The h/f half runs in a second call when
  // `collide_now` is false (prologue).
  Stencil27<R> fd;
  R rgx = 0, rgy = 0, rgz = 0, rlap = 0, pgx = 0, pgy = 0, pgz = 0;
  CellForce<R> F;
  P2 cen;
  auto b_stencil = [&](int p) {
    const P2* pm = pt_ptr(p - 1);
    const P2* pc = pt_ptr(p);
    const P2* pp = pt_ptr(p + 1);
    const int c0 = (ty + 1) * G::HXB + (tx + 1);
    cen = pc[c0];
    eval_pairs<G::HXB>(fd, pm, pc, pp, c0);
    if constexpr (QF == 0) {
      rk_std_pairs<P2, R, G::HXB>(pm, pc, pp, c0, rgx, rgy, rgz, rlap);
      if constexpr (EXT)
        if (P.alpha_ratio && !P.rk_iso) central_phi_pairs<P2, R, G::HXB>(pm, pc, pp, c0, pgx, pgy, pgz);
    }
    const size_t cell = cell_index(P, x, y, p);
    if (mode & MODE_SAVE) save_stencil<S>(P, A, cell, cen.x, cen.y, fd);
    F = cell_force<R, EXT>(P, x, y, p, cen.x, cen.y, fd.gpx, fd.gpy, fd.gpz, fd.lp, fd.gtx, fd.gty, fd.gtz);
    *xb(p, 0) = cen.x;
    *xb(p, 1) = F.ax;
    *xb(p, 2) = F.ay;
    *xb(p, 3) = F.az;
  };
  auto b_collide = [&](int p) {
    const R phi = cen.x, Tc = cen.y;
    const size_t cell = cell_index(P, x, y, p);
    const CellFlow<R> f = cell_velocity<R>(F.ax, F.ay, F.az, F.rho, *xb(p, 4), *xb(p, 5), *xb(p, 6));
    cell_outputs<S>(P, A, x, y, p, cell, mode, phi, Tc, *xb(p, 7), f, dsum);
    if (!(mode & MODE_COLLIDE)) return;
    const bool lo = P.walls && p == 0, hi = P.walls && p == P.nz - 1;
    const size_t pcell = pdf_index(P, x, y, p);
    const S* hrow = hf_ptr(p) + (size_t)(ty + (AAM ? 0 : 1)) * G::W + col;   // direction 0, this cell
    const R shf = (R)RP<R>(P).shift_f;
    auto run = [&](auto btag) {
      constexpr bool BOUNCE = decltype(btag)::value;
      auto geth = [&](auto I) {
        constexpr int i = decltype(I)::value;
        const bool b = BOUNCE && ((cz<QH>(i) > 0 && lo) || (cz<QH>(i) < 0 && hi));
        const S* p_ = hrow + (size_t)i * L::HFP;
        R v = Store<S>::ld_s((AAM == 1 || b) ? p_ : p_ - cx<QH>(i));
        if constexpr (EXT && BOUNCE && cz<QH>(i) != 0)
          if (b && P.moving_walls) v += phi * wall_momentum<QH, i, R>(P, cz<QH>(i) > 0 ? 0 : 1);
        return v;
      };
      auto getf = [&](auto I) {
        if constexpr (QF > 0) {
          constexpr int i = decltype(I)::value;
          const bool b = BOUNCE && ((cz<QF>(i) > 0 && lo) || (cz<QF>(i) < 0 && hi));
          const S* p_ = hrow + (size_t)(QH + i) * L::HFP;
          const R v = Store<S>::ld_s((AAM == 1 || b) ? p_ : p_ - cx<QF>(i));
          // anti-bounce-back in stored form: -v_s + 2 w_i (T_w E_i - s), E_i = 1 at rest
          return b ? (-v + (R)(2.0 * weight<QF>(i)) * abb_wall_value<S, QF, i, EXT, BOUNCE>(P, x, shf)) : v;
        } else {
          return (R)0;
        }
      };
      if constexpr (AAM == 2) {
        const size_t pc_m = pcell + (size_t)off_below(p), pc_p = pcell + (size_t)off_above(p);
        collide_h<S, QH>(P, A, pcell, phi, fd.gpx, fd.gpy, fd.gpz, f, geth, [&](auto I, R v) {
          aa_store_even<S, QH, decltype(I)::value, BOUNCE>(P, A.hd, A.h_src, pcell, pc_m, pc_p, lo, hi, v);
        });
        auto putf = [&](auto I, R v) {
          if constexpr (QF > 0)
            aa_store_even<S, QF, decltype(I)::value, BOUNCE>(P, A.fd, A.f_src, pcell, pc_m, pc_p, lo, hi, v);
        };
        if (EXT && P.alpha_ratio)
          collide_f<S, QF, EXT>(P, A, x, y, p, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf,
                                putf);
        else
          collide_f<S, QF, false>(P, A, x, y, p, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f,
                                  getf, putf);
      } else if constexpr (AAM == 1) {
        collide_h<S, QH>(P, A, pcell, phi, fd.gpx, fd.gpy, fd.gpz, f, geth);
        if (EXT && P.alpha_ratio)
          collide_f<S, QF, EXT>(P, A, x, y, p, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
        else
          collide_f<S, QF, false>(P, A, x, y, p, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
      } else {
        collide_h<S, QH>(P, A, pcell, phi, fd.gpx, fd.gpy, fd.gpz, f, geth);
        if (EXT && P.alpha_ratio)
          collide_f<S, QF, EXT>(P, A, x, y, p, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
        else
          collide_f<S, QF, false>(P, A, x, y, p, cell, pcell, phi, Tc, fd, rgx, rgy, rgz, rlap, pgx, pgy, pgz, f, getf);
      }
    };
    if (lo || hi) run(std::true_type{});
    else run(std::false_type{});
  };

  GMoments<R> mA0, mA1;   // g role: moments of planes z and z + 1 at the start of iteration z
  if (z0 < z1) {
    // ---------------- prologue: phi/T of z0 - 1 .. z0 + 1, m(z0), m(z0 + 1),
    // stencils and force of z0, h/f collisions of z0
    // (test of the timeout path: 16 bytes more than the copies deliver, so
    // the first stage never completes and its bounded wait runs out)
    issue_hf(z0 - 1, P.test_stall ? 16u : 0u);
    issue_hf(z0, 0);
    issue_hf(z0 + 1, 0);
    if (role_g) {
      issue_g(z0);
      if (GR == 2 && z0 + 1 < z1) issue_g(z0 + 1);
    }
    for (int p = z0 - 1; p <= z0 + 1; ++p) {
      ok = ok && wait_slot(hf_slot(p), hf_par(p));
      if (ok) sum_plane(p, tid, NT);
    }
    // every thread has summed HF(z0 - 1), whose slot HF(z0 + 2) reuses
    if (__syncthreads_or(!ok)) ok = false;
    if (ok) {
      if (z0 + 2 <= z1) issue_hf(z0 + 2, 0);
      if (role_g) {
        ok = wait_slot(3 + g_slot(z0), g_par(z0));
        if (ok && active) {
          mA0 = moments(z0);
          publish_moments(z0, mA0);
        }
        // after consuming G(p) its slot takes G(p + GR)
        if (z0 + GR < z1) {
          a_barrier();   // every g-role thread has read G(z0)
          if (ok) issue_g(z0 + GR);
        }
      } else if (active) {
        b_stencil(z0);
      }
    }
    // j(z0), p*(z0) and phi(z0), a(z0) are in the exchange
    if (__syncthreads_or(!ok)) ok = false;
    if (ok) {
      if (role_g) {
        if (z0 + 1 < z1) {
          ok = wait_slot(3 + g_slot(z0 + 1), g_par(z0 + 1));
          if (ok && active) {
            mA1 = moments(z0 + 1);
            publish_moments(z0 + 1, mA1);
          }
          const int next = z0 + 1 + GR;   // the slot just read takes G(z0 + 1 + GR)
          if (next < z1) {
            a_barrier();
            if (ok) issue_g(next);
          }
        }
      } else if (active) {
        b_collide(z0);
      }
    }
    if (__syncthreads_or(!ok)) ok = false;
  }

  for (int z = z0; z < z1 && ok; ++z) {
    // h/f boxes of plane z + 3 into the slot of plane z (its collisions were
    // done in the previous iteration)
    if (z + 3 <= z1) issue_hf(z + 3, 0);
    if constexpr (AAM != 0) {
      if (z + 3 <= z1 && t_item_valid) f_next = field_raw(z + 3, k_me);
    } else if constexpr (QF == 0) {
      if (z + 3 <= z1) t_next = t_item(z + 3);
    }
    if (role_g) {
      // the g role's share of phi / T of plane z + 2, first
      if (z + 2 <= z1) {
        ok = ok && wait_slot(hf_slot(z + 2), hf_par(z + 2));
        if (ok) sum_plane(z + 2, cidx, NC, L::SUM_A, QF == 0 ? &t_cur : nullptr, &f_cur);
      }
      sum_arrive();
      if (active && (mode & MODE_COLLIDE)) g_collide(z, mA0);
      mA0 = mA1;
      if (z + 2 < z1) {
        ok = ok && wait_slot(3 + g_slot(z + 2), g_par(z + 2));
        if (ok && active) {
          mA1 = moments(z + 2);
          publish_moments(z + 2, mA1);
        }
        const int next = z + 2 + GR;
        if (next < z1) {
          a_barrier();   // every g-role thread has read G(z + 2)
          if (ok) issue_g(next);
        }
      }
    } else {
      if (z + 2 <= z1) {
        ok = ok && wait_slot(hf_slot(z + 2), hf_par(z + 2));
        if (ok) sum_plane(z + 2, L::SUM_A + cidx, NC, G::HPB, QF == 0 ? &t_cur : nullptr, &f_cur);
      }
      sum_wait();   // phi / T of plane z + 2 complete (both shares)
      if (ok && z + 1 < z1 && active) {
        b_stencil(z + 1);
        b_collide(z + 1);
      }
    }
    if constexpr (AAM != 0) f_cur = f_next;
    else if constexpr (QF == 0) t_cur = t_next;
    if (__syncthreads_or(!ok)) { ok = false; break; }
  }

  if (!ok) {
    // raise the error flag, drain outstanding copies (bounded), leave
    if (tid == 0 && A.error_flag) atomicExch(A.error_flag, 1);
    for (int k = 0; k < 5; ++k)
      if (pending & (1u << k)) mbar_wait(&bar[k], (pend_par >> k) & 1u);
    return;
  }
  // the reduction's scratch reuses the h/f ring (no copies in flight)
  if (mode & MODE_DIAG) {
    double ds[kDiagVals];
    dsum.flush(ds);
    diag_block_reduce_in<NT>(ds, A.diag_partials, reinterpret_cast<double*>(smem + L::off_hf));
  }
}

// After a tiled in-place step from an even level (the skewed kernel with
// AAM = 2): the cells on the lattice's x / y edges scattered their new values
// of direction i to x + c_i, which may be a periodic ghost column or row of
// the padded arrays; copy each such ghost value to the interior cell it
// stands for.  One thread per (written ghost position, plane zd, array q):
// positions written by the columns x = 0 / nx - 1 (c_x != 0; ny of them) and
// by the rows y = 0 / ny - 1 (c_y != 0; nx, the corners counted with the
// columns).  The writers sit on plane zd - c_z; beyond a z wall they stored
// locally instead.
template <class S, int QH, int QF>
__global__ void __launch_bounds__(128) aa_fold_kernel(const DevParams P, S* __restrict__ set) {
  const int q = blockIdx.z, zd = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  int k27;
  if (q < QH) k27 = rt_to27<QH>(q);
  else if (q < QH + 27) k27 = q - QH;
  else k27 = QF == 15 ? rt_to27<15>(q - QH - 27) : q - QH - 27;
  const int ex = kDir27.c[k27][0], ey = kDir27.c[k27][1], ez = kDir27.c[k27][2];
  if (P.walls && (zd - ez < 0 || zd - ez >= P.nz)) return;
  int xs, ys;
  if (r < P.ny) {
    if (ex == 0) return;
    xs = ex > 0 ? P.nx - 1 : 0;
    ys = r;
  } else {
    const int j = r - P.ny;
    if (j >= P.nx || ey == 0) return;
    xs = j;
    ys = ey > 0 ? P.ny - 1 : 0;
    if (ex != 0 && (xs + ex < 0 || xs + ex >= P.nx)) return;   // a corner: done by the column
  }
  const int xg = xs + ex, yg = ys + ey;
  if (xg >= 0 && xg < P.nx && yg >= 0 && yg < P.ny) return;
  const int xi = xg < 0 ? xg + P.nx : (xg >= P.nx ? xg - P.nx : xg);
  const int yi = yg < 0 ? yg + P.ny : (yg >= P.ny ? yg - P.ny : yg);
  S* a = set + (size_t)q * P.Np;
  a[pdf_index(P, xi, yi, zd)] = a[pdf_index(P, xg, yg, zd)];
}



// (phi, T) of a level of the in-place layout on the tiled kernels' geometry:
// the h / f boxes of each plane are staged by tensor-TMA exactly as the
// in-place step of that level stages them (AAM = 1, odd: array i at the
// cell; AAM = 2, even: array opp(i) shifted by -c_i, or the direction's own
// array where the source lies beyond a z wall, with the periodic ghosts
// refreshed first), and each thread sums its cell's gathered populations in
// the two-grid kernels' order: phi = s_h + sum_i h*_i, T = s_f + sum_i f*_i
// with the anti-bounce-back at walls (LB; EXT: the modulated bottom wall and
// moving walls), or the stored T (RK).  A ring of two stages; one thread per
// cell of the TXB x TYB tile.
template <class S, int QH, int QF>
struct AaMomSmem {
  using G = typename BulkSmem<S, QH, QF>::G;
  static constexpr int NHF = QH + QF;
  static constexpr size_t stage = (size_t)NHF * G::GB;   // elements
  static constexpr uint32_t tx = (uint32_t)((size_t)NHF * G::W * G::TYB * sizeof(S));
  static constexpr size_t off_bar = (2 * stage * sizeof(S) + 15) & ~size_t(15);
  static constexpr size_t bytes = off_bar + 2 * sizeof(uint64_t) + 128;
};

template <class S, int QH, int QF, int AAM, bool EXT>
__global__ void __launch_bounds__(AaMomSmem<S, QH, QF>::G::NT)
aa_moments_tiled_kernel(const DevParams P, const __grid_constant__ CUtensorMap mh,
                        const __grid_constant__ CUtensorMap mf, const BulkSched sched,
                        const typename Store<S>::R* __restrict__ Tfield,
                        typename PairOf<typename Store<S>::R>::type* __restrict__ phiT, int* error_flag) {
  using R = typename Store<S>::R;
  using L = AaMomSmem<S, QH, QF>;
  using G = typename L::G;
  constexpr int NT = G::NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  S* st = (S*)smem;
  uint64_t* bar = (uint64_t*)(smem + L::off_bar);
  const int tid = threadIdx.x;
  const int tx = tid % G::TXB, ty = tid / G::TXB;
  int tcol, trow, z0, z1;
  bulk_unit(sched, P.nz, (int)blockIdx.x, tcol, trow, z0, z1);
  const int x0 = tcol * G::TXB, y0 = trow * G::TYB;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < P.nx && y < P.ny;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  } else if (tid == 32) {
    tma_prefetch_desc(&mh);
    tma_prefetch_desc(&mf);
  }
  __syncthreads();
  auto issue = [&](int p) {
    const int k = (p - z0) & 1;
    if (tid == 0) mbar_expect_tx(&bar[k], L::tx);
    issue_stage<S, G, QH, QF, 0, AAM>(P, &mh, &mh, &mf, st + (size_t)k * L::stage, &bar[k], p, x0, y0, tid,
                                      NT / 32);
  };
  const auto& rp = RP<R>(P);
  const R shh = (R)rp.shift_h, shf = (R)rp.shift_f;
  // slots with a copy in flight, and the phase parity each will complete
  uint32_t pending = 0, pend_par = 0;
  auto mark = [&](int p) {
    const int k = (p - z0) & 1;
    pending |= 1u << k;
    pend_par = (pend_par & ~(1u << k)) | ((uint32_t)(((p - z0) >> 1) & 1) << k);
  };
  bool ok = true;
  if (z0 < z1) {
    issue(z0);
    mark(z0);
    if (z0 + 1 < z1) {
      issue(z0 + 1);
      mark(z0 + 1);
    }
  }
  for (int p = z0; p < z1; ++p) {
    const int k = (p - z0) & 1;
    if (ok) {
      ok = mbar_wait(&bar[k], (uint32_t)(((p - z0) >> 1) & 1));
      if (ok) pending &= ~(1u << k);
    }
    if (ok && active) {
      const bool lo = P.walls && p == 0, hi = P.walls && p == P.nz - 1;
      const S* row = st + (size_t)k * L::stage + (size_t)ty * G::W + tx + G::GXP;
      auto run = [&](auto btag) {
        constexpr bool BOUNCE = decltype(btag)::value;
        R phi = 0;
        static_for<0, QH>([&](auto I) {
          constexpr int i = decltype(I)::value;
          const bool b = BOUNCE && ((cz<QH>(i) > 0 && lo) || (cz<QH>(i) < 0 && hi));
          const S* q = row + (size_t)i * G::GB;
          phi += Store<S>::ld_s((AAM == 1 || b) ? q : q - cx<QH>(i));
        });
        phi += shh;
        R T;
        if constexpr (QF > 0) {
          T = shf;
          static_for<0, QF>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const bool b = BOUNCE && ((cz<QF>(i) > 0 && lo) || (cz<QF>(i) < 0 && hi));
            const S* q = row + (size_t)(QH + i) * G::GB;
            const R v = Store<S>::ld_s((AAM == 1 || b) ? q : q - cx<QF>(i));
            T += b ? (-v + (R)(2.0 * weight<QF>(i)) * abb_wall_value<S, QF, i, EXT, BOUNCE>(P, x, shf)) : v;
          });
        } else {
          T = Tfield[cell_index(P, x, y, p)];
        }
        typename PairOf<R>::type v;
        v.x = phi;
        v.y = T;
        phiT[cell_index(P, x, y, p)] = v;
      };
      if (lo || hi) run(std::true_type{});
      else run(std::false_type{});
    }
    // every thread has read the stage before it takes plane p + 2
    if (__syncthreads_or(!ok)) ok = false;
    if (ok && p + 2 < z1) {
      issue(p + 2);
      mark(p + 2);
    }
  }
  if (!ok) {
    // raise the error flag, drain outstanding copies (bounded), leave
    if (tid == 0 && error_flag) atomicExch(error_flag, 1);
    for (int k = 0; k < 2; ++k)
      if (pending & (1u << k)) mbar_wait(&bar[k], (pend_par >> k) & 1u);
  }
}

}  // namespace lbm
