// wenoc_window.cuh -- the direction sweep with one cell per lane: a warp
// takes a window of 32 consecutive cells of one pencil from a dynamic queue,
// reconstructs and limits all 32 (Eq. 15-21), solves the Riemann problems at
// the 31 faces between them with the neighbour's face state from a warp
// shuffle, and updates the 30 inner cells.  The primitive states of the 32
// cells and of the two stencil cells beyond each end are copied from the
// stage's primitive slots (k_prim_slots), or, without them, converted here
// (four extra conversions for the outer cells).  Windows are handed out one
// at a time (an atomic ticket per warp), so warps that meet cheap cells take
// more windows: the cost of the limiter branches, clustered in space, no
// longer sets the time of whole SMs.
#pragma once
#include <type_traits>

#include "wenoc_sweep.cuh"

namespace wc {

constexpr int WIN = 30;        // cells updated per window
constexpr int WIN_SLOTS = 36;  // cells c0-3 .. c0+32 held in shared memory
constexpr int WIN_SLOTS_MAX = 72;  // slots of a warp whose groups hold pencil tails
constexpr int WIN_BLOCK = 128;  // threads per block unless configured

// The queue of a direction sweep: wfull full windows of WIN cells per pencil
// (window-major, pencil fastest), then the tails, wtail = n - WIN wfull cells
// of each pencil.  A tail of up to 14 cells takes a group of wtail + 2 lanes
// (the two outer lanes reconstruct its neighbours), and one warp takes the
// tails of wgrp = 32 / (wtail + 2) pencils at once; a longer tail takes a
// whole warp (wgrp = 1).  Bundling the tails saves the passes that a 32-lane
// window spends on a few cells: 18 -> 17.1 warp passes per 512-cell pencil.
struct WinPlan {
  int wfull, wtail, wgrp, slots;
  unsigned nitems;
};
inline WinPlan win_plan(int n, long npencil) {
  WinPlan w;
  w.wfull = n / WIN;
  w.wtail = n - WIN * w.wfull;
  w.wgrp = w.wtail == 0 ? 0 : (w.wtail + 2 <= 16 ? 32 / (w.wtail + 2) : 1);
  const long ntail = w.wtail == 0 ? 0 : (npencil + w.wgrp - 1) / w.wgrp;
  w.nitems = (unsigned)(npencil * w.wfull + ntail);
  w.slots = w.wgrp > 1 ? w.wgrp * (w.wtail + 6) : WIN_SLOTS;
  if (w.slots < WIN_SLOTS) w.slots = WIN_SLOTS;
  return w;
}

template <int N, int D, typename T>
struct WinSmem {
  static constexpr int SLOTD = Ring<N, D, T>::SLOTD;     // doubles per cell slot
  static constexpr int FSC = 4 * N + 2 * (D + 1);        // face values per lane
};

template <int N, int D>
__device__ __forceinline__ void shfl_face_down(const Face<N, D>& f, Face<N, D>& g) {
  using I = Idx<N, D>;
#pragma unroll
  for (int v = 0; v < I::NV; v++) g.U[v] = __shfl_down_sync(0xffffffffu, f.U[v], 1);
#pragma unroll
  for (int j = 0; j < D; j++) g.u[j] = __shfl_down_sync(0xffffffffu, f.u[j], 1);
  g.P = __shfl_down_sync(0xffffffffu, f.P, 1);
}

template <int N, int D, typename TF>
__device__ __forceinline__ void put_face(const SweepArgs& a, int side, long pencil, int c,
                                         const Face<N, D>& f) {
  using B = FaceBuf<N, D, TF>;
  using I = Idx<N, D>;
  const long np2 = a.n + 2;
  double* q = a.fbuf + ((long)side * B::K * a.npencil + pencil) * np2 + (c + 1);
  const long ks = a.npencil * np2;  // component stride
  if constexpr (B::FULL) {
#pragma unroll
    for (int v = 0; v < I::NV; v++) q[v * ks] = f.U[v];
  } else {
#pragma unroll
    for (int p = 0; p < N; p++) {
      q[p * ks] = f.U[p];
      q[(N + p) * ks] = f.U[I::A(p)];
    }
  }
  const int o = B::FULL ? I::NV : 2 * N;
#pragma unroll
  for (int j = 0; j < D; j++) q[(o + j) * ks] = f.u[j];
  q[(o + D) * ks] = f.P;
}

template <int N, int D, typename TF>
__device__ __forceinline__ void get_face(const SweepArgs& a, int side, long pencil, int c,
                                         Face<N, D>& f) {
  using B = FaceBuf<N, D, TF>;
  using I = Idx<N, D>;
  const long np2 = a.n + 2;
  const double* q = a.fbuf + ((long)side * B::K * a.npencil + pencil) * np2 + (c + 1);
  const long ks = a.npencil * np2;
  if constexpr (B::FULL) {
#pragma unroll
    for (int v = 0; v < I::NV; v++) f.U[v] = __ldg(q + v * ks);
  } else {
#pragma unroll
    for (int p = 0; p < N; p++) {
      f.U[p] = __ldg(q + p * ks);
      f.U[I::A(p)] = __ldg(q + (N + p) * ks);
    }
#pragma unroll
    for (int j = 0; j < D; j++) f.U[I::U(j)] = 0.0;  // not read by the remainder form
    f.U[I::E] = 0.0;
  }
  const int o = B::FULL ? I::NV : 2 * N;
#pragma unroll
  for (int j = 0; j < D; j++) f.u[j] = __ldg(q + (o + j) * ks);
  f.P = __ldg(q + (o + D) * ks);
}

// Eq. 3 (Eq. 5 for kind 1) for one cell from the fluxes at its two faces
// (F right, Fl left) and u-hat there, applied per a.mode: L = part, L +=
// part, or the Runge-Kutta stage with the direction accumulator.
template <int N, int D, int LW>
__device__ __forceinline__ void update_cell(const SweepArgs& a, const Mat& m, long cell,
                                            const double* F, const double* Fl, double uh,
                                            double uhl, const double* Ub, double Pb, double dt,
                                            unsigned& bad) {
  using I = Idx<N, D>;
  constexpr int NV = I::NV;
  const double du = (uh - uhl) * a.inv_dx;
  // Eq. 3: -div F + alpha (1 + K) div u_hat;  Eq. 5: +div F^PF
  const double sdx = a.kind == 1 ? a.inv_dx : -a.inv_dx;
  // (the source factors serve Eq. 3 only; Eq. 5 has no source term)
  double sf[N] = {};
  if (a.kind == 0) source_factors<N, D>(m, Ub, Pb, sf);
  const double r2dt = a.rk2 * dt;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double val = (F[v] - Fl[v]) * sdx;
    if (a.kind == 0 && v >= N + D + 1) val = fma(sf[v - (N + D + 1)], du, val);
    const long idx = (long)v * a.ncell + cell;
    if (not_finite(val)) bad |= ST_NAN;
    if (a.mode == 0) {
      a.L[idx] = val;
    } else if (a.mode == 1) {
      a.L[idx] += val;
    } else {
      const double Lt = a.mode == 2 ? a.L[idx] + val : val;
      // masses >= 0 and fractions in [0, 1] up to the rounding of the
      // stage sum (not in the comparison schemes, which have no bounds)
      a.Uout[idx] = rk_combine(a.rk0, a.U0[idx], a.rk1, Ub[v], r2dt, Lt,
                               LW != 2 && (v < N || v >= I::A(0)), v >= I::A(0));
    }
  }
}

// update_cell for a cell of the Phase-Field step (kind 1) whose two faces
// carry no flux (G_p = 0 for every phase on both): F = Fl = 0, so the value
// of each variable is (0 - 0) a.inv_dx = 0 and the cell takes the same
// stage combination as update_cell gives it, without its face states.  A
// non-finite cell value is reported as update_cell reports it through the
// faces it spoils.  Kept out of line: the hot sweep's code stays as small.
template <int N, int D, int LW>
__device__ __noinline__ unsigned update_cell_still(const SweepArgs& a, long cell, double dt) {
  using I = Idx<N, D>;
  unsigned bad = 0u;
  const double r2dt = a.rk2 * dt;
#pragma unroll 1
  for (int v = 0; v < I::NV; v++) {
    const long idx = (long)v * a.ncell + cell;
    const double ub = __ldg(a.U + idx);
    if (not_finite(ub)) bad |= ST_NAN;
    if (a.mode == 0) {
      a.L[idx] = 0.0;
    } else if (a.mode == 1) {
      a.L[idx] += 0.0;
    } else {
      const double Lt = a.mode == 2 ? a.L[idx] + 0.0 : 0.0;
      a.Uout[idx] = rk_combine(a.rk0, a.U0[idx], a.rk1, ub, r2dt, Lt,
                               LW != 2 && (v < N || v >= I::A(0)), v >= I::A(0));
    }
  }
  return bad;
}

// One window: the warp's lanes form groups of G consecutive lanes (one group
// of 32 for a full window); lane j of a group owns cell c = c0 - 1 + j of the
// pencil at `base`, and slot sb + s of `slots` holds the primitive state of
// cell c0 - 3 + s (pressure in FP64, V in T), s = 0 .. G + 3.  Lanes
// 1 .. G - 2 of an active group update cells c0 .. c0 + G - 3 (those below
// a.n).  A lane with store = false (beyond the last group) keeps its slots
// untouched and updates nothing.  Variant LW as in sweep_segment (0 scheme,
// 1 learned weights, 2 comparison schemes).
//
// PART = 1 (the split sweep's face pass) stops after the limiter chain: the
// face states of the cells -1 .. n go to a.fbuf with the cells' pressures,
// and the flux pass (k_flux_win) does the rest.
template <int N, int D, typename T, typename TF, int LW, int PART>
__device__ __forceinline__ void sweep_window(const SweepArgs& a, const Mat& m, long base,
                                             long pencil, int c0, int j, int G, int sb,
                                             bool active, bool store, double* slots,
                                             double* fsc, double dt, unsigned& bad,
                                             unsigned* lstat) {
  using I = Idx<N, D>;
  constexpr int NV = I::NV;
  constexpr int SLOTD = WinSmem<N, D, T>::SLOTD;
  // cells beyond the three ghost layers (lanes past the end of a short
  // pencil, whose results are not used) read the outermost ghost: the
  // boundary maps stay inside the pencil
  auto ghost_clamp = [&](int c) { return c < -3 ? -3 : (c > a.n + 2 ? a.n + 2 : c); };
  auto load_cons = [&](int c, double* u) {
    bool flip;
    const int j = bc_index(ghost_clamp(c), a.n, a.bclo, a.bchi, flip);
    const long cell = base + (long)j * a.stride;
#pragma unroll
    for (int k = 0; k < NV; k++) u[k] = __ldg(a.U + (long)k * a.ncell + cell);
#pragma unroll
    for (int jj = 0; jj < D; jj++) {
      long long mask = (flip && jj == a.dir) ? (long long)0x8000000000000000ULL : 0LL;
      u[I::U(jj)] = __longlong_as_double(__double_as_longlong(u[I::U(jj)]) ^ mask);
    }
  };
  auto store_slot = [&](int s, const double* u, double* v) {
    cons_to_prim<N, D>(m, u, v);
    put_slot<N, D, T>(slots + s * SLOTD, v);
  };
  // reduced precision: mass and fraction faces = FP64 cell value (a
  // conservative and primitive variable alike) + offset in T
  constexpr bool OFFSET = !std::is_same<T, double>::value;

  const int c = c0 - 1 + j;
  double Ub[NV], Vtmp[NV];
  load_cons(c, Ub);
  // Phase-Field step (kind 1): the gradients G_p at x_{c+1/2} from Q and the
  // cell fractions on both sides.  A face with G_p = 0 for every phase carries
  // no flux (Eq. 5 with R12's flux: every term has a factor max(G_p, 0) or
  // min(G_p, 0)), so a window in which every face that an owned cell touches
  // has G = 0 leaves those cells unchanged: its cells take the update of a
  // zero flux (the face pass writes no faces, which the flux pass then does
  // not read), and the reconstruction, limiter and flux are skipped.  Only
  // the interface band and its neighbours carry a flux.  (Not with the face
  // dump of wc_faces, which wants every face.)
  if (a.kind == 1 && !a.faceL) {
    bool flip;
    const long cq =
        base + (long)bc_index(ghost_clamp(c), a.n, a.bclo, a.bchi, flip) * a.stride;
    bool loud = false;
#pragma unroll
    for (int p = 0; p < N; p++) {
      const double q = __ldg(a.Q + (long)p * a.ncell + cq);
      const double qn = __shfl_down_sync(0xffffffffu, q, 1);
      const double an = __shfl_down_sync(0xffffffffu, Ub[I::A(p)], 1);
      // (unlimited here: a limit |G| <= g > 0 keeps G = 0 where it is 0, and
      // the face pass has no time step for it)
      const double gq = pf_gradient(q, qn, Ub[I::A(p)], an, a.inv_dx, 0.0);
      loud = loud || (dbits(gq) & 0x7FFFFFFFFFFFFFFFLL) != 0;
    }
    // (lane j - 1 holds the face x_{c-1/2})
    const bool loud_left = __shfl_up_sync(0xffffffffu, (int)loud, 1) != 0;
    // the cells whose face states this window provides: the updated ones
    // (PART 0), or the owned ones with the boundary cells -1 and n (PART 1)
    bool need = active && j >= 1 && j <= G - 2 && c < a.n;
    if constexpr (PART == 1) need = need || (active && (c == -1 || c == a.n));
    if (__ballot_sync(0xffffffffu, need && (loud || loud_left)) == 0u) {
      if constexpr (PART == 0) {
        if (need) bad |= update_cell_still<N, D, LW>(a, base + (long)c * a.stride, dt);
      }
      __syncwarp();
      return;
    }
  }
  if (store && a.Vs) {
    // the slots from the stage's primitive slots; a mirrored boundary image
    // (reflective side) is converted here from its flipped state
    auto fill_slot = [&](int s, int cc, const double* u0) {
      bool flip;
      const int jj = bc_index(ghost_clamp(cc), a.n, a.bclo, a.bchi, flip);
      if (!flip) {
        copy_slot<N, D, T>(a, base + (long)jj * a.stride, slots + s * SLOTD);
      } else {
        double u[NV], v[NV];
        if (u0) {
#pragma unroll
          for (int k = 0; k < NV; k++) u[k] = u0[k];
        } else {
          load_cons(cc, u);
        }
        store_slot(s, u, v);
      }
    };
    fill_slot(sb + j + 2, c, Ub);
    for (int e = j; e < 4; e += G) {
      const int s = e < 2 ? e : G + e;
      fill_slot(sb + s, c0 - 3 + s, nullptr);
    }
  } else if (store) {
    store_slot(sb + j + 2, Ub, Vtmp);
    // the group's outer stencil cells: slots 0, 1, G + 2, G + 3
    for (int e = j; e < 4; e += G) {
      const int s = e < 2 ? e : G + e;
      double u[NV], v[NV];
      load_cons(c0 - 3 + s, u);
      store_slot(sb + s, u, v);
    }
  }
  __syncwarp();
  const T* V[5];
#pragma unroll
  for (int k = 0; k < 5; k++)
    V[k] = reinterpret_cast<const T*>(slots + (sb + j + k) * SLOTD + 1);
  const double Pb = slots[(sb + j + 2) * SLOTD];

  // The reconstructions of the variables run in loops that are not
  // unrolled: one copy of the weight and candidate code serves every
  // variable, which keeps the window's hot code small enough for the
  // instruction cache.  Each lane's face values go through its column of the
  // warp's scratch (fsc[k * 32]): masses L/R, fractions L/R, then the
  // velocity components and the pressure L/R.
  {
    bool flip;
    const long cellc = base + (long)bc_index(ghost_clamp(c), a.n, a.bclo, a.bchi, flip) * a.stride;
    // Eq. 16: masses and fractions with the weights of the masses
#pragma unroll 1
    for (int p = 0; p < N; p++) {
      const int ia = I::A(p);
      Stencil<T> st = stencil<T>(V[0][p], V[1][p], V[2][p], V[3][p], V[4][p]);
      W6<T> w = sweep_weights<LW, T>(m, st);
      const Stencil<T> sa = stencil<T>(V[0][ia], V[1][ia], V[2][ia], V[3][ia], V[4][ia]);
      if constexpr (LW == 1) {
        // learned weights of an interior cell, accepted per face side when
        // the mass and the fraction reconstructed with them are each within
        // tau times their stencil's range of the plain reconstructions
        // (boundary cells keep the plain weights)
        if (p < 3 && c >= 0 && c < a.n) {
          const float* Wp = a.Wm + (long)(3 * p) * a.ncell + base + (long)c * a.stride;
          W6<T> wl;
          wl.aL0 = T(__ldg(Wp));
          wl.aL1 = T(__ldg(Wp + a.ncell));
          wl.aL2 = T(__ldg(Wp + 2 * a.ncell));
          wl.aR0 = T(__ldg(Wp + 9 * a.ncell));
          wl.aR1 = T(__ldg(Wp + 10 * a.ncell));
          wl.aR2 = T(__ldg(Wp + 11 * a.ncell));
          wl.invL = wl.invR = T(1) / T(6);
          bool okL = true, okR = true, flat = true;
          auto judge = [&](const Stencil<T>& q) {
            // offsets from the cell value with the plain and the learned weights
            T pl, pr, ql, qr;
            offsets(w, q, pl, pr);
            offsets(wl, q, ql, qr);
            const T hi = fmax(fmax(fmax(T(0), q.da), fmax(q.db, q.dd)), q.de);
            const T lo = fmin(fmin(fmin(T(0), q.da), fmin(q.db, q.dd)), q.de);
            const T tol = T(a.tau) * (hi - lo);
            okL = okL && fabs(ql - pl) <= tol;
            okR = okR && fabs(qr - pr) <= tol;
            flat = flat && !(hi > lo);
          };
          judge(st);
          judge(sa);
          if (okL) {
            w.aL0 = wl.aL0;
            w.aL1 = wl.aL1;
            w.aL2 = wl.aL2;
            w.invL = wl.invL;
          }
          if (okR) {
            w.aR0 = wl.aR0;
            w.aR1 = wl.aR1;
            w.aR2 = wl.aR2;
            w.invR = wl.invR;
          }
          if (!flat) {
            lstat[0] += 2u;
            lstat[1] += unsigned(!okL) + unsigned(!okR);
          }
        }
      }
      // (the comparison schemes: the fraction with its own weights)
      W6<T> wa = w;
      if constexpr (LW == 2) wa = sweep_weights<LW, T>(m, sa);
      double ml, mr, al, ar;
      if constexpr (OFFSET) {
        reconstruct_offset(w, st, __ldg(a.U + (long)p * a.ncell + cellc), ml, mr);
        reconstruct_offset(wa, sa, __ldg(a.U + (long)ia * a.ncell + cellc), al, ar);
      } else {
        T fl, fr;
        reconstruct(w, st, fl, fr);
        ml = wide(fl);
        mr = wide(fr);
        reconstruct(wa, sa, fl, fr);
        al = wide(fl);
        ar = wide(fr);
      }
      fsc[(4 * p + 0) * 32] = ml;
      fsc[(4 * p + 1) * 32] = mr;
      fsc[(4 * p + 2) * 32] = al;
      fsc[(4 * p + 3) * 32] = ar;
    }
  }
  // velocity and pressure, each with its own weights
  face_velocity_pressure_rolled<N, D, T, LW>(m, V, Pb, fsc + 4 * N * 32);
  double mL[N], mR[N], aL[N], aR[N], uL[D], uR[D], PL, PR;
#pragma unroll
  for (int p = 0; p < N; p++) {
    mL[p] = fsc[(4 * p + 0) * 32];
    mR[p] = fsc[(4 * p + 1) * 32];
    aL[p] = fsc[(4 * p + 2) * 32];
    aR[p] = fsc[(4 * p + 3) * 32];
  }
#pragma unroll
  for (int q = 0; q < D; q++) {
    uL[q] = fsc[(4 * N + 2 * q) * 32];
    uR[q] = fsc[(4 * N + 2 * q + 1) * 32];
  }
  PL = fsc[(4 * N + 2 * D) * 32];
  PR = fsc[(4 * N + 2 * D + 1) * 32];
  Face<N, D> fL, fR;
  limit_chain<N, D, LW != 2>(m, Ub, Pb, mL, aL, mR, aR, uL, PL, uR, PR, a.energy_limiter, fL, fR,
                    nullptr);
  if (a.faceL && active && j >= 1 && j <= G - 2 && c < a.n) {
    const long cell = base + (long)c * a.stride;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      a.faceL[(long)v * a.ncell + cell] = fL.U[v];
      a.faceR[(long)v * a.ncell + cell] = fR.U[v];
    }
  }
  if constexpr (PART == 1) {
    // the cells this group owns, and the boundary cells -1 and n at the
    // pencil's ends (the first and the last window hold them)
    const bool own = active && ((j >= 1 && j <= G - 2 && c < a.n) || c == -1 || c == a.n);
    if (own) {
      put_face<N, D, TF>(a, 0, pencil, c, fL);
      put_face<N, D, TF>(a, 1, pencil, c, fR);
      a.fbuf[(2L * FaceBuf<N, D, TF>::K * a.npencil + pencil) * (a.n + 2) + (c + 1)] = Pb;
    }
    __syncwarp();  // the slots are refilled by the next window
    return;
  }
  // the face x_{c+1/2}: this lane's fL and the right neighbour's fR
  Face<N, D> fRn;
  shfl_face_down<N, D>(fR, fRn);
  double F[NV], uh = 0.0;
  if (a.kind == 1) {
    double q[N], G[N];
    bool flip;
    const long cell =
        base + (long)bc_index(ghost_clamp(c), a.n, a.bclo, a.bchi, flip) * a.stride;
#pragma unroll
    for (int p = 0; p < N; p++) q[p] = __ldg(a.Q + (long)p * a.ncell + cell);
#pragma unroll
    for (int p = 0; p < N; p++) {
      const double qn = __shfl_down_sync(0xffffffffu, q[p], 1);
      const double an = __shfl_down_sync(0xffffffffu, Ub[I::A(p)], 1);
      G[p] = pf_gradient(q[p], qn, Ub[I::A(p)], an, a.inv_dx,
                         a.gcoef > 0.0 ? a.gcoef / dt : a.gmax);
    }
    pf_flux<N, D>(m, fL, fRn, G, F);
  } else {
    riemann<N, D, TF>(m, a.dir, a.hllc, fL, fRn, F, uh);
  }
  // the face x_{c-1/2} from the left neighbour
  double Fl[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) Fl[v] = __shfl_up_sync(0xffffffffu, F[v], 1);
  const double uhl = __shfl_up_sync(0xffffffffu, uh, 1);
  if (active && j >= 1 && j <= G - 2 && c < a.n)
    update_cell<N, D, LW>(a, m, base + (long)c * a.stride, F, Fl, uh, uhl, Ub, Pb, dt, bad);
  __syncwarp();  // the slots are refilled by the next window
}

// Persistent launch: every warp takes windows (pencil fastest, so warps that
// run together read neighbouring pencils) from the queue a.ticket[0] until
// it is empty; the last warp to leave resets the queue for the next launch.
// Minimum resident blocks for the register budget: every window sweep is
// held to 128 registers, four blocks (16 warps) an SM instead of three.  The
// reduced precisions' face pass spills 16-64 bytes a thread and keeps its
// FP64 pipe busier (mixed step on the 2048^2 N = 3 circles 18.24 -> 17.73
// ms; 192^3 3-D spheres 57.5 -> 55.1 ms); the FP64 sweep (142 registers
// otherwise, 56-116 bytes of spills) gains 0.6 % (36.00 -> 35.80 ms a step;
// 3-D 108.85 -> 108.24 ms).
#ifndef WC_WIN_MINB64
#define WC_WIN_MINB64 4
#endif
#ifndef WC_WIN_MINB32
#define WC_WIN_MINB32 4
#endif
template <int N, int D, typename T, typename TF, int LW = 0, int PART = 0>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? WC_WIN_MINB64 : WC_WIN_MINB32)
    k_sweep_win(SweepArgs a, Mat m) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  using WS = WinSmem<N, D, T>;
  double* slots = smem + (threadIdx.x >> 5) * (a.wslots * WS::SLOTD + 32 * WS::FSC);
  double* fsc = slots + a.wslots * WS::SLOTD + lane;  // this lane's scratch column
  const unsigned nitems = a.nitems;
  const unsigned nfull = (unsigned)(a.npencil * a.wfull);
  unsigned bad = 0u;
  unsigned lstat[2] = {0u, 0u};
  double dt = 0.0;
  // the stage modes, and every direction of a Phase-Field stage (its gradient
  // limit is gcoef / dt)
  if (PART == 0 && (a.mode >= 2 || a.gcoef > 0.0))
    dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.cfl / *a.rate;
  for (;;) {
    unsigned it = 0u;
    if (lane == 0) it = atomicAdd(a.ticket, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= nitems) break;
    long tr;
    int c0, G = 32, j = lane, sb = 0;
    bool active = true, store = true;
    if (it < nfull) {
      tr = (long)(it % (unsigned)a.npencil);
      c0 = (int)(it / (unsigned)a.npencil) * WIN;
    } else {
      const unsigned t = it - nfull;
      c0 = a.wfull * WIN;
      if (a.wgrp <= 1) {
        tr = (long)t;
      } else {
        // tails of pencils t wgrp .. t wgrp + wgrp - 1, one per group
        G = a.wtail + 2;
        int gi = lane / G;
        j = lane - gi * G;
        if (gi >= a.wgrp) {  // lanes past the last group: read its slots only
          gi = a.wgrp - 1;
          j = G - 1;
          active = store = false;
        }
        sb = gi * (G + 4);
        tr = (long)t * a.wgrp + gi;
        if (tr >= a.npencil) {  // past the last pencil: a copy of it, no update
          tr = a.npencil - 1;
          active = false;
        }
      }
    }
    const long base = pencil_base(a, tr);
    sweep_window<N, D, T, TF, LW, PART>(a, m, base, tr, c0, j, G, sb, active, store, slots, fsc,
                                        dt, bad, lstat);
  }
  if (lane == 0) {
    __threadfence();
    const unsigned done = atomicAdd(a.ticket + 1, 1u);
    if (done == a.nwarps - 1) {
      a.ticket[0] = 0u;
      a.ticket[1] = 0u;
    }
  }
  if (bad) atomicOr(a.status, bad);
  if constexpr (LW == 1) {
    if (a.lcount) {
#pragma unroll
      for (int k = 0; k < 2; k++) {
        unsigned v = lstat[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(a.lcount + k, (unsigned long long)v);
      }
    }
  }
}

// Launch of the window sweep: bps resident blocks of `block` threads (32,
// 64, 96 or 128: one to four warps) on every SM (persistent; bps <= 0: the
// occupancy limit), at most one warp per window.  Smaller blocks let the
// register file hold more warps (at 104 registers a thread an SM takes 19
// one-warp blocks but only 4 blocks of four warps); the FP64 sweep runs
// equally fast with either, its FP64 pipe being as busy at 16 warps as at 19.
// Number of SMs of the current device (cached per device ordinal).
inline int device_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      return 148;
    cache[dev] = n;
  }
  return cache[dev];
}

// The flux pass of the split sweep: a warp takes windows of WINF cells of a
// pencil (pencil fastest; a static grid-stride walk: the cost per face is
// nearly uniform); lane j solves the Riemann problem at the face between
// cells c = c0 - 1 + j and c + 1 from the face states the face pass stored
// (the right state of cell c + 1 may be the boundary cell n), and lanes
// 1 .. 31 update their cells with the left neighbour's flux.
constexpr int WINF = 31;
template <int N, int D, typename TF, int LW>
__global__ void __launch_bounds__(128) k_flux_win(SweepArgs a, Mat m) {
  using I = Idx<N, D>;
  constexpr int NV = I::NV;
  const int lane = threadIdx.x & 31;
  const long nwf = (a.n + WINF - 1) / WINF;
  const long items = a.npencil * nwf;
  const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
  unsigned bad = 0u;
  double dt = 0.0;
  if (a.mode >= 2 || a.gcoef > 0.0) dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.cfl / *a.rate;
  for (long it = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nwarps) {
    const long tr = it % a.npencil;
    const int c0 = (int)(it / a.npencil) * WINF;
    const long base = pencil_base(a, tr);
    const int c = c0 - 1 + lane;
    const bool live = c <= a.n - 1;
    const int cc = live ? c : a.n - 1;  // lanes past the pencil's end: a copy, no update
    Face<N, D> fL, fR;
    double F[NV], uh = 0.0;
    if (a.kind == 1) {
      double G[N];
      bool flip, loud = false;
      const long cl = base + (long)bc_index(cc, a.n, a.bclo, a.bchi, flip) * a.stride;
      const long cr = base + (long)bc_index(cc + 1, a.n, a.bclo, a.bchi, flip) * a.stride;
#pragma unroll
      for (int p = 0; p < N; p++) {
        const long o = (long)I::A(p) * a.ncell;
        G[p] = pf_gradient(__ldg(a.Q + (long)p * a.ncell + cl), __ldg(a.Q + (long)p * a.ncell + cr),
                           __ldg(a.U + o + cl), __ldg(a.U + o + cr), a.inv_dx,
                           a.gcoef > 0.0 ? a.gcoef / dt : a.gmax);
        loud = loud || (dbits(G[p]) & 0x7FFFFFFFFFFFFFFFLL) != 0;
      }
      // a face with G = 0 carries no flux; its face states, which the face
      // pass did not write where every face near them has G = 0, are not read
      if (loud) {
        get_face<N, D, TF>(a, 0, tr, cc, fL);
        get_face<N, D, TF>(a, 1, tr, cc + 1, fR);
        pf_flux<N, D>(m, fL, fR, G, F);
      } else {
#pragma unroll
        for (int v = 0; v < NV; v++) F[v] = 0.0;
      }
    } else {
      get_face<N, D, TF>(a, 0, tr, cc, fL);
      get_face<N, D, TF>(a, 1, tr, cc + 1, fR);
      riemann<N, D, TF>(m, a.dir, a.hllc, fL, fR, F, uh);
    }
    double Fl[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) Fl[v] = __shfl_up_sync(0xffffffffu, F[v], 1);
    const double uhl = __shfl_up_sync(0xffffffffu, uh, 1);
    if (lane >= 1 && live) {
      const long cell = base + (long)c * a.stride;
      double Ub[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) Ub[v] = __ldg(a.U + (long)v * a.ncell + cell);
      const double Pb = __ldg(a.fbuf + (2L * FaceBuf<N, D, TF>::K * a.npencil + tr) * (a.n + 2) +
                              (c + 1));
      update_cell<N, D, LW>(a, m, cell, F, Fl, uh, uhl, Ub, Pb, dt, bad);
    }
  }
  if (bad) atomicOr(a.status, bad);
}

template <int N, int D, typename T, typename TF, int LW, int PART = 0>
cudaError_t launch_window(const SweepArgs& a0, const Mat& m, int block, int bps,
                          cudaStream_t st) {
  if (block < 32 || block > 128 || block % 32 != 0) return cudaErrorInvalidValue;
  if (a0.wslots < WIN_SLOTS || a0.wslots > WIN_SLOTS_MAX) return cudaErrorInvalidValue;
  const int smem =
      (a0.wslots * WinSmem<N, D, T>::SLOTD + 32 * WinSmem<N, D, T>::FSC) * 8 * (block / 32);
  auto k = k_sweep_win<N, D, T, TF, LW, PART>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long items = a0.nitems;
  if (bps <= 0) {
    // as many resident blocks as registers and shared memory allow (queried
    // once per instantiation and block size; every caller gets the same
    // answer)
    static int occ[4] = {0, 0, 0, 0};
    int& o = occ[block / 32 - 1];
    if (o == 0) {
      int q = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k, block, smem);
      if (e != cudaSuccess) return e;
      o = q < 1 ? 1 : q;
    }
    bps = o;
  }
  long blocks = (long)device_sms() * bps;
  const long need = (items + block / 32 - 1) / (block / 32);
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  SweepArgs a = a0;
  a.nwarps = (unsigned)(blocks * (block / 32));
  k<<<(unsigned)blocks, block, smem, st>>>(a, m);
  return cudaGetLastError();
}

// The split sweep: the face pass (reconstruction and limiter chain into
// a.fbuf), then the flux pass (Riemann problems and update).  Two compact
// kernels instead of one long loop body: more warps fit, and the hot code
// of each fits the instruction cache.
template <int N, int D, typename T, typename TF, int LW>
cudaError_t launch_split(const SweepArgs& a, const Mat& m, int block, cudaStream_t st) {
  cudaError_t e = launch_window<N, D, T, TF, LW, 1>(a, m, block, 0, st);
  if (e != cudaSuccess) return e;
  auto k = k_flux_win<N, D, TF, LW == 2 ? 2 : 0>;
  static int occ = 0;
  if (occ == 0) {
    int q = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k, 128, 0);
    if (e != cudaSuccess) return e;
    occ = q < 1 ? 1 : q;
  }
  const long items = a.npencil * ((a.n + WINF - 1) / WINF);
  long blocks = (long)device_sms() * occ;
  const long need = (items + 3) / 4;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  k<<<(unsigned)blocks, 128, 0, st>>>(a, m);
  return cudaGetLastError();
}

}  // namespace wc
