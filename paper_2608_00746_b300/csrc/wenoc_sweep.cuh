// wenoc_sweep.cuh -- the direction sweep: one launch per direction per
// Runge-Kutta stage evaluates that direction's part of Eq. 3 for every cell.
//
// Each thread owns a segment of `seg` consecutive cells of one pencil along
// the sweep direction and marches through it.  Consecutive threads own
// consecutive pencils, so for the y and z sweeps a warp reads 32 consecutive
// x cells of each variable (coalesced structure-of-arrays loads).  A ring of
// five primitive states per thread in shared memory holds the stencil; each
// cell's primitive state is computed once per sweep.  For every cell the
// thread reconstructs both faces (Eq. 15-21), solves the Riemann problem at
// the left face with the previous cell's right-face state kept in registers,
// and updates the previous cell.  Boundary cells come from the boundary
// condition on the fly (no ghost storage).
#pragma once
#include <type_traits>

#include "wenoc_device.cuh"

namespace wc {

struct SweepArgs {
  const double* U;     // state differentiated by this sweep [NV][ncell]
  double* L;           // direction accumulator / rhs output [NV][ncell]
  const double* U0;    // Runge-Kutta base state U^n (stage modes)
  double* Uout;        // Runge-Kutta destination
  const double* rate;  // device max rate (dt = cfl / rate) or null
  double cfl, dt_fixed;
  double rk0, rk1, rk2;  // Uout = rk0 U0 + rk1 U + rk2 dt L
  long ncell;
  int nx, ny, nz;
  int dir;             // 0, 1, 2
  int n;               // cells along dir
  long stride;         // index step along dir
  long npencil;        // ncell / n
  int nseg, seg;       // segments per pencil, cells per segment
  long max_threads;    // launch size cap (whole blocks per SM); items loop beyond it
  const double* Q;     // Phase-Field auxiliary fields [N][ncell] (kind 1)
  double gmax;         // kind 1: limit of |grad Q| on a face (0 = none) ...
  double gcoef;        // ... or, in the stage modes, gcoef / dt when gcoef > 0
  int kind;            // 0: hyperbolic step (Eq. 3); 1: Phase-Field step (Eq. 5)
  double inv_dx;
  int bclo, bchi;
  int mode;            // 0: L = dir part; 1: L += dir part; 2: stage with L + dir part; 3: stage with dir part only
  int hllc;
  int energy_limiter;
  unsigned* status;
  // learned weights (template LW = 1): the surrogate's weights of the masses
  // for this direction, W[(9 side + 3 p + s) ncell + cell]; tau is the
  // acceptance threshold; lcount[0] counts face sides decided, lcount[1]
  // those that fell back to the plain weights
  const float* Wm;
  float tau;
  unsigned long long* lcount;
  // window schedule (nwin > 0, wenoc_window.cuh): windows per pencil, the
  // two-word queue (next window, warps finished) and the launched warps;
  // the queue's plan (WinPlan: full windows per pencil, tail cells, tails
  // per warp, queue items) and the slots a warp holds
  int nwin;
  unsigned* ticket;
  unsigned nwarps;
  int wfull, wtail, wgrp, wslots;
  unsigned nitems;
  // face dump (window schedule only; null in the operator's own launches):
  // the limited conservative face states U^L_{i+1/2} and U^R_{i-1/2} of
  // every cell, [NV][ncell] each
  double* faceL;
  double* faceR;
  // split sweep (fbuf not null): the face pass writes the limited face
  // states of the cells -1 .. n of every pencil (boundary cells included)
  // and the cells' pressures there, and the flux pass reads them.  Layout:
  // fbuf[((side * K + k) * npencil + pencil) * (n + 2) + c + 1], k < K the
  // stored components of a face state (FaceBuf), then the pressures
  // fbuf[(2 K * npencil + pencil) * (n + 2) + c + 1]
  double* fbuf;
  // pencils of a set of equal cube patches (window schedule; null for a
  // grid): pencil tr lies in patch tr / (nx ny), whose first cell in the
  // pooled state is poff[tr / (nx ny)], at the patch's own pencil tr % (nx ny)
  const long* poff;
  // first pencil of a band launch (pencils tr0 .. tr0 + npencil - 1 of the
  // grid's direction sweep; 0 for the whole sweep): the host-buffer step
  // starts the first sweep on the rows already uploaded and returns the
  // last sweep's bands while the next ones run
  long tr0;
  // primitive slots of the state U (window schedule; null: each sweep
  // converts its cells itself): the put_slot image of every cell, word k of
  // cell c at Vs[k ncell + c], written once a stage by k_prim_slots and
  // copied by the sweeps of its directions
  const double* Vs;
};

// First cell of pencil tr of a direction sweep (x fastest; for dir 1 the
// pencils run over x, then z).
__device__ __forceinline__ long pencil_base(const SweepArgs& a, long tr) {
  long o = 0;
  tr += a.tr0;
  if (a.poff) {
    const long np = (long)a.nx * a.ny;  // pencils a patch (cube: every direction)
    o = __ldg(a.poff + tr / np);
    tr %= np;
  }
  if (a.dir == 0) return o + tr * a.nx;
  if (a.dir == 1) return o + (tr / a.nx) * ((long)a.nx * a.ny) + tr % a.nx;
  return o + tr;
}

// The components of a face state that the flux pass needs: all of U, the
// velocity and the pressure for an FP64 flux (the physical fluxes of Eq. 1);
// for a reduced-precision flux (remainder form) the masses, fractions,
// velocity and pressure only.
template <int N, int D, typename TF>
struct FaceBuf {
  static constexpr int NV = 2 * N + D + 1;
  static constexpr bool FULL = sizeof(TF) == 8;
  static constexpr int K = FULL ? NV + D + 1 : NV;
};
__host__ __device__ inline long fbuf_doubles(int K, long npencil, int n) {
  return (2L * K + 1) * npencil * (n + 2);
}

enum { BC_PERIODIC = 0, BC_REFLECTIVE = 1, BC_OUTFLOW = 2 };

__device__ __forceinline__ int bc_index(int j, int n, int bclo, int bchi, bool& flip) {
  flip = false;
  if (j < 0) {
    if (bclo == BC_PERIODIC) return j + n * ((-j + n - 1) / n);
    if (bclo == BC_REFLECTIVE) {
      flip = true;
      return -1 - j;
    }
    return 0;
  }
  if (j >= n) {
    if (bchi == BC_PERIODIC) return j % n;
    if (bchi == BC_REFLECTIVE) {
      flip = true;
      return 2 * n - 1 - j;
    }
    return n - 1;
  }
  return j;
}

// Ring slot layout in shared memory (per thread, 5 slots): the pressure in
// FP64 (for psi at the cell average) and the primitive state V[NV] in the
// reconstruction precision T.  Conservative cell values are re-read from
// global memory (L1-resident: each cell is read twice within 3 iterations).
//
// In reduced precision a slot also holds, after V, the residues
// v - (double) cvt<T>(v) of the velocity components and the pressure in T
// (hi/lo pairs), so their stencil differences are known to the precision of
// the differences themselves, not of the values.
template <int N, int D, typename T>
struct Ring {
  static constexpr int NV = Idx<N, D>::NV;
  static constexpr bool HILO = !std::is_same<T, double>::value;
  static constexpr int SLOT_BYTES = 8 + (NV + (HILO ? D + 1 : 0)) * (int)sizeof(T);
  static constexpr int SLOTD = (SLOT_BYTES + 7) / 8;   // doubles per slot
  static constexpr int BYTES = 5 * SLOTD * 8;          // per thread
};

// Fills a slot from the FP64 primitive state v of a cell.
template <int N, int D, typename T>
__device__ __forceinline__ void put_slot(double* sl, const double* v) {
  using I = Idx<N, D>;
  sl[0] = v[I::E];
  T* Vs = reinterpret_cast<T*>(sl + 1);
#pragma unroll
  for (int k = 0; k < I::NV; k++) Vs[k] = cvt<T>(v[k]);
  if constexpr (Ring<N, D, T>::HILO) {
#pragma unroll
    for (int q = 0; q <= D; q++) Vs[I::NV + q] = cvt<T>(v[N + q] - wide(Vs[N + q]));
  }
}

// The primitive slots of cells c0 .. c1 - 1 of U (Eq. 27 and put_slot, the
// same steps the sweeps take): word k of cell c to Vs[k ncell + c], through
// the thread's part of shared memory.  One pass a Runge-Kutta stage with
// every lane converting, where each direction sweep converted its cells and
// with four lanes of a warp the two stencil cells beyond each end of a
// window.  RATE: the pass over a step's first stage input also reduces the
// CFL rate max_cells sum_d (|u_d| + c)/dx_d into *rate_bits (the caller
// clears it) from the primitive state it has just formed, with the steps and
// the status bits of k_max_rate (a cell with rho <= 0 is inadmissible and
// left out of the rate, a non-finite rate is reported): the same rate bit
// for bit, the maximum being independent of the order.
template <int N, int D, typename T, bool RATE = false>
__global__ void __launch_bounds__(256) k_prim_slots(const double* __restrict__ U,
                                                    double* __restrict__ Vs, long ncell, long c0,
                                                    long c1, Mat m, double idx0 = 0.0,
                                                    double idx1 = 0.0, double idx2 = 0.0,
                                                    unsigned long long* rate_bits = nullptr,
                                                    unsigned* status = nullptr) {
  using I = Idx<N, D>;
  constexpr int SLOTD = Ring<N, D, T>::SLOTD;
  extern __shared__ double psl[];
  double* sl = psl + threadIdx.x * SLOTD;
  double best = 0.0;
  unsigned bad = 0u;
  for (long c = c0 + (long)blockIdx.x * blockDim.x + threadIdx.x; c < c1;
       c += (long)gridDim.x * blockDim.x) {
    double u[I::NV], v[I::NV];
#pragma unroll
    for (int k = 0; k < I::NV; k++) u[k] = __ldg(U + (long)k * ncell + c);
    cons_to_prim<N, D>(m, u, v);
    put_slot<N, D, T>(sl, v);
#pragma unroll
    for (int k = 0; k < SLOTD; k++) Vs[(long)k * ncell + c] = sl[k];
    if constexpr (RATE) {
      double rho = u[0];
#pragma unroll
      for (int p = 1; p < N; p++) rho += u[p];
      if (!(rho > 0.0)) {
        bad |= ST_INADMISSIBLE;
        continue;
      }
      const double cs = sound_speed<N, D, double>(m, u, rho, v[I::E]);
      double r = (fabs(v[I::U(0)]) + cs) * idx0;
      if (D > 1) r += (fabs(v[I::U(1)]) + cs) * idx1;
      if (D > 2) r += (fabs(v[I::U(D > 2 ? 2 : 0)]) + cs) * idx2;
      if (!(r <= 1.7e308)) bad |= ST_NAN;
      else best = fmax(best, r);
    }
  }
  if constexpr (RATE) {
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ double wmax[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wmax[wid] = best;
    __syncthreads();
    if (wid == 0) {
      best = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
      if (lane == 0) atomicMax(rate_bits, (unsigned long long)__double_as_longlong(best));
    }
    if (bad) atomicOr(status, bad);
  }
}

// A slot copied from the primitive slots of cell `cell` (a cell of the
// grid, not a mirrored boundary image: the sweep converts those itself).
template <int N, int D, typename T>
__device__ __forceinline__ void copy_slot(const SweepArgs& a, long cell, double* sl) {
  constexpr int SLOTD = Ring<N, D, T>::SLOTD;
#pragma unroll
  for (int k = 0; k < SLOTD; k++) sl[k] = __ldg(a.Vs + (long)k * a.ncell + cell);
}

// face_velocity_pressure with the loop over the variables not unrolled (one
// copy of the code for all of them) and the faces written to out[k * 32]:
// u_0 L, u_0 R, ..., P L, P R (a lane's column of the window scratch).
template <int N, int D, typename T, int LW>
__device__ __forceinline__ void face_velocity_pressure_rolled(const Mat& m, const T* const* V,
                                                              double Pb, double* out) {
  using I = Idx<N, D>;
#pragma unroll 1
  for (int v = N; v <= N + D; v++) {
    double fl, fr;
    if constexpr (Ring<N, D, T>::HILO) {
      const int q = v - N;
      const T c = V[2][v], cl = V[2][I::NV + q];
      auto dlt = [&](int k) { return (V[k][v] - c) + (V[k][I::NV + q] - cl); };
      const Stencil<T> st{c, dlt(0), dlt(1), dlt(3), dlt(4)};
      const W6<T> w = sweep_weights<LW, T>(m, st);
      T oL, oR;
      offsets(w, st, oL, oR);
      const T res = fabs(c) * T(0x1p-24);
      if (fabs(oL) < res) oL = T(0);
      if (fabs(oR) < res) oR = T(0);
      const double cv = v < N + D ? wide(c) + wide(cl) : Pb;
      fl = cv + wide(oL);
      fr = cv + wide(oR);
    } else {
      const Stencil<T> st = stencil<T>(V[0][v], V[1][v], V[2][v], V[3][v], V[4][v]);
      const W6<T> w = sweep_weights<LW, T>(m, st);
      T tl, tr;
      reconstruct(w, st, tl, tr);
      fl = wide(tl);
      fr = wide(tr);
    }
    out[2 * (v - N) * 32] = fl;
    out[(2 * (v - N) + 1) * 32] = fr;
  }
}

// Faces of the velocity components and the pressure, each with its own
// weights (V[k] = the slots of the stencil's five cells, Pb the cell's FP64
// pressure).  FP64: value form.  Reduced precision: the stencil of the
// differences to the cell value, formed from the hi/lo pairs, reconstructed
// in T as offsets that are added to the FP64 cell value; an offset below
// the T resolution of the cell value (|value| 2^-24) is dropped.  So a
// uniform stencil, or one that varies only below what T can resolve, gives
// faces equal to the cell value, and the FP64 noise of a uniform field
// stays a cell's own instead of being quantised to T steps.
template <int N, int D, typename T, int LW>
__device__ __forceinline__ void face_velocity_pressure(const Mat& m, const T* const* V, double Pb,
                                                       double* uL, double* uR, double& PL,
                                                       double& PR) {
  using I = Idx<N, D>;
#pragma unroll
  for (int v = N; v <= N + D; v++) {
    double fl, fr;
    if constexpr (Ring<N, D, T>::HILO) {
      const int q = v - N;
      const T c = V[2][v], cl = V[2][I::NV + q];
      auto dlt = [&](int k) { return (V[k][v] - c) + (V[k][I::NV + q] - cl); };
      const Stencil<T> st{c, dlt(0), dlt(1), dlt(3), dlt(4)};
      const W6<T> w = sweep_weights<LW, T>(m, st);
      T oL, oR;
      offsets(w, st, oL, oR);
      const T res = fabs(c) * T(0x1p-24);
      if (fabs(oL) < res) oL = T(0);
      if (fabs(oR) < res) oR = T(0);
      const double cv = v < N + D ? wide(c) + wide(cl) : Pb;
      fl = cv + wide(oL);
      fr = cv + wide(oR);
    } else {
      const Stencil<T> st = stencil<T>(V[0][v], V[1][v], V[2][v], V[3][v], V[4][v]);
      const W6<T> w = sweep_weights<LW, T>(m, st);
      T tl, tr;
      reconstruct(w, st, tl, tr);
      fl = wide(tl);
      fr = wide(tr);
    }
    if (v < N + D) {
      uL[v - N] = fl;
      uR[v - N] = fr;
    } else {
      PL = fl;
      PR = fr;
    }
  }
}

// March through cells [s, e) of one pencil (first cell at index `base`,
// step `a.stride`, `a.n` cells, boundary conditions a.bclo/a.bchi):
// reconstruct, limit, solve the Riemann problems and update per a.mode.
// `ring` is this thread's five-slot stencil ring in shared memory.  Variant
// LW: 0 the scheme (WENO-C / WENO-CL), 1 with learned mass weights, 2 the
// comparison schemes (own weights per variable, no limiters, no stage bound).
template <int N, int D, typename T, typename TF, int LW = 0>
__device__ __forceinline__ void sweep_segment(const SweepArgs& a, const Mat& m, long base, int s,
                                              int e, double* ring, double dt, unsigned& bad,
                                              unsigned* lstat = nullptr) {
  using I = Idx<N, D>;
  constexpr int NV = I::NV;
  constexpr int SLOTD = Ring<N, D, T>::SLOTD;
  // conservative values of cell c (boundary cells mapped, normal momentum
  // negated behind reflective walls)
  auto load_cons = [&](int c, double* u) {
    bool flip;
    int j = bc_index(c, a.n, a.bclo, a.bchi, flip);
    long cell = base + (long)j * a.stride;
#pragma unroll
    for (int k = 0; k < NV; k++) u[k] = __ldg(a.U + (long)k * a.ncell + cell);
    // sign flip of the normal momentum on the bit pattern (no FP64 op, no
    // runtime-indexed register array)
#pragma unroll
    for (int jj = 0; jj < D; jj++) {
      long long mask = (flip && jj == a.dir) ? (long long)0x8000000000000000ULL : 0LL;
      u[I::U(jj)] = __longlong_as_double(__double_as_longlong(u[I::U(jj)]) ^ mask);
    }
  };
  auto load = [&](int c) {
    double u[NV], v[NV];
    load_cons(c, u);
    cons_to_prim<N, D>(m, u, v);
    put_slot<N, D, T>(ring + ((c + 15) % 5) * SLOTD, v);
  };

  for (int c = s - 3; c <= s; c++) load(c);

  Face<N, D> prevL;
  double Fprev[NV], Uprev[NV], sfprev[N];
  double uprev = 0.0;
  double Qprev[N], Qcur[N];
  auto load_q = [&](int c, double* q) {
    bool flip;
    int j = bc_index(c, a.n, a.bclo, a.bchi, flip);
    long cell = base + (long)j * a.stride;
#pragma unroll
    for (int p = 0; p < N; p++) q[p] = __ldg(a.Q + (long)p * a.ncell + cell);
  };
  if (a.kind == 1) load_q(s - 1, Qprev);
  for (int c = s - 1; c <= e; c++) {
    load(c + 2);
    const T* V[5];
#pragma unroll
    for (int k = 0; k < 5; k++)
      V[k] = reinterpret_cast<const T*>(ring + ((c - 2 + k + 15) % 5) * SLOTD + 1);
    const double Pb = ring[((c + 15) % 5) * SLOTD];
    double Ub[NV];
    load_cons(c, Ub);
    // reduced precision: mass and fraction faces = FP64 cell value (a
    // conservative and primitive variable alike) + offset in T
    constexpr bool OFFSET = !std::is_same<T, double>::value;

    // Eq. 16: masses and fractions with the weights of the masses
    double mL[N], mR[N], aL[N], aR[N];
#pragma unroll
    for (int p = 0; p < N; p++) {
      Stencil<T> st = stencil<T>(V[0][p], V[1][p], V[2][p], V[3][p], V[4][p]);
      W6<T> w = sweep_weights<LW, T>(m, st);
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
          const int ia = I::A(p);
          const Stencil<T> sa = stencil<T>(V[0][ia], V[1][ia], V[2][ia], V[3][ia], V[4][ia]);
          bool okL = true, okR = true, flat = true;
          auto judge = [&](const Stencil<T>& q) {
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
          // counted: face sides of stencils that are not flat (on a flat
          // stencil every convex weight gives the cell value)
          if (!flat) {
            lstat[0] += 2u;
            lstat[1] += unsigned(!okL) + unsigned(!okR);
          }
        }
      }
      const int ia = I::A(p);
      const Stencil<T> sa = stencil<T>(V[0][ia], V[1][ia], V[2][ia], V[3][ia], V[4][ia]);
      // (the comparison schemes: the fraction with its own weights)
      W6<T> wa = w;
      if constexpr (LW == 2) wa = sweep_weights<LW, T>(m, sa);
      if constexpr (OFFSET) {
        reconstruct_offset(w, st, Ub[p], mL[p], mR[p]);
        reconstruct_offset(wa, sa, Ub[ia], aL[p], aR[p]);
      } else {
        T fl, fr;
        reconstruct(w, st, fl, fr);
        mL[p] = wide(fl);
        mR[p] = wide(fr);
        reconstruct(wa, sa, fl, fr);
        aL[p] = wide(fl);
        aR[p] = wide(fr);
      }
    }
    // velocity and pressure, each with its own weights
    double uL[D], uR[D], PL, PR;
    face_velocity_pressure<N, D, T, LW>(m, V, Pb, uL, uR, PL, PR);
    Face<N, D> fL, fR;
    limit_chain<N, D, LW != 2>(m, Ub, Pb, mL, aL, mR, aR, uL, PL, uR, PR, a.energy_limiter, fL, fR,
                      nullptr);
    if (a.kind == 1) load_q(c, Qcur);
    if (c >= s) {
      double F[NV], uh = 0.0;
      if (a.kind == 1) {
        double G[N];
#pragma unroll
        for (int p = 0; p < N; p++)
          G[p] = pf_gradient(Qprev[p], Qcur[p], Uprev[I::A(p)], Ub[I::A(p)], a.inv_dx,
                             a.gcoef > 0.0 ? a.gcoef / dt : a.gmax);
        pf_flux<N, D>(m, prevL, fR, G, F);
      } else {
        riemann<N, D, TF>(m, a.dir, a.hllc, prevL, fR, F, uh);
      }
      if (c > s) {
        // update cell c-1 (interior, no boundary mapping)
        long cell = base + (long)(c - 1) * a.stride;
        const double du = (uh - uprev) * a.inv_dx;
#pragma unroll
        for (int v = 0; v < NV; v++) {
          // Eq. 3: -div F + alpha (1 + K) div u_hat;  Eq. 5: +div F^PF
          double val = (a.kind == 1 ? 1.0 : -1.0) * (F[v] - Fprev[v]) * a.inv_dx;
          if (a.kind == 0 && v >= N + D + 1) val = fma(sfprev[v - (N + D + 1)], du, val);
          long idx = (long)v * a.ncell + cell;
          if (not_finite(val)) bad |= ST_NAN;
          if (a.mode == 0) {
            a.L[idx] = val;
          } else if (a.mode == 1) {
            a.L[idx] += val;
          } else {
            double Lt = a.mode == 2 ? a.L[idx] + val : val;
            // masses >= 0 and fractions in [0, 1] up to the rounding of the
            // stage sum (not in the comparison schemes, which have no bounds)
            a.Uout[idx] = rk_combine(a.rk0, a.U0[idx], a.rk1, Uprev[v], a.rk2 * dt, Lt,
                                     LW != 2 && (v < N || v >= I::A(0)), v >= I::A(0));
          }
        }
      }
#pragma unroll
      for (int v = 0; v < NV; v++) Fprev[v] = F[v];
      uprev = uh;
    }
    prevL = fL;
#pragma unroll
    for (int v = 0; v < NV; v++) Uprev[v] = Ub[v];
    // source factors alpha_p (1 + K_p) of this cell, used when it is updated
    source_factors<N, D>(m, Ub, Pb, sfprev);
    if (a.kind == 1) {
#pragma unroll
      for (int p = 0; p < N; p++) Qprev[p] = Qcur[p];
    }
  }
}

template <int N, int D, typename T, typename TF, int LW = 0>
__global__ void __launch_bounds__(128) k_sweep(SweepArgs a, Mat m) {
  constexpr int SLOTD = Ring<N, D, T>::SLOTD;
  extern __shared__ double smem[];
  double* ring = smem + (long)threadIdx.x * 5 * SLOTD;
  const long nthreads = (long)gridDim.x * blockDim.x;
  const long nitems = a.npencil * a.nseg;
  unsigned bad = 0u;
  unsigned lstat[2] = {0u, 0u};
  double dt = 0.0;
  // the stage modes, and every direction of a Phase-Field stage (its gradient
  // limit is gcoef / dt)
  if (a.mode >= 2 || a.gcoef > 0.0) dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.cfl / *a.rate;

  // work item = (pencil, segment); consecutive threads take consecutive
  // pencils of one segment row, so y and z sweeps read coalesced
  for (long item = (long)blockIdx.x * blockDim.x + threadIdx.x; item < nitems;
       item += nthreads) {
    const long tr = item % a.npencil;
    const int sg = (int)(item / a.npencil);
    long base;
    if (a.dir == 0) base = tr * a.nx;
    else if (a.dir == 1) base = (tr / a.nx) * ((long)a.nx * a.ny) + tr % a.nx;
    else base = tr;
    const int s = sg * a.seg;
    const int e = min(s + a.seg, a.n);
    sweep_segment<N, D, T, TF, LW>(a, m, base, s, e, ring, dt, bad, lstat);
  }
  if (bad) atomicOr(a.status, bad);
  if constexpr (LW == 1) {
    if (a.lcount) {
#pragma unroll
      for (int k = 0; k < 2; k++) {
        unsigned v = lstat[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.lcount + k, (unsigned long long)v);
      }
    }
  }
}

}  // namespace wc
