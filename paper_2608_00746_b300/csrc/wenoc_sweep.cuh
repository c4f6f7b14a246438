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
  double inv_dx;
  int bclo, bchi;
  int mode;            // 0: L = dir part; 1: L += dir part; 2: stage with L + dir part; 3: stage with dir part only
  int hllc;
  int energy_limiter;
  unsigned* status;
};

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

// Ring slot layout in shared memory (per thread, 5 slots):
//   V[NV] of type T (primitive, for the reconstruction), U[NV] FP64
//   (conservative, for the limiter and the update), P FP64.
template <int N, int D, typename T>
struct Ring {
  static constexpr int NV = Idx<N, D>::NV;
  static constexpr int SLOT_BYTES = NV * (int)sizeof(T) + NV * 8 + 8;
  static constexpr int BYTES = 5 * ((SLOT_BYTES + 7) / 8) * 8;
};

template <int N, int D, typename T, typename TF>
__global__ void __launch_bounds__(128) k_sweep(SweepArgs a, Mat m) {
  using I = Idx<N, D>;
  constexpr int NV = I::NV;
  constexpr int SLOTD = (Ring<N, D, T>::SLOT_BYTES + 7) / 8;  // doubles per slot
  extern __shared__ double smem[];
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= a.npencil * a.nseg) return;
  long tr = tid % a.npencil;
  int sg = (int)(tid / a.npencil);
  // first cell of the pencil
  long base;
  if (a.dir == 0) base = tr * a.nx;
  else if (a.dir == 1) base = (tr / a.nx) * ((long)a.nx * a.ny) + tr % a.nx;
  else base = tr;
  int s = sg * a.seg;
  int e = min(s + a.seg, a.n);
  double* ring = smem + (long)threadIdx.x * 5 * SLOTD;

  auto load = [&](int c) {
    bool flip;
    int j = bc_index(c, a.n, a.bclo, a.bchi, flip);
    long cell = base + (long)j * a.stride;
    double* sl = ring + ((c + 15) % 5) * SLOTD;
    double* Us = sl;                       // NV doubles
    double* Ps = sl + NV;                  // 1 double
    T* Vs = reinterpret_cast<T*>(sl + NV + 1);
    double u[NV], v[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) u[k] = __ldg(a.U + (long)k * a.ncell + cell);
    if (flip) {
#pragma unroll
      for (int j = 0; j < D; j++)
        if (j == a.dir) u[I::U(j)] = -u[I::U(j)];
    }
    cons_to_prim<N, D>(m, u, v);
#pragma unroll
    for (int k = 0; k < NV; k++) {
      Us[k] = u[k];
      Vs[k] = T(v[k]);
    }
    *Ps = v[I::E];
  };

  for (int c = s - 3; c <= s; c++) load(c);

  Face<N, D> prevL;
  double Fprev[NV];
  double uprev = 0.0;
  double dt = 0.0;
  if (a.mode >= 2) dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.cfl / *a.rate;
  unsigned bad = 0u;

  for (int c = s - 1; c <= e; c++) {
    load(c + 2);
    const double* slot[5];
#pragma unroll
    for (int k = 0; k < 5; k++) slot[k] = ring + ((c - 2 + k + 15) % 5) * SLOTD;
    const T* V0 = reinterpret_cast<const T*>(slot[0] + NV + 1);
    const T* V1 = reinterpret_cast<const T*>(slot[1] + NV + 1);
    const T* V2 = reinterpret_cast<const T*>(slot[2] + NV + 1);
    const T* V3 = reinterpret_cast<const T*>(slot[3] + NV + 1);
    const T* V4 = reinterpret_cast<const T*>(slot[4] + NV + 1);
    const double* Ub = slot[2];
    double Pb = slot[2][NV];

    // Eq. 16: masses and fractions with the weights of the masses
    double mL[N], mR[N], aL[N], aR[N];
#pragma unroll
    for (int p = 0; p < N; p++) {
      Stencil<T> st = stencil<T>(V0[p], V1[p], V2[p], V3[p], V4[p]);
      W6<T> w = weights_of<T>(st);
      T fl, fr;
      reconstruct(w, st, fl, fr);
      mL[p] = double(fl);
      mR[p] = double(fr);
      const int ia = I::A(p);
      st = stencil<T>(V0[ia], V1[ia], V2[ia], V3[ia], V4[ia]);
      reconstruct(w, st, fl, fr);
      aL[p] = double(fl);
      aR[p] = double(fr);
    }
    // velocity and pressure, each with its own weights
    double uL[D], uR[D], PL, PR;
#pragma unroll
    for (int v = N; v <= N + D; v++) {
      Stencil<T> st = stencil<T>(V0[v], V1[v], V2[v], V3[v], V4[v]);
      W6<T> w = weights_of<T>(st);
      T fl, fr;
      reconstruct(w, st, fl, fr);
      if (v < N + D) {
        uL[v - N] = double(fl);
        uR[v - N] = double(fr);
      } else {
        PL = double(fl);
        PR = double(fr);
      }
    }
    Face<N, D> fL, fR;
    limit_chain<N, D>(m, Ub, Pb, mL, aL, mR, aR, uL, PL, uR, PR, a.energy_limiter, fL, fR,
                      nullptr);
    if (c >= s) {
      double F[NV], uh;
      riemann<N, D, TF>(m, a.dir, a.hllc, prevL, fR, F, uh);
      if (c > s) {
        // update cell c-1 (interior index, no boundary mapping)
        long cell = base + (long)(c - 1) * a.stride;
        const double* Uc = slot[1];   // cell c-1
#pragma unroll
        for (int v = 0; v < NV; v++) {
          double val = -(F[v] - Fprev[v]) * a.inv_dx;
          if (v >= N + D + 1) val = fma(Uc[v], (uh - uprev) * a.inv_dx, val);
          long idx = (long)v * a.ncell + cell;
          if (!(fabs(val) <= 1.7e308)) bad |= ST_NAN;
          if (a.mode == 0) {
            a.L[idx] = val;
          } else if (a.mode == 1) {
            a.L[idx] += val;
          } else {
            double Lt = a.mode == 2 ? a.L[idx] + val : val;
            double u0 = a.U0[idx];
            a.Uout[idx] = a.rk0 * u0 + a.rk1 * Uc[v] + a.rk2 * dt * Lt;
          }
        }
      }
#pragma unroll
      for (int v = 0; v < NV; v++) Fprev[v] = F[v];
      uprev = uh;
    }
    prevL = fL;
  }
  if (bad) atomicOr(a.status, bad);
}

}  // namespace wc
