// wenoc_patches.cuh -- batched AMR-like patches: many independent uniform
// cube patches (each its own resolution, outflow boundary cells produced by
// index mapping, i.e. zero-gradient ghost layers of depth 3) advanced by one
// persistent launch per Runge-Kutta stage.
//
// A CTA takes one whole patch at a time -- from an atomic queue ordered by
// decreasing patch size (largest first), or statically round-robin -- and
// runs the x, y and z sweeps of the patch back to back (the y and z sweeps
// accumulate into the stage accumulator; the z sweep also applies the
// Shu-Osher combination).  Each thread owns whole pencils of the patch, so
// there is no redundant reconstruction inside a patch.
#pragma once
#include "wenoc_sweep.cuh"

namespace wc {

struct PatchArgs {
  const double* U;     // pooled state of all patches [NV][ncell]
  double* L;           // pooled accumulator
  const double* U0;    // pooled U^n
  double* Uout;        // pooled stage output
  const double* rate;  // device max rate (dt = cfl / rate)
  double cfl, dt_fixed;
  double rk0, rk1, rk2;
  long ncell;          // total cells of all patches
  const int* edge;     // patch edge e (cells per axis)
  const long* off;     // first cell of the patch in the pool
  const int* order;    // processing order (largest first)
  int npatch;
  int* counter;        // queue head of this launch (dynamic schedule)
  int dynamic;         // 1: atomic queue; 0: static round-robin
  int rhs_only;        // 1: write dU/dt into L (no Runge-Kutta combination)
  int hllc;
  int energy_limiter;
  unsigned* status;
};

template <int N, typename T, typename TF>
__global__ void __launch_bounds__(128) k_patch_stage(PatchArgs pa, Mat m) {
  constexpr int D = 3;
  constexpr int SLOTD = Ring<N, D, T>::SLOTD;
  extern __shared__ double smem[];
  __shared__ int s_item;
  double* ring = smem + (long)threadIdx.x * 5 * SLOTD;
  unsigned bad = 0u;
  double dt = 0.0;
  if (!pa.rhs_only) dt = pa.dt_fixed > 0.0 ? pa.dt_fixed : pa.cfl / *pa.rate;
  for (int k = 0;; k++) {
    int it;
    if (pa.dynamic) {
      if (threadIdx.x == 0) s_item = atomicAdd(pa.counter, 1);
      __syncthreads();
      it = s_item;
      __syncthreads();
    } else {
      it = blockIdx.x + k * gridDim.x;
    }
    if (it >= pa.npatch) break;
    const int p = pa.order[it];
    const int e = pa.edge[p];
    const long off = pa.off[p];
    for (int dir = 0; dir < D; dir++) {
      SweepArgs a;
      a.U = pa.U;
      a.L = pa.L;
      a.U0 = pa.U0;
      a.Uout = pa.Uout;
      a.rate = pa.rate;
      a.cfl = pa.cfl;
      a.dt_fixed = pa.dt_fixed;
      a.rk0 = pa.rk0;
      a.rk1 = pa.rk1;
      a.rk2 = pa.rk2;
      a.ncell = pa.ncell;
      a.nx = a.ny = a.nz = e;
      a.dir = dir;
      a.n = e;
      a.stride = dir == 0 ? 1 : (dir == 1 ? (long)e : (long)e * e);
      a.npencil = (long)e * e;
      a.nseg = 1;
      a.seg = e;
      a.max_threads = 0;
      a.Q = nullptr;
      a.kind = 0;
      a.inv_dx = (double)e;  // unit-cube patch: dx = 1/e
      a.bclo = a.bchi = BC_OUTFLOW;
      if (pa.rhs_only) a.mode = dir == 0 ? 0 : 1;
      else a.mode = dir == 0 ? 0 : (dir == 1 ? 1 : 2);
      a.hllc = pa.hllc;
      a.energy_limiter = pa.energy_limiter;
      a.status = pa.status;
      a.faceL = a.faceR = nullptr;
      a.fbuf = nullptr;
      a.poff = nullptr;
      a.tr0 = 0;
      for (int pc = threadIdx.x; pc < e * e; pc += blockDim.x) {
        long base;
        if (dir == 0) base = off + (long)pc * e;
        else if (dir == 1) base = off + (long)(pc / e) * e * e + pc % e;
        else base = off + pc;
        sweep_segment<N, D, T, TF>(a, m, base, 0, e, ring, dt, bad);
      }
      __syncthreads();  // this direction's accumulator complete for the patch
    }
  }
  if (bad) atomicOr(pa.status, bad);
}

// CFL rate over all patches, each with its own cell size (one CTA per patch).
template <int N>
__global__ void k_patch_rate(const double* __restrict__ U, long ncell, const int* edge,
                             const long* off, int npatch, Mat m, unsigned long long* rate_bits,
                             unsigned* status) {
  constexpr int D = 3;
  using I = Idx<N, D>;
  double best = 0.0;
  unsigned bad = 0u;
  for (int p = blockIdx.x; p < npatch; p += gridDim.x) {
    const int e = edge[p];
    const long o = off[p];
    const long nc = (long)e * e * e;
    const double idx = (double)e;
    for (long c = threadIdx.x; c < nc; c += blockDim.x) {
      double u[I::NV], v[I::NV];
#pragma unroll
      for (int k = 0; k < I::NV; k++) u[k] = __ldg(U + (long)k * ncell + o + c);
      double rho = u[0];
#pragma unroll
      for (int q = 1; q < N; q++) rho += u[q];
      if (!(rho > 0.0)) {
        bad |= ST_INADMISSIBLE;
        continue;
      }
      cons_to_prim<N, D>(m, u, v);
      double cs = sound_speed<N, D, double>(m, u, rho, v[I::E]);
      double r = (fabs(v[I::U(0)]) + fabs(v[I::U(1)]) + fabs(v[I::U(2)]) + 3.0 * cs) * idx;
      if (!(r <= 1.7e308)) bad |= ST_NAN;
      else best = fmax(best, r);
    }
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ double wmax[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wmax[wid] = best;
  __syncthreads();
  if (wid == 0) {
    best = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) atomicMax(rate_bits, (unsigned long long)__double_as_longlong(best));
  }
  if (bad) atomicOr(status, bad);
}

cudaError_t launch_patch_stage(int N, int mixed, const PatchArgs& pa, const Mat& m, int block,
                               int grid, cudaStream_t st);
cudaError_t launch_patch_rate(int N, const double* U, long ncell, const int* edge,
                              const long* off, int npatch, const Mat& m,
                              unsigned long long* rate_bits, unsigned* status, cudaStream_t st);

}  // namespace wc
