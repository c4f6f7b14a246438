// wenoc_kernels.cuh -- the small kernels around the sweep: the time-step
// reduction, the primitive/conservative maps, the isolated limiter chain and
// the FP64 peak probe.  Declarations of the per-precision sweep dispatchers.
#pragma once
#include "wenoc_sweep.cuh"

namespace wc {

// Largest sum_d (|u_d| + c)/dx_d over the cells (the CFL rate), reduced with
// atomicMax on the bit pattern of a non-negative double (order independent).
template <int N, int D>
__global__ void k_max_rate(const double* __restrict__ U, long ncell, Mat m, double idx0,
                           double idx1, double idx2, unsigned long long* rate_bits,
                           unsigned* status) {
  using I = Idx<N, D>;
  double best = 0.0;
  unsigned bad = 0u;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    double u[I::NV], v[I::NV];
#pragma unroll
    for (int k = 0; k < I::NV; k++) u[k] = __ldg(U + (long)k * ncell + c);
    double rho = u[0];
#pragma unroll
    for (int p = 1; p < N; p++) rho += u[p];
    if (!(rho > 0.0)) {
      bad |= ST_INADMISSIBLE;
      continue;
    }
    cons_to_prim<N, D>(m, u, v);
    double cs = sound_speed<N, D, double>(m, u, rho, v[I::E]);
    double r = (fabs(v[I::U(0)]) + cs) * idx0;
    if (D > 1) r += (fabs(v[I::U(1)]) + cs) * idx1;
    if (D > 2) r += (fabs(v[I::U(D > 2 ? 2 : 0)]) + cs) * idx2;
    if (!(r <= 1.7e308)) bad |= ST_NAN;
    else best = fmax(best, r);
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

static __global__ void k_dt_from_rate(const double* rate, double cfl, double* dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dt = cfl / *rate;
}

template <int N, int D>
__global__ void k_prim_to_cons(const double* __restrict__ V, double* __restrict__ U, long ncell,
                               Mat m) {
  using I = Idx<N, D>;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    double v[I::NV], u[I::NV];
#pragma unroll
    for (int k = 0; k < I::NV; k++) v[k] = V[(long)k * ncell + c];
    prim_to_cons<N, D>(m, v, u);
#pragma unroll
    for (int k = 0; k < I::NV; k++) U[(long)k * ncell + c] = u[k];
  }
}

template <int N, int D>
__global__ void k_cons_to_prim(const double* __restrict__ U, double* __restrict__ V, long ncell,
                               Mat m) {
  using I = Idx<N, D>;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    double v[I::NV], u[I::NV];
#pragma unroll
    for (int k = 0; k < I::NV; k++) u[k] = U[(long)k * ncell + c];
    cons_to_prim<N, D>(m, u, v);
#pragma unroll
    for (int k = 0; k < I::NV; k++) V[(long)k * ncell + c] = v[k];
  }
}

// Per-phase heat capacities C_p^T of the temperature law (Eq. 26).
struct HeatCap {
  double cT[MAXP];
};

// Mixture temperature of Eq. 29: (rho E - |rho u|^2 / (2 rho) - sum_p B_p^T
// alpha_p - sum_p D_p (alpha rho)_p) / sum_p C_p^T (alpha rho)_p with
// B_p^T = Pinf_p (Eq. 26).
template <int N, int D>
__global__ void k_temperature(const double* __restrict__ U, double* __restrict__ T, long ncell,
                              Mat m, HeatCap h) {
  using I = Idx<N, D>;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    double rho = 0.0, den = 0.0;
#pragma unroll
    for (int p = 0; p < N; p++) {
      const double mp = U[(long)p * ncell + c];
      rho += mp;
      den += h.cT[p] * mp;
    }
    double mom2 = 0.0;
#pragma unroll
    for (int j = 0; j < D; j++) {
      const double mj = U[(long)I::U(j) * ncell + c];
      mom2 += mj * mj;
    }
    double num = U[(long)I::E * ncell + c] - 0.5 * mom2 / rho;
#pragma unroll
    for (int p = 0; p < N; p++)
      num -= m.pinf[p] * U[(long)I::A(p) * ncell + c] + m.D[p] * U[(long)p * ncell + c];
    T[c] = num / den;
  }
}

// Membership of each cell average in the admissible set of Eq. 8: masses
// >= 0, fractions in [0, 1] summing to one within sum_tol, a positive
// density and psi >= 0 (Eq. 9 with the phasic minimum pressures), every
// value finite.  Counts the cells outside it (bad[0]) and the first such
// cell (atomicMin on bad[1]).
template <int N, int D>
__global__ void k_check_state(const double* __restrict__ U, long ncell, Mat m, double sum_tol,
                              unsigned long long* bad) {
  using I = Idx<N, D>;
  unsigned long long nbad = 0;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    double u[I::NV];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < I::NV; k++) {
      u[k] = __ldg(U + (long)k * ncell + c);
      ok = ok && !not_finite(u[k]);
    }
    double rho = 0.0, s = 0.0;
#pragma unroll
    for (int p = 0; p < N; p++) {
      ok = ok && u[p] >= 0.0 && u[I::A(p)] >= 0.0 && u[I::A(p)] <= 1.0;
      rho += u[p];
      s += u[I::A(p)];
    }
    ok = ok && rho > 0.0 && fabs(s - 1.0) <= sum_tol && psi_cons<N, D>(m, u) >= 0.0;
    if (!ok) {
      nbad++;
      atomicMin(bad + 1, (unsigned long long)c);
    }
  }
  for (int o = 16; o > 0; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
  if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, nbad);
}

// Eq. 17-21 on caller-given raw primitive faces of independent cells.
template <int N, int D>
__global__ void k_limit(const double* __restrict__ Ub, const double* __restrict__ VL,
                        const double* __restrict__ VR, double* __restrict__ UL,
                        double* __restrict__ UR, double* __restrict__ TH, long ncell, Mat m,
                        int energy_limiter) {
  using I = Idx<N, D>;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    double ub[I::NV], vb[I::NV];
#pragma unroll
    for (int k = 0; k < I::NV; k++) ub[k] = Ub[(long)k * ncell + c];
    cons_to_prim<N, D>(m, ub, vb);
    double mL[N], mR[N], aL[N], aR[N], uL[D], uR[D];
#pragma unroll
    for (int p = 0; p < N; p++) {
      mL[p] = VL[(long)p * ncell + c];
      mR[p] = VR[(long)p * ncell + c];
      aL[p] = VL[(long)I::A(p) * ncell + c];
      aR[p] = VR[(long)I::A(p) * ncell + c];
    }
#pragma unroll
    for (int j = 0; j < D; j++) {
      uL[j] = VL[(long)I::U(j) * ncell + c];
      uR[j] = VR[(long)I::U(j) * ncell + c];
    }
    double PL = VL[(long)I::E * ncell + c], PR = VR[(long)I::E * ncell + c];
    Face<N, D> fL, fR;
    double th[3];
    limit_chain<N, D>(m, ub, vb[I::E], mL, aL, mR, aR, uL, PL, uR, PR, energy_limiter, fL, fR,
                      th);
#pragma unroll
    for (int k = 0; k < I::NV; k++) {
      UL[(long)k * ncell + c] = fL.U[k];
      UR[(long)k * ncell + c] = fR.U[k];
    }
    if (TH)
      for (int t = 0; t < 3; t++) TH[(long)t * ncell + c] = th[t];
  }
}

// Per-precision sweep dispatch (defined in wenoc_fp64.cu / wenoc_mixed.cu /
// wenoc_learned.cu; the FP64 comparison schemes in wenoc_compare.cu).
cudaError_t launch_sweep_fp64(int N, int D, const SweepArgs& a, const Mat& m, int block,
                              cudaStream_t st);
cudaError_t launch_sweep_mixed(int N, int D, const SweepArgs& a, const Mat& m, int block,
                               cudaStream_t st);
cudaError_t launch_sweep_learned(int N, int D, const SweepArgs& a, const Mat& m, int block,
                                 cudaStream_t st);
cudaError_t launch_sweep_compare(int N, int D, const SweepArgs& a, const Mat& m, int block,
                                 cudaStream_t st);
int sweep_smem_bytes_fp64(int N, int D);
int sweep_smem_bytes_mixed(int N, int D);

}  // namespace wc
