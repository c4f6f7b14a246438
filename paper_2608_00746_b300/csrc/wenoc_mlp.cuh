// wenoc_mlp.cuh -- the learned WENO-weight surrogate: a 32 -> 64 -> 64 -> 64
// -> 16 ReLU network (30 used inputs, 9 used outputs = three softmax weights
// per phase for N <= 3) evaluated and trained on the fifth-generation tensor
// cores: BF16 weights and activations, FP32 accumulation in tensor memory.
//
// Parameter block (one contiguous buffer): BF16 weights W1[64][32],
// W2[64][64], W3[64][64], W4[16][64] (row = output), then FP32 biases
// b1[64], b2[64], b3[64], b4[16].  FP32 master copies, gradients and Adam
// moments use one FP32 array of MLP_NPARAM entries in the same order.
#pragma once
#include "wenoc_sweep.cuh"
#include "wenoc_umma.cuh"

namespace wc {

constexpr int MLP_IN = 32, MLP_H = 64, MLP_OUT = 16, MLP_NW = 9, MLP_MAXP = 3;
constexpr int MLP_W1 = 0, MLP_W2 = MLP_W1 + MLP_H * MLP_IN, MLP_W3 = MLP_W2 + MLP_H * MLP_H,
              MLP_W4 = MLP_W3 + MLP_H * MLP_H, MLP_NWEIGHT = MLP_W4 + MLP_OUT * MLP_H;
constexpr int MLP_B1 = 0, MLP_B2 = 64, MLP_B3 = 128, MLP_B4 = 192, MLP_NBIAS = 208;
constexpr int MLP_NPARAM = MLP_NWEIGHT + MLP_NBIAS;
constexpr size_t MLP_PARAM_BYTES = (size_t)MLP_NWEIGHT * 2 + (size_t)MLP_NBIAS * 4;

// Features of one face side (reading of the learned-weight workload): for
// each phase p the five masses of the stencil, ordered towards the face,
// minus the cell's own mass and divided by the largest such difference (0
// for a flat stencil: largest difference at most 1e-300), then the five
// fractions as they are.  Weights of
// Eq. 15 are invariant under f -> a f + b, so the scaled masses lose nothing.
template <int N>
__device__ __forceinline__ void mlp_features(const double (*m)[5], const double (*al)[5],
                                             __nv_bfloat16* x) {
#pragma unroll
  for (int p = 0; p < N; p++) {
    double c = m[p][2], mx = 0.0;
#pragma unroll
    for (int k = 0; k < 5; k++) mx = fmax(mx, fabs(m[p][k] - c));
    // deviations below 1e-300 count as flat (no overflow of 1 / mx)
    double r = mx > 1e-300 ? 1.0 / mx : 0.0;
#pragma unroll
    for (int k = 0; k < 5; k++) {
      x[p * 10 + k] = __float2bfloat16((float)((m[p][k] - c) * r));
      x[p * 10 + 5 + k] = __float2bfloat16((float)al[p][k]);
    }
  }
#pragma unroll
  for (int k = N * 10; k < MLP_IN; k++) x[k] = __float2bfloat16(0.0f);
}

// Geometry of the rows of a direction's weight inference: row = 2 cell +
// side, side 0 = the face x_{i+1/2}, side 1 = x_{i-1/2} (mirrored stencil).
struct MlpGeom {
  const double* U;  // state [NV][ncell]
  long ncell;
  int nx, ny, nz, dir, n;
  long stride;
  int bclo, bchi;
  int N;            // phases (masses at 0..N-1, fractions at NV-N..NV-1)
  int nv;
};

cudaError_t launch_mlp_forward(const __nv_bfloat16* X, long nrows, const void* params, float* Y,
                               unsigned* status, cudaStream_t st);
cudaError_t launch_mlp_infer(const MlpGeom& g, const void* params, float* Wsoa,
                             unsigned* status, cudaStream_t st);
cudaError_t launch_mlp_features(const MlpGeom& g, long row0, __nv_bfloat16* X, float* T,
                                long* list, unsigned long long* count, long cap,
                                cudaStream_t st);
cudaError_t launch_mlp_train(const __nv_bfloat16* X, const float* T, const int* idx, int batch,
                             const void* params, float* grads, float* loss, unsigned* status,
                             cudaStream_t st);
cudaError_t launch_mlp_adam(float* master, void* params, float* grads, float* m, float* v,
                            float lr, float beta1, float beta2, float eps, int step,
                            cudaStream_t st);

}  // namespace wc
