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

// Roundings of FP64 values on the integer pipe (the FP64 pipe is slow on
// this part): to FP32 and to BF16, to nearest with ties to even; magnitudes
// below 2^-126 become zero.
// x * 2^k (k >= -1023) rounded to FP32; subnormal x counts as zero
__device__ __forceinline__ float f64_to_f32_flush(double x, int k = 0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const int ef = e == 0 ? 0 : e - 1023 + 127 + k;
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  if (ef <= 0) return __uint_as_float(sign);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned int q = (unsigned int)(m >> 29);
  const unsigned long long rem = m & ((1ull << 29) - 1), half = 1ull << 28;
  unsigned int r = ((unsigned int)(ef < 255 ? ef : 255) << 23) | (ef < 255 ? q : 0u);
  if (ef < 255 && (rem > half || (rem == half && (q & 1u)))) r += 1u;
  return __uint_as_float(r | sign);
}
__device__ __forceinline__ __nv_bfloat16 f64_to_bf16_flush(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  const unsigned short sign = (unsigned short)((b >> 48) & 0x8000u);
  if (ef <= 0) return __ushort_as_bfloat16(sign);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned int q = (unsigned int)(m >> 45);
  const unsigned long long rem = m & ((1ull << 45) - 1), half = 1ull << 44;
  unsigned int r = ((unsigned int)(ef < 255 ? ef : 255) << 7) | (ef < 255 ? q : 0u);
  if (ef < 255 && (rem > half || (rem == half && (q & 1u)))) r += 1u;
  return __ushort_as_bfloat16((unsigned short)(r | sign));
}

// Features of both face sides of one cell (reading of the learned-weight
// workload): for each phase p the five masses of the stencil, ordered
// towards the face, minus the cell's own mass (FP64 differences d_k), scaled
// by the power of two 2^s that brings max |d_k| into [1, 2) and rounded to
// FP32 (values below 2^-126 and subnormal d_k to zero), divided in FP32 by
// their largest magnitude; a stencil with max |d_k| below 2^-1022 is flat
// (all zero).  Then the five fractions rounded once from FP64 to BF16 (below
// 2^-126 to zero).  Everything ends as BF16.  Side 0 (x_{i+1/2}) takes the
// stencil f_{i-2..i+2}, side 1 (x_{i-1/2}) its mirror image.  Eq. 15 is
// invariant under f -> a f + b, so the scaled masses lose nothing; only the
// differences use the FP64 pipe.
template <int N>
__device__ __forceinline__ void mlp_features2(const double (*m)[5], const double (*al)[5],
                                              __nv_bfloat16* x0, __nv_bfloat16* x1) {
#pragma unroll
  for (int p = 0; p < N; p++) {
    double dd[5];
    long long mxb = 0;
#pragma unroll
    for (int k = 0; k < 5; k++) {
      dd[k] = k == 2 ? 0.0 : m[p][k] - m[p][2];
      const long long ab = __double_as_longlong(dd[k]) & 0x7FFFFFFFFFFFFFFFLL;
      mxb = ab > mxb ? ab : mxb;
    }
    const int E = (int)(mxb >> 52);  // biased exponent of max |d_k|
    float d[5], mx = 0.0f;
#pragma unroll
    for (int k = 0; k < 5; k++) {
      d[k] = E == 0 ? 0.0f : f64_to_f32_flush(dd[k], 1023 - E);
      mx = fmaxf(mx, fabsf(d[k]));
    }
    const float r = mx > 0.0f ? 1.0f / mx : 0.0f;
#pragma unroll
    for (int k = 0; k < 5; k++) {
      const __nv_bfloat16 xm = __float2bfloat16(d[k] * r);
      const __nv_bfloat16 xa = f64_to_bf16_flush(al[p][k]);
      if (x0) {
        x0[p * 10 + k] = xm;
        x0[p * 10 + 5 + k] = xa;
      }
      if (x1) {
        x1[p * 10 + 4 - k] = xm;
        x1[p * 10 + 9 - k] = xa;
      }
    }
  }
#pragma unroll
  for (int k = N * 10; k < MLP_IN; k++) {
    if (x0) x0[k] = __float2bfloat16(0.0f);
    if (x1) x1[k] = __float2bfloat16(0.0f);
  }
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
