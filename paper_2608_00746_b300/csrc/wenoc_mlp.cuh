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
// this part), to nearest with ties to even.
// x rounded once to BF16 (8 significant bits, the exponent range of binary32
// including its subnormals, spacing 2^-133 below 2^-126); |x| < 2^128
__device__ __forceinline__ unsigned short f64_to_bf16_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 48) & 0x8000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const int ef = e - 1023 + 127;
  if (ef >= 1) {
    const unsigned int q = (unsigned int)(m >> 45);
    const unsigned long long rem = m & ((1ull << 45) - 1), half = 1ull << 44;
    unsigned int r = ((unsigned int)ef << 7) | q;
    if (rem > half || (rem == half && (q & 1u))) r += 1u;
    return (unsigned short)(r | sign);
  }
  // x = M 2^(e - 1075) with M = 2^52 + m: in units of 2^-133 that is
  // M / 2^(942 - e); below 2^-134 (and FP64 subnormals) it rounds to 0
  const int sh = 942 - e;  // >= 46 here
  if (e == 0 || sh >= 54) return (unsigned short)sign;
  const unsigned long long M = m | (1ull << 52);
  const unsigned int q = (unsigned int)(M >> sh);
  const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  unsigned int r = q;
  if (rem > half || (rem == half && (q & 1u))) r += 1u;
  return (unsigned short)(r | sign);
}

// x * 2^k (k >= -1023) rounded to FP32 on the integer pipe; results below
// 2^-126 (and subnormal x) become zero -- callers treat those as a slow case.
// (The hardware conversions cvt.rn.f32.f64 and cvt.rn.bf16.f64 give the same
// roundings but measured slower here: 0.84 against 0.78 ms an inference
// launch on the 2048^2 circles.)
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

// Features of both face sides of one cell (reading of the learned-weight
// workload): for each phase p the differences d_k = f_k - f_i (FP64) of the
// five masses of the stencil, ordered towards the face, to the cell's own,
// divided by the largest |d_k| (all zero for a flat stencil), then the five
// fractions, each value rounded once to BF16.  Side 0 (x_{i+1/2}) takes the
// stencil f_{i-2..i+2}, side 1 (x_{i-1/2}) its mirror image, whose features
// are the same values reversed.
//
// The quotients are formed in FP32 from the differences scaled by the power
// of two that brings max |d_k| into [1, 2): three roundings of 2^-24 and
// one of the product, so the FP32 quotient is within 4 of its units in the
// last place of d_k / max |d_k|.  Its BF16 rounding is then that of the FP64
// quotient except within 16 such units of a BF16 halfway point (and for
// quotients below 2^-126, where FP32 loses bits); those few values (about
// one in 2,000) are divided in FP64 and rounded from there, so every
// feature is the FP64 quotient rounded once to BF16.  Only the differences
// use the FP64 pipe otherwise.
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
      const unsigned int qb = __float_as_uint(d[k] * r);
      const unsigned int rem = qb & 0xFFFFu;
      // slow: near a halfway point, below 2^-126 in FP32 (flushed or
      // subnormal), or a subnormal largest difference
      const bool slow = (mxb != 0 && E == 0) ||
                        (dd[k] != 0.0 && (qb & 0x7F800000u) == 0u) ||
                        (rem >= 0x8000u - 16u && rem <= 0x8000u + 16u);
      unsigned short xb;
      if (!slow) {
        xb = (unsigned short)((qb + 0x7FFFu + ((qb >> 16) & 1u)) >> 16);
      } else {
        xb = f64_to_bf16_bits(dd[k] / __longlong_as_double(mxb));
      }
      const __nv_bfloat16 xm = __ushort_as_bfloat16(mxb == 0 ? (unsigned short)0 : xb);
      const __nv_bfloat16 xa = __ushort_as_bfloat16(f64_to_bf16_bits(al[p][k]));
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
