// wenoc_mlp.cu -- tensor-core (tcgen05) inference, training (forward +
// backward) and Adam kernels of the learned WENO-weight surrogate, the
// feature / target extraction from a state, and their C ABI.
//
// Every network kernel is one CTA of 128 threads per 128-row tile: thread t
// owns row t of the tile, which is lane t of the tensor-memory accumulator.
// Operands live in shared memory in the no-swizzle core-matrix layout; one
// elected thread issues the MMAs and commits them to an mbarrier that every
// thread waits on (bounded: a timeout sets status bit 4 and the kernel
// returns after releasing its tensor memory).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../../include/wenoc.h"
#include "wenoc_kernels.cuh"
#include "wenoc_mlp.cuh"

namespace wc {

enum : unsigned { ST_TIMEOUT = 4u };
constexpr long kWaitPolls = 1L << 24;

struct MlpPtrs {
  const __nv_bfloat16* W;
  const float* b;
};
__device__ __forceinline__ MlpPtrs mlp_ptrs(const void* params) {
  MlpPtrs p;
  p.W = reinterpret_cast<const __nv_bfloat16*>(params);
  p.b = reinterpret_cast<const float*>(reinterpret_cast<const char*>(params) +
                                       (size_t)MLP_NWEIGHT * sizeof(__nv_bfloat16));
  return p;
}

// Row-major [R][K] BF16 matrix into the core-matrix layout (TRANS: its
// transpose, [K][R]).
template <int R, int K, bool TRANS>
__device__ __forceinline__ void stage_matrix(unsigned char* dst, const __nv_bfloat16* src) {
  for (int i = threadIdx.x; i < R * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    const uint32_t o = TRANS ? cm_offset(k, r, R) : cm_offset(r, k, K);
    *reinterpret_cast<__nv_bfloat16*>(dst + o) = src[i];
  }
}

// This thread's row of a [128][K] operand.
template <int K>
__device__ __forceinline__ void put_row(unsigned char* dst, int row, const float* v) {
#pragma unroll
  for (int k = 0; k < K; k += 8) {
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int j = 0; j < 8; j++) h[j] = __float2bfloat16(v[k + j]);
    *reinterpret_cast<uint4*>(dst + cm_offset(row, k, K)) = *reinterpret_cast<const uint4*>(h);
  }
}
// This thread's row as column `col` of a [R][128] operand.
template <int R>
__device__ __forceinline__ void put_col(unsigned char* dst, int col, const float* v) {
#pragma unroll
  for (int r = 0; r < R; r++)
    *reinterpret_cast<__nv_bfloat16*>(dst + cm_offset(r, col, 128)) = __float2bfloat16(v[r]);
}
template <int K>
__device__ __forceinline__ void get_row(const unsigned char* src, int row, float* v) {
#pragma unroll
  for (int k = 0; k < K; k++)
    v[k] = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(src + cm_offset(row, k, K)));
}

// relu(a) and relu(b) rounded to BF16 (nearest even) and packed, a in the
// low half.
__device__ __forceinline__ uint32_t bf16x2_relu(float a, float b) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
  return d;
}

// Hidden-layer epilogue of this thread's row: 64 accumulator columns from
// tensor memory, + bias, ReLU, BF16, into row `row` of a [128][64] operand.
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* bias,
                                                unsigned char* out, int row) {
#pragma unroll
  for (int c = 0; c < MLP_H; c += 32) {
    float h[32];
    tmem_ld32(taddr + c, h);
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
      // bias added two columns at a time (packed FP32, each sum rounded as
      // a scalar add would be)
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const float2 s = __fadd2_rn(make_float2(h[k + 2 * q], h[k + 2 * q + 1]),
                                    *reinterpret_cast<const float2*>(bias + c + k + 2 * q));
        w[q] = bf16x2_relu(s.x, s.y);
      }
      *reinterpret_cast<uint4*>(out + cm_offset(row, c + k, MLP_H)) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

struct MmaSync {
  uint64_t* bar;
  uint32_t phase;
  // every thread waits for the committed MMAs; false on timeout, uniform
  // over the CTA
  __device__ __forceinline__ bool wait() {
    bool ok = mbar_wait_bounded(bar, phase, kWaitPolls);
    phase ^= 1u;
    tc_fence_after();
    return __syncthreads_and(ok) != 0;
  }
  // after a timeout: wait (bounded) once more for the MMAs still in flight
  __device__ __forceinline__ void drain() { (void)mbar_wait_bounded(bar, phase ^ 1u, kWaitPolls); }
};

// Generic-proxy shared-memory writes made visible to the tensor core, and
// every thread's earlier tensor-memory reads ordered before the next MMA.
__device__ __forceinline__ void operands_ready() {
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void tile_setup(uint32_t* tbase, uint64_t* bar, uint32_t ncols) {
  if ((threadIdx.x >> 5) == 0) {
    tmem_alloc(tbase, ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

__device__ __forceinline__ void tile_teardown(uint32_t tm, uint32_t ncols) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tm, ncols);
}

// One hidden layer: out = relu(in W^T + b) for the 128 rows of the tile.
template <int K>
__device__ __forceinline__ bool fwd_layer(uint32_t a_in, uint32_t b_w, const float* bias,
                                          unsigned char* out, uint32_t tm, uint32_t lane_off,
                                          MmaSync& ms) {
  if (threadIdx.x == 0) {
    umma_tile(tm, a_in, b_w, MLP_H, K, 0);
    umma_commit(ms.bar);
  }
  if (!ms.wait()) return false;
  // the MMA that read `out` (in place for inference) has completed
  hidden_epilogue(tm + lane_off, bias, out, threadIdx.x);
  operands_ready();
  return true;
}

// Output layer logits z = a3 W4^T + b4 (16 columns, 9 used).
__device__ __forceinline__ bool out_layer(uint32_t a_in, uint32_t b_w, const float* bias,
                                          float* z, uint32_t tm, uint32_t lane_off,
                                          MmaSync& ms) {
  if (threadIdx.x == 0) {
    umma_tile(tm, a_in, b_w, MLP_OUT, MLP_H, 0);
    umma_commit(ms.bar);
  }
  if (!ms.wait()) return false;
  tmem_ld16(tm + lane_off, z);
#pragma unroll
  for (int j = 0; j < MLP_OUT; j++) z[j] += bias[j];
  return true;
}

// Softmax over each phase's three logits.
__device__ __forceinline__ void softmax3(const float* z, float* y) {
#pragma unroll
  for (int p = 0; p < MLP_MAXP; p++) {
    float a0 = z[3 * p], a1 = z[3 * p + 1], a2 = z[3 * p + 2];
    float mx = fmaxf(a0, fmaxf(a1, a2));
    float e0 = __expf(a0 - mx), e1 = __expf(a1 - mx), e2 = __expf(a2 - mx);
    float r = 1.0f / (e0 + e1 + e2);
    y[3 * p] = e0 * r;
    y[3 * p + 1] = e1 * r;
    y[3 * p + 2] = e2 * r;
  }
}

// Shared-memory plan of the inference kernel.
struct FwdSmem {
  static constexpr int W1 = 0, W2 = W1 + 64 * 32 * 2, W3 = W2 + 64 * 64 * 2,
                       W4 = W3 + 64 * 64 * 2, X = W4 + 16 * 64 * 2, A = X + 128 * 32 * 2,
                       BIAS = A + 128 * 64 * 2, BYTES = BIAS + MLP_NBIAS * 4;
};

__device__ __forceinline__ void stage_weights_fwd(unsigned char* sm, const MlpPtrs& P) {
  stage_matrix<64, 32, false>(sm + FwdSmem::W1, P.W + MLP_W1);
  stage_matrix<64, 64, false>(sm + FwdSmem::W2, P.W + MLP_W2);
  stage_matrix<64, 64, false>(sm + FwdSmem::W3, P.W + MLP_W3);
  stage_matrix<16, 64, false>(sm + FwdSmem::W4, P.W + MLP_W4);
  float* sb = reinterpret_cast<float*>(sm + FwdSmem::BIAS);
  for (int i = threadIdx.x; i < MLP_NBIAS; i += blockDim.x) sb[i] = P.b[i];
}

// Rows of a row-major BF16 feature matrix in, row-major FP32 weights out.
struct SrcRows {
  const __nv_bfloat16* X;
  float* Y;
  long nrows;
  __device__ __forceinline__ long rows() const { return nrows; }
  __device__ __forceinline__ void load(long row, unsigned char* sX) const {
    const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      uint4 v = row < nrows ? reinterpret_cast<const uint4*>(X + row * MLP_IN)[c] : z;
      *reinterpret_cast<uint4*>(sX + cm_offset(threadIdx.x, c * 8, MLP_IN)) = v;
    }
  }
  __device__ __forceinline__ void store(long row, const float* y) const {
    if (row < nrows) {
#pragma unroll
      for (int j = 0; j < MLP_NW; j++) Y[row * MLP_NW + j] = y[j];
    }
  }
};

// Stencil gather of one face side of one cell from the state, with the
// boundary condition of the sweep direction (masses and fractions need no
// sign flip).  Side 0: values f_{i-2..i+2} for x_{i+1/2}; side 1: the mirror
// image for x_{i-1/2}.
template <int N, int D>
__device__ __forceinline__ void gather_stencil(const MlpGeom& g, long cell, int side,
                                               double (*ms)[5], double (*as)[5]) {
  using I = Idx<N, D>;
  int i, j, k;
  if (g.ncell <= 0xFFFFFFFFL) {  // 32-bit index arithmetic
    const unsigned c = (unsigned)cell, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
    const unsigned r = c / nx;
    i = (int)(c - r * nx);
    j = (int)(r % ny);
    k = (int)(r / ny);
  } else {
    i = (int)(cell % g.nx);
    j = (int)((cell / g.nx) % g.ny);
    k = (int)(cell / ((long)g.nx * g.ny));
  }
  const int pos = g.dir == 0 ? i : (g.dir == 1 ? j : k);
  const long base = cell - (long)pos * g.stride;
#pragma unroll
  for (int s = 0; s < 5; s++) {
    const int o = side == 0 ? s : 4 - s;
    bool flip;
    const int jj = bc_index(pos - 2 + o, g.n, g.bclo, g.bchi, flip);
    const long c2 = base + (long)jj * g.stride;
#pragma unroll
    for (int p = 0; p < N; p++) {
      ms[p][s] = __ldg(g.U + (long)p * g.ncell + c2);
      as[p][s] = __ldg(g.U + (long)I::A(p) * g.ncell + c2);
    }
  }
}

// ------------------------------------------------------------------ inference
template <class Src>
__global__ void __launch_bounds__(128) k_mlp_fwd(Src src, const void* params, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int t = threadIdx.x;
  stage_weights_fwd(sm, mlp_ptrs(params));
  tile_setup(&tbase, &bar, 64);
  operands_ready();
  const uint32_t tm = tbase, lane_off = (uint32_t)(32 * (t >> 5)) << 16;
  const float* sb = reinterpret_cast<const float*>(sm + FwdSmem::BIAS);
  unsigned char* sX = sm + FwdSmem::X;
  unsigned char* sA = sm + FwdSmem::A;
  const uint32_t aX = smem_u32(sX), aA = smem_u32(sA);
  MmaSync ms{&bar, 0u};
  bool ok = true;
  const long ntile = (src.rows() + 127) / 128;
  for (long tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
    const long row = tile * 128 + t;
    // the previous tile's MMAs have completed and every thread has passed
    // the barrier after its last accumulator read
    src.load(row, sX);
    operands_ready();
    ok = fwd_layer<MLP_IN>(aX, smem_u32(sm + FwdSmem::W1), sb + MLP_B1, sA, tm, lane_off, ms) &&
         fwd_layer<MLP_H>(aA, smem_u32(sm + FwdSmem::W2), sb + MLP_B2, sA, tm, lane_off, ms) &&
         fwd_layer<MLP_H>(aA, smem_u32(sm + FwdSmem::W3), sb + MLP_B3, sA, tm, lane_off, ms);
    float z[MLP_OUT], y[MLP_NW];
    if (ok) ok = out_layer(aA, smem_u32(sm + FwdSmem::W4), sb + MLP_B4, z, tm, lane_off, ms);
    if (ok) {
      softmax3(z, y);
      src.store(row, y);
    }
  }
  if (!ok) {
    ms.drain();
    if (t == 0) atomicOr(status, ST_TIMEOUT);
  }
  tile_teardown(tm, 64);
}

// Inference of one sweep direction straight from the state: each iteration
// takes 128 cells, thread t gathers cell t's stencil once and builds the
// features of both its face sides (tile A: side 0 rows, tile B: side 1
// rows); the two tiles' MMAs of a layer are issued back to back into
// tensor-memory columns [0, 64) and [64, 128) and share one commit.
// Weights go to W[(9 side + j) ncell + cell].
// The features ([128][32] per tile) are built in the activation buffers
// themselves: layer 1 reads them before its epilogue overwrites them, which
// keeps the CTA at 56 KB of shared memory (4 CTAs per SM).
struct Infer2Smem {
  static constexpr int W1 = 0, W2 = W1 + 64 * 32 * 2, W3 = W2 + 64 * 64 * 2,
                       W4 = W3 + 64 * 64 * 2, AA = W4 + 16 * 64 * 2, AB = AA + 128 * 64 * 2,
                       BIAS = AB + 128 * 64 * 2, BYTES = BIAS + MLP_NBIAS * 4;
};

template <int K>
__device__ __forceinline__ bool fwd_layer2(uint32_t aA, uint32_t aB, uint32_t b_w,
                                           const float* bias, unsigned char* outA,
                                           unsigned char* outB, uint32_t tm, uint32_t lane_off,
                                           MmaSync& ms) {
  if (threadIdx.x == 0) {
    umma_tile(tm, aA, b_w, MLP_H, K, 0);
    umma_tile(tm + 64, aB, b_w, MLP_H, K, 0);
    umma_commit(ms.bar);
  }
  if (!ms.wait()) return false;
  hidden_epilogue(tm + lane_off, bias, outA, threadIdx.x);
  hidden_epilogue(tm + lane_off + 64, bias, outB, threadIdx.x);
  operands_ready();
  return true;
}

template <int N, int D>
__global__ void __launch_bounds__(128) k_mlp_infer2(MlpGeom g, const void* params, float* W,
                                                    unsigned* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int t = threadIdx.x;
  {
    const MlpPtrs P = mlp_ptrs(params);
    stage_matrix<64, 32, false>(sm + Infer2Smem::W1, P.W + MLP_W1);
    stage_matrix<64, 64, false>(sm + Infer2Smem::W2, P.W + MLP_W2);
    stage_matrix<64, 64, false>(sm + Infer2Smem::W3, P.W + MLP_W3);
    stage_matrix<16, 64, false>(sm + Infer2Smem::W4, P.W + MLP_W4);
    float* sb = reinterpret_cast<float*>(sm + Infer2Smem::BIAS);
    for (int i = t; i < MLP_NBIAS; i += blockDim.x) sb[i] = P.b[i];
  }
  tile_setup(&tbase, &bar, 128);
  operands_ready();
  const uint32_t tm = tbase, lane_off = (uint32_t)(32 * (t >> 5)) << 16;
  const float* sb = reinterpret_cast<const float*>(sm + Infer2Smem::BIAS);
  unsigned char* sAA = sm + Infer2Smem::AA;
  unsigned char* sAB = sm + Infer2Smem::AB;
  const uint32_t aAA = smem_u32(sAA), aAB = smem_u32(sAB);
  MmaSync ms{&bar, 0u};
  bool ok = true;
  const long nit = (g.ncell + 127) / 128;
  for (long it = blockIdx.x; it < nit && ok; it += gridDim.x) {
    const long cell = it * 128 + t;
    __align__(16) __nv_bfloat16 x0[MLP_IN], x1[MLP_IN];
    if (cell < g.ncell) {
      double mstc[N][5], astc[N][5];
      gather_stencil<N, D>(g, cell, 0, mstc, astc);
      mlp_features2<N>(mstc, astc, x0, x1);
    } else {
#pragma unroll
      for (int k = 0; k < MLP_IN; k++) x0[k] = x1[k] = __float2bfloat16(0.0f);
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
      *reinterpret_cast<uint4*>(sAA + cm_offset(t, c * 8, MLP_IN)) =
          reinterpret_cast<const uint4*>(x0)[c];
      *reinterpret_cast<uint4*>(sAB + cm_offset(t, c * 8, MLP_IN)) =
          reinterpret_cast<const uint4*>(x1)[c];
    }
    operands_ready();
    ok = fwd_layer2<MLP_IN>(aAA, aAB, smem_u32(sm + Infer2Smem::W1), sb + MLP_B1, sAA, sAB, tm,
                            lane_off, ms) &&
         fwd_layer2<MLP_H>(aAA, aAB, smem_u32(sm + Infer2Smem::W2), sb + MLP_B2, sAA, sAB, tm,
                           lane_off, ms) &&
         fwd_layer2<MLP_H>(aAA, aAB, smem_u32(sm + Infer2Smem::W3), sb + MLP_B3, sAA, sAB, tm,
                           lane_off, ms);
    if (ok) {
      if (t == 0) {
        umma_tile(tm, aAA, smem_u32(sm + Infer2Smem::W4), MLP_OUT, MLP_H, 0);
        umma_tile(tm + 64, aAB, smem_u32(sm + Infer2Smem::W4), MLP_OUT, MLP_H, 0);
        umma_commit(ms.bar);
      }
      ok = ms.wait();
    }
    if (ok) {
#pragma unroll
      for (int side = 0; side < 2; side++) {
        float z[MLP_OUT], y[MLP_NW];
        tmem_ld16(tm + lane_off + 64 * side, z);
#pragma unroll
        for (int j = 0; j < MLP_OUT; j++) z[j] += sb[MLP_B4 + j];
        softmax3(z, y);
        if (cell < g.ncell) {
#pragma unroll
          for (int j = 0; j < 3 * N; j++) W[(long)(MLP_NW * side + j) * g.ncell + cell] = y[j];
        }
      }
      // the next iteration's MMAs overwrite the accumulator only after every
      // thread has read it (barrier in operands_ready)
    }
  }
  if (!ok) {
    ms.drain();
    if (t == 0) atomicOr(status, ST_TIMEOUT);
  }
  tile_teardown(tm, 128);
}

// ------------------------------------------------------------------ training
struct TrainSmem {
  static constexpr int W1 = 0, W2 = W1 + 64 * 32 * 2, W3 = W2 + 64 * 64 * 2,
                       W4 = W3 + 64 * 64 * 2, W2T = W4 + 16 * 64 * 2, W3T = W2T + 64 * 64 * 2,
                       W4T = W3T + 64 * 64 * 2, X = W4T + 64 * 16 * 2, A1 = X + 128 * 32 * 2,
                       A2 = A1 + 128 * 64 * 2, A3 = A2 + 128 * 64 * 2,
                       D = A3 + 128 * 64 * 2,        // delta rows [128][<=64]
                       DT = D + 128 * 64 * 2,        // delta^T [128][128]
                       AT = DT + 128 * 128 * 2,      // input activations^T [<=64][128]
                       BIAS = AT + 64 * 128 * 2, DB = BIAS + MLP_NBIAS * 4,
                       BYTES = DB + 64 * 4;
};

// Backward through one layer (input width IN, output width OUT): weight and
// bias gradients accumulated into gW / gb, and, when BELOW, the delta of the
// layer underneath (dA = delta W on the tensor cores, times relu').
template <int IN, int OUT, bool BELOW>
__device__ __forceinline__ bool bwd_layer(float (&d)[MLP_H], unsigned char* sm,
                                          const unsigned char* sIn, uint32_t w_t, float* gW,
                                          float* gb, uint32_t tm, uint32_t lane_off,
                                          MmaSync& ms) {
  const int t = threadIdx.x, lane = t & 31;
  float* s_db = reinterpret_cast<float*>(sm + TrainSmem::DB);
  unsigned char* sD = sm + TrainSmem::D;
  unsigned char* sDT = sm + TrainSmem::DT;
  unsigned char* sAT = sm + TrainSmem::AT;
  const uint32_t dW_t = tm, dA_t = tm + 64;
  if (t < 64) s_db[t] = 0.0f;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < OUT; j++) {
    float v = d[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(&s_db[j], v);
  }
  float act[IN];
  get_row<IN>(sIn, t, act);
  put_col<OUT>(sDT, t, d);
  put_col<IN>(sAT, t, act);
  if (BELOW) put_row<OUT>(sD, t, d);
  operands_ready();
  if (t == 0) {
    // dW[j][k] = sum_s delta[s][j] act[s][k]  (M = 128 rows of delta^T, N = IN)
    umma_tile(dW_t, smem_u32(sDT), smem_u32(sAT), IN, 128, 0);
    // dA[s][k] = sum_j delta[s][j] W[j][k]  (B = W^T stored [IN][OUT])
    if (BELOW) umma_tile(dA_t, smem_u32(sD), w_t, IN, OUT, 0);
    umma_commit(ms.bar);
  }
  if (!ms.wait()) return false;
#pragma unroll
  for (int c = 0; c < IN; c += 16) {
    float g[16];
    tmem_ld16(dW_t + lane_off + c, g);
    if (t < OUT) {
#pragma unroll
      for (int q = 0; q < 16; q++) atomicAdd(&gW[t * IN + c + q], g[q]);
    }
  }
  if (t < OUT) atomicAdd(&gb[t], s_db[t]);
  if (BELOW) {
#pragma unroll
    for (int c = 0; c < IN; c += 16) {
      float da[16];
      tmem_ld16(dA_t + lane_off + c, da);
#pragma unroll
      for (int q = 0; q < 16; q++) d[c + q] = act[c + q] > 0.0f ? da[q] : 0.0f;
    }
  }
  tc_fence_before();
  __syncthreads();
  return true;
}

// Weight of the reconstruction terms of the loss.
constexpr float kReconWeight = 1.0f;

// Candidate values (Eq. 10, minus the cell value) of one phase's normalised
// mass stencil xm[0..5) (cell value 0) and of its fraction stencil xa[0..5)
// shifted by the cell's fraction and divided by its largest absolute
// deviation (0 when that deviation is at most 1e-30), for the face the
// stencil is ordered towards.
__device__ __forceinline__ void recon_candidates(const float* xm, const float* xa, float* qm,
                                                 float* qa) {
  const float s6 = 1.0f / 6.0f;
  qm[0] = (2.0f * xm[0] - 7.0f * xm[1]) * s6;
  qm[1] = (2.0f * xm[3] - xm[1]) * s6;
  qm[2] = (5.0f * xm[3] - xm[4]) * s6;
  float da[5], mx = 0.0f;
#pragma unroll
  for (int k = 0; k < 5; k++) {
    da[k] = xa[k] - xa[2];
    mx = fmaxf(mx, fabsf(da[k]));
  }
  const float r = mx > 1e-30f ? 1.0f / mx : 0.0f;  // flat below 1e-30
  qa[0] = (2.0f * da[0] - 7.0f * da[1]) * s6 * r;
  qa[1] = (2.0f * da[3] - da[1]) * s6 * r;
  qa[2] = (5.0f * da[3] - da[4]) * s6 * r;
}

// One tile of 128 samples idx[128 blockIdx ..]: forward with the activations
// kept, softmax, loss, backward on the tensor cores, FP32 gradients
// accumulated into grads (atomics) and the loss into *loss.  Loss of a
// sample, summed over the phases p: sum_s e_ps^2 + lambda ((sum_s e_ps
// qm_ps)^2 + (sum_s e_ps qa_ps)^2), e = y - target, where qm, qa are the
// candidate values of the normalised mass and fraction stencils (the error of
// the reconstructions the acceptance test compares, in units of the
// stencil's deviation); the batch mean of that sum.
__global__ void __launch_bounds__(128) k_mlp_train(const __nv_bfloat16* __restrict__ X,
                                                   const float* __restrict__ T,
                                                   const int* __restrict__ idx, int batch,
                                                   const void* params, float* grads, float* loss,
                                                   unsigned* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ float s_loss[4];
  const int t = threadIdx.x;
  const MlpPtrs P = mlp_ptrs(params);
  stage_matrix<64, 32, false>(sm + TrainSmem::W1, P.W + MLP_W1);
  stage_matrix<64, 64, false>(sm + TrainSmem::W2, P.W + MLP_W2);
  stage_matrix<64, 64, false>(sm + TrainSmem::W3, P.W + MLP_W3);
  stage_matrix<16, 64, false>(sm + TrainSmem::W4, P.W + MLP_W4);
  stage_matrix<64, 64, true>(sm + TrainSmem::W2T, P.W + MLP_W2);
  stage_matrix<64, 64, true>(sm + TrainSmem::W3T, P.W + MLP_W3);
  stage_matrix<16, 64, true>(sm + TrainSmem::W4T, P.W + MLP_W4);
  float* sb = reinterpret_cast<float*>(sm + TrainSmem::BIAS);
  for (int i = t; i < MLP_NBIAS; i += blockDim.x) sb[i] = P.b[i];
  // delta^T rows beyond a layer's width stay zero
  for (int i = t; i < 128 * 128 * 2 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sm + TrainSmem::DT)[i] = make_uint4(0, 0, 0, 0);
  tile_setup(&tbase, &bar, 128);
  const int s = blockIdx.x * 128 + t;
  const bool valid = s < batch;
  const long sample = valid ? (long)idx[s] : 0;
  {
    const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      uint4 v = valid ? reinterpret_cast<const uint4*>(X + sample * MLP_IN)[c] : z;
      *reinterpret_cast<uint4*>(sm + TrainSmem::X + cm_offset(t, c * 8, MLP_IN)) = v;
    }
  }
  operands_ready();
  const uint32_t tm = tbase, lane_off = (uint32_t)(32 * (t >> 5)) << 16;
  MmaSync ms{&bar, 0u};
  float z[MLP_OUT];
  bool ok =
      fwd_layer<MLP_IN>(smem_u32(sm + TrainSmem::X), smem_u32(sm + TrainSmem::W1), sb + MLP_B1,
                        sm + TrainSmem::A1, tm, lane_off, ms) &&
      fwd_layer<MLP_H>(smem_u32(sm + TrainSmem::A1), smem_u32(sm + TrainSmem::W2), sb + MLP_B2,
                       sm + TrainSmem::A2, tm, lane_off, ms) &&
      fwd_layer<MLP_H>(smem_u32(sm + TrainSmem::A2), smem_u32(sm + TrainSmem::W3), sb + MLP_B3,
                       sm + TrainSmem::A3, tm, lane_off, ms) &&
      out_layer(smem_u32(sm + TrainSmem::A3), smem_u32(sm + TrainSmem::W4), sb + MLP_B4, z, tm,
                lane_off, ms);
  if (ok) {
    // softmax, squared error and the gradient of the logits
    float d[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; j++) d[j] = 0.0f;
    float lsum = 0.0f;
    if (valid) {
      float y[MLP_NW], x[MLP_IN];
      softmax3(z, y);
      get_row<MLP_IN>(sm + TrainSmem::X, t, x);
      const float* tg = T + sample * MLP_NW;
      const float scale = 2.0f / (float)batch;
#pragma unroll
      for (int p = 0; p < MLP_MAXP; p++) {
        float qm[3], qa[3], err[3];
        recon_candidates(x + 10 * p, x + 10 * p + 5, qm, qa);
        float em = 0.0f, ea = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
          err[k] = y[3 * p + k] - tg[3 * p + k];
          lsum += err[k] * err[k];
          em += err[k] * qm[k];
          ea += err[k] * qa[k];
        }
        lsum += kReconWeight * (em * em + ea * ea);
        float dy[3], dot = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
          dy[k] = scale * (err[k] + kReconWeight * (em * qm[k] + ea * qa[k]));
          dot += dy[k] * y[3 * p + k];
        }
#pragma unroll
        for (int k = 0; k < 3; k++) d[3 * p + k] = y[3 * p + k] * (dy[k] - dot);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0) s_loss[t >> 5] = lsum;
    tc_fence_before();
    __syncthreads();
    if (t == 0) atomicAdd(loss, (s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3]) / (float)batch);
    ok = bwd_layer<MLP_H, MLP_OUT, true>(d, sm, sm + TrainSmem::A3,
                                         smem_u32(sm + TrainSmem::W4T), grads + MLP_W4,
                                         grads + MLP_NWEIGHT + MLP_B4, tm, lane_off, ms) &&
         bwd_layer<MLP_H, MLP_H, true>(d, sm, sm + TrainSmem::A2, smem_u32(sm + TrainSmem::W3T),
                                       grads + MLP_W3, grads + MLP_NWEIGHT + MLP_B3, tm,
                                       lane_off, ms) &&
         bwd_layer<MLP_H, MLP_H, true>(d, sm, sm + TrainSmem::A1, smem_u32(sm + TrainSmem::W2T),
                                       grads + MLP_W2, grads + MLP_NWEIGHT + MLP_B2, tm,
                                       lane_off, ms) &&
         bwd_layer<MLP_IN, MLP_H, false>(d, sm, sm + TrainSmem::X, 0u, grads + MLP_W1,
                                         grads + MLP_NWEIGHT + MLP_B1, tm, lane_off, ms);
  }
  if (!ok) {
    ms.drain();
    if (t == 0) atomicOr(status, ST_TIMEOUT);
  }
  tile_teardown(tm, 128);
}

// Is entry i of the parameter array padding (inputs 30, 31 of W1; outputs
// 9..15 of W4 and b4)?  Padding stays zero.
__host__ __device__ __forceinline__ bool is_padding(int i) {
  if (i < MLP_W2) return (i % MLP_IN) >= 30;
  if (i >= MLP_W4 && i < MLP_NWEIGHT) return ((i - MLP_W4) / MLP_H) >= MLP_NW;
  if (i >= MLP_NWEIGHT) return (i - MLP_NWEIGHT) >= MLP_B4 + MLP_NW;
  return false;
}

__device__ __forceinline__ void store_param(void* params, int i, float p) {
  if (i < MLP_NWEIGHT)
    reinterpret_cast<__nv_bfloat16*>(params)[i] = __float2bfloat16(p);
  else
    reinterpret_cast<float*>(reinterpret_cast<char*>(params) +
                             (size_t)MLP_NWEIGHT * sizeof(__nv_bfloat16))[i - MLP_NWEIGHT] = p;
}

// Adam (Kingma & Ba) on the FP32 masters, bias-corrected with c1 = 1/(1 -
// beta1^step), c2 = 1/(1 - beta2^step); refreshes the BF16 weights and the
// biases of the parameter block and clears the gradients.
__global__ void k_mlp_adam(float* master, void* params, float* grads, float* m, float* v,
                           float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NPARAM;
       i += gridDim.x * blockDim.x) {
    const float g = grads[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float p = master[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    if (is_padding(i)) p = 0.0f;
    master[i] = p;
    store_param(params, i, p);
    grads[i] = 0.0f;
  }
}

__global__ void k_mlp_pack(const float* master, void* params) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NPARAM;
       i += gridDim.x * blockDim.x)
    store_param(params, i, is_padding(i) ? 0.0f : master[i]);
}

// Features and plain-weight targets of both face sides of every cell for
// one sweep direction; row = row0 + 2 cell + side.  Targets: the Eq. 15
// weights of each phase's masses on the oriented stencil (the weights the
// coupled reconstruction, Eq. 16, applies to masses and fractions); phases
// beyond N get the ideal weights, which is what Eq. 15 gives on an absent
// (all-zero) phase.  Rows whose targets differ from the ideal weights by more
// than 1e-3 somewhere are counted in *count and, when list is not null,
// appended to it (up to cap entries).
template <int N, int D>
__global__ void k_mlp_features(MlpGeom g, long row0, __nv_bfloat16* X, float* T, long* list,
                               unsigned long long* count, long cap) {
  for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < 2 * g.ncell;
       r += (long)gridDim.x * blockDim.x) {
    const long cell = r >> 1;
    const int side = (int)(r & 1);
    double ms[N][5], as[N][5];
    gather_stencil<N, D>(g, cell, 0, ms, as);
    const long row = row0 + r;
    __align__(16) __nv_bfloat16 x[MLP_IN];
    mlp_features2<N>(ms, as, side == 0 ? x : nullptr, side == 1 ? x : nullptr);
#pragma unroll
    for (int c = 0; c < 4; c++)
      reinterpret_cast<uint4*>(X + row * MLP_IN)[c] = reinterpret_cast<const uint4*>(x)[c];
    if (!T) continue;
    const double ideal[3] = {0.1, 0.6, 0.3};
    bool inter = false;
#pragma unroll
    for (int p = 0; p < MLP_MAXP; p++) {
      double w[3] = {ideal[0], ideal[1], ideal[2]};
      if (p < N) {
        // the stencil ordered towards this side's face
        const int o = side == 0 ? 0 : 4;
        const Stencil<double> st = stencil<double>(ms[p][o], ms[p][o ? 3 : 1], ms[p][2],
                                                   ms[p][o ? 1 : 3], ms[p][o ? 0 : 4]);
        const W6<double> wt = weights_of<double>(st);
        const double s6 = 6.0 * wt.invL;
        w[0] = wt.aL0 * s6;
        w[1] = wt.aL1 * s6;
        w[2] = wt.aL2 * s6;
      }
#pragma unroll
      for (int k = 0; k < 3; k++) {
        T[row * MLP_NW + 3 * p + k] = (float)w[k];
        inter |= fabs(w[k] - ideal[k]) > 1e-3;
      }
    }
    if (inter && count) {
      const unsigned long long slot = atomicAdd(count, 1ull);
      if (list && (long)slot < cap) list[slot] = row;
    }
  }
}

cudaError_t launch_mlp_forward(const __nv_bfloat16* X, long nrows, const void* params, float* Y,
                               unsigned* status, cudaStream_t st) {
  auto k = k_mlp_fwd<SrcRows>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       FwdSmem::BYTES);
  if (e != cudaSuccess) return e;
  const long ntile = (nrows + 127) / 128;
  const int grid = (int)std::max(1L, std::min(ntile, 148L * 4));
  k<<<grid, 128, FwdSmem::BYTES, st>>>(SrcRows{X, Y, nrows}, params, status);
  return cudaGetLastError();
}

template <int N, int D>
static cudaError_t infer_nd(const MlpGeom& g, const void* params, float* W, unsigned* status,
                            cudaStream_t st) {
  auto k = k_mlp_infer2<N, D>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Infer2Smem::BYTES);
  if (e != cudaSuccess) return e;
  const long nit = (g.ncell + 127) / 128;
  const int grid = (int)std::max(1L, std::min(nit, 148L * 4));
  k<<<grid, 128, Infer2Smem::BYTES, st>>>(g, params, W, status);
  return cudaGetLastError();
}

template <int N>
static cudaError_t infer_n(int D, const MlpGeom& g, const void* params, float* W,
                           unsigned* status, cudaStream_t st) {
  if (D == 1) return infer_nd<N, 1>(g, params, W, status, st);
  if (D == 2) return infer_nd<N, 2>(g, params, W, status, st);
  return infer_nd<N, 3>(g, params, W, status, st);
}

cudaError_t launch_mlp_infer(const MlpGeom& g, const void* params, float* W, unsigned* status,
                             cudaStream_t st) {
  const int D = g.nv - 2 * g.N - 1;
  if (g.N == 1) return infer_n<1>(D, g, params, W, status, st);
  if (g.N == 2) return infer_n<2>(D, g, params, W, status, st);
  if (g.N == 3) return infer_n<3>(D, g, params, W, status, st);
  return cudaErrorInvalidValue;
}

template <int N, int D>
static cudaError_t features_nd(const MlpGeom& g, long row0, __nv_bfloat16* X, float* T,
                               long* list, unsigned long long* count, long cap,
                               cudaStream_t st) {
  const long rows = 2 * g.ncell;
  const int grid = (int)std::max(1L, std::min((rows + 255) / 256, 148L * 16));
  k_mlp_features<N, D><<<grid, 256, 0, st>>>(g, row0, X, T, list, count, cap);
  return cudaGetLastError();
}

template <int N>
static cudaError_t features_n(int D, const MlpGeom& g, long row0, __nv_bfloat16* X, float* T,
                              long* list, unsigned long long* count, long cap, cudaStream_t st) {
  if (D == 1) return features_nd<N, 1>(g, row0, X, T, list, count, cap, st);
  if (D == 2) return features_nd<N, 2>(g, row0, X, T, list, count, cap, st);
  return features_nd<N, 3>(g, row0, X, T, list, count, cap, st);
}

cudaError_t launch_mlp_features(const MlpGeom& g, long row0, __nv_bfloat16* X, float* T,
                                long* list, unsigned long long* count, long cap,
                                cudaStream_t st) {
  const int D = g.nv - 2 * g.N - 1;
  if (g.N == 1) return features_n<1>(D, g, row0, X, T, list, count, cap, st);
  if (g.N == 2) return features_n<2>(D, g, row0, X, T, list, count, cap, st);
  if (g.N == 3) return features_n<3>(D, g, row0, X, T, list, count, cap, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_mlp_train(const __nv_bfloat16* X, const float* T, const int* idx, int batch,
                             const void* params, float* grads, float* loss, unsigned* status,
                             cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TrainSmem::BYTES);
  if (e != cudaSuccess) return e;
  const int grid = (batch + 127) / 128;
  k_mlp_train<<<grid, 128, TrainSmem::BYTES, st>>>(X, T, idx, batch, params, grads, loss,
                                                   status);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* master, void* params, float* grads, float* m, float* v,
                            float lr, float beta1, float beta2, float eps, int step,
                            cudaStream_t st) {
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)step)));
  k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(master, params, grads, m, v, lr, beta1,
                                                       beta2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace wc

using namespace wc;

static wc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WC_OK : WC_ERR_CUDA; }

extern "C" size_t wc_mlp_param_bytes(void) { return MLP_PARAM_BYTES; }
extern "C" int wc_mlp_nparam(void) { return MLP_NPARAM; }

extern "C" wc_status wc_mlp_init_master(float* master_host, unsigned long long seed) {
  if (!master_host) return WC_ERR_ARG;
  std::mt19937_64 rng(seed);
  auto fill = [&](int off, int out, int in, int used_out, int used_in) {
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (double)used_in));
    for (int o = 0; o < out; o++)
      for (int i = 0; i < in; i++)
        master_host[off + o * in + i] = (o < used_out && i < used_in) ? (float)nd(rng) : 0.0f;
  };
  fill(MLP_W1, MLP_H, MLP_IN, MLP_H, 30);
  fill(MLP_W2, MLP_H, MLP_H, MLP_H, MLP_H);
  fill(MLP_W3, MLP_H, MLP_H, MLP_H, MLP_H);
  fill(MLP_W4, MLP_OUT, MLP_H, MLP_NW, MLP_H);
  for (int i = 0; i < MLP_NBIAS; i++) master_host[MLP_NWEIGHT + i] = 0.0f;
  return WC_OK;
}

extern "C" wc_status wc_mlp_pack(const float* master_dev, void* params_dev, void* stream) {
  if (!master_dev || !params_dev) return WC_ERR_ARG;
  k_mlp_pack<<<(MLP_NPARAM + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      master_dev, params_dev);
  return cuda_status(cudaGetLastError());
}

extern "C" wc_status wc_mlp_forward(const void* X_dev, long nrows, const void* params_dev,
                                    float* Y_dev, unsigned* status_dev, void* stream) {
  if (!X_dev || !params_dev || !Y_dev || !status_dev || nrows < 0) return WC_ERR_ARG;
  if (nrows == 0) return WC_OK;
  return cuda_status(launch_mlp_forward(reinterpret_cast<const __nv_bfloat16*>(X_dev), nrows,
                                        params_dev, Y_dev, status_dev,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" wc_status wc_mlp_gradients(const void* X_dev, const float* T_dev, const int* idx_dev,
                                      int batch, const void* params_dev, float* grads_dev,
                                      float* loss_dev, unsigned* status_dev, void* stream) {
  if (!X_dev || !T_dev || !idx_dev || batch < 1 || !params_dev || !grads_dev || !loss_dev ||
      !status_dev)
    return WC_ERR_ARG;
  return cuda_status(launch_mlp_train(reinterpret_cast<const __nv_bfloat16*>(X_dev), T_dev,
                                      idx_dev, batch, params_dev, grads_dev, loss_dev,
                                      status_dev, reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" wc_status wc_mlp_adam(float* master_dev, void* params_dev, float* grads_dev,
                                 float* m_dev, float* v_dev, float lr, int step, void* stream) {
  if (!master_dev || !params_dev || !grads_dev || !m_dev || !v_dev || step < 1 || !(lr > 0.0f))
    return WC_ERR_ARG;
  return cuda_status(launch_mlp_adam(master_dev, params_dev, grads_dev, m_dev, v_dev, lr, 0.9f,
                                     0.999f, 1e-8f, step,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" wc_status wc_mlp_train_step(const void* X_dev, const float* T_dev, const int* idx_dev,
                                       int batch, void* params_dev, float* master_dev,
                                       float* grads_dev, float* m_dev, float* v_dev, float lr,
                                       int step, float* loss_dev, unsigned* status_dev,
                                       void* stream) {
  wc_status s = wc_mlp_gradients(X_dev, T_dev, idx_dev, batch, params_dev, grads_dev, loss_dev,
                                 status_dev, stream);
  if (s != WC_OK) return s;
  return wc_mlp_adam(master_dev, params_dev, grads_dev, m_dev, v_dev, lr, step, stream);
}
