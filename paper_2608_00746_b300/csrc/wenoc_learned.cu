// wenoc_learned.cu -- instantiations of the direction sweep with learned
// mass weights (FP32 reconstruction and flux as in the mixed precision, the
// surrogate's weights accepted against the plain ones) for N = 1..3 phases
// and d = 1..3 directions.
#include "wenoc_kernels.cuh"
#include "wenoc_window.cuh"

namespace wc {

template <int N, int D>
static cudaError_t go(const SweepArgs& a, const Mat& m, int block, cudaStream_t st) {
  if (a.nwin > 0) {
    if (a.fbuf) return launch_split<N, D, float, float, 1>(a, m, block, st);
    const int bps = (int)(a.max_threads / (148L * block));  // 0: occupancy limit
    return launch_window<N, D, float, float, 1>(a, m, block, bps, st);
  }
  const int smem = Ring<N, D, float>::BYTES * block;
  auto k = k_sweep<N, D, float, float, 1>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  long threads = a.npencil * a.nseg;
  if (a.max_threads > 0 && threads > a.max_threads) threads = a.max_threads;
  long blocks = (threads + block - 1) / block;
  k<<<(unsigned)blocks, block, smem, st>>>(a, m);
  return cudaGetLastError();
}

template <int N>
static cudaError_t goN(int D, const SweepArgs& a, const Mat& m, int block, cudaStream_t st) {
  if (D == 1) return go<N, 1>(a, m, block, st);
  if (D == 2) return go<N, 2>(a, m, block, st);
  return go<N, 3>(a, m, block, st);
}

cudaError_t launch_sweep_learned(int N, int D, const SweepArgs& a, const Mat& m, int block,
                                 cudaStream_t st) {
  switch (N) {
    case 1: return goN<1>(D, a, m, block, st);
    case 2: return goN<2>(D, a, m, block, st);
    case 3: return goN<3>(D, a, m, block, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wc
