// wenoc_compare.cu -- instantiations of the direction sweep for the
// comparison schemes of Sec. 4.1.1 (WENO-W and WENO-JS weights, every
// primitive variable with its own weights, no limiters) in FP64, for N =
// 1..5 phases and d = 1..3 directions.
#include "wenoc_kernels.cuh"
#include "wenoc_window.cuh"

namespace wc {

template <int N, int D>
static cudaError_t go(const SweepArgs& a, const Mat& m, int block, cudaStream_t st) {
  if (a.nwin > 0) {
    const int bps = (int)(a.max_threads / (148L * block));  // 0: occupancy limit
    return launch_window<N, D, double, double, 2>(a, m, block, bps, st);
  }
  const int smem = Ring<N, D, double>::BYTES * block;
  auto k = k_sweep<N, D, double, double, 2>;
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

cudaError_t launch_sweep_compare(int N, int D, const SweepArgs& a, const Mat& m, int block,
                                 cudaStream_t st) {
  switch (N) {
    case 1: return goN<1>(D, a, m, block, st);
    case 2: return goN<2>(D, a, m, block, st);
    case 3: return goN<3>(D, a, m, block, st);
    case 4: return goN<4>(D, a, m, block, st);
    case 5: return goN<5>(D, a, m, block, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wc
