// wenoc_mixed.cu -- instantiations of the direction sweep with reconstruction
// type float and flux type float for N = 1..5 phases and d = 1..3 directions.
#include "wenoc_kernels.cuh"
#include "wenoc_window.cuh"

namespace wc {

template <int N, int D>
static cudaError_t go(const SweepArgs& a, const Mat& m, int block, cudaStream_t st) {
  if (a.nwin > 0) {
    if (a.fbuf) return launch_split<N, D, float, float, 0>(a, m, block, st);
    const int bps = (int)(a.max_threads / (148L * block));  // 0: occupancy limit
    return launch_window<N, D, float, float, 0>(a, m, block, bps, st);
  }
  const int smem = Ring<N, D, float>::BYTES * block;
  auto k = k_sweep<N, D, float, float>;
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

cudaError_t launch_sweep_mixed(int N, int D, const SweepArgs& a, const Mat& m, int block,
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

template <int N>
static int bytesN(int D) {
  if (D == 1) return Ring<N, 1, float>::BYTES;
  if (D == 2) return Ring<N, 2, float>::BYTES;
  return Ring<N, 3, float>::BYTES;
}

int sweep_smem_bytes_mixed(int N, int D) {
  switch (N) {
    case 1: return bytesN<1>(D);
    case 2: return bytesN<2>(D);
    case 3: return bytesN<3>(D);
    case 4: return bytesN<4>(D);
    case 5: return bytesN<5>(D);
  }
  return 0;
}

}  // namespace wc
