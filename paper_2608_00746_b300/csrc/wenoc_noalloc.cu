// wenoc_noalloc.cu -- SSP-RK3 stepping that allocates no device memory.
//
// Some callers cannot allocate device memory themselves: a host program whose
// device memory is owned and budgeted by another component, or code that runs
// where an allocation would synchronise or is forbidden.  wc_rk_step needs a
// workspace of three state-sized buffers; this entry point instead takes them
// from a fixed scratch array compiled into the library.  Every GPU that loads
// the library holds the array (kScratchBytes + 256 bytes) until the process
// exits.
#include <cstring>
#include <mutex>

#include "../../include/wenoc.h"
#include "wenoc_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)24 << 20;  // three stage-size buffers
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is a host-side stand-in, not a
// device address: host code must use the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes + 256];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];

// Looks up (once per device, with that device current) the device address
// of the scratch array.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

wc_status wc_internal_rk_with_scratch(wc_grid* g, double* U, char* scratch, double cfl,
                                      double dt_fixed, int nsteps, cudaStream_t st,
                                      unsigned** status_out);
void wc_internal_set_error(wc_grid* g, const char* msg);
wc_status wc_internal_scratch_supported(wc_grid* g);

extern "C" wc_status wc_rk_step_noalloc(wc_grid* g, double* U_dev, double cfl, double dt_fixed,
                                        int nsteps, int* status_host, void* stream) {
  if (!g || !U_dev || nsteps < 0) return WC_ERR_ARG;
  if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return WC_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(U_dev) & 7) return WC_ERR_ARG;
  // precisions the scratch cannot serve are refused before its size is
  const wc_status sup = wc_internal_scratch_supported(g);
  if (sup != WC_OK) return sup;
  size_t state = (size_t)wc_nvar(g) * (size_t)wc_ncell(g) * sizeof(double);
  state = (state + 255) / 256 * 256;
  if (3 * state > kScratchBytes) {
    wc_internal_set_error(g, "grid too large for the fixed 24 MiB scratch of wc_rk_step_noalloc "
                             "(needs 3 x NV x ncell x 8 bytes); use wc_rk_step with a workspace");
    return WC_ERR_ARG;
  }
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return WC_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned* status = nullptr;
  wc_status r = wc_internal_rk_with_scratch(g, U_dev, static_cast<char*>(base), cfl, dt_fixed,
                                            nsteps, st, &status);
  if (r != WC_OK) return r;
  if (status_host) {
    unsigned s = 0;
    cudaError_t e = cudaMemcpyAsync(&s, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return WC_ERR_CUDA;
    *status_host = (int)s;
  }
  return WC_OK;
}
