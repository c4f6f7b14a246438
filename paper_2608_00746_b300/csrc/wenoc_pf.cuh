// wenoc_pf.cuh -- the Phase-Field mechanism of one time step on the device
// (Sec. 2.2): the conservative Allen-Cahn divergence [div J_p]^ of Eq. 28
// from the fractions of the hyperbolic result, and the auxiliary fields Q_p
// of Eq. 4 (degenerate elliptic, one per phase, solved together).
//
// Readings (R17): eta = dx, M = 0.5 eta max|u|; second-order central
// Laplacian with mirrored cells at reflective/outflow sides; midpoint-rule
// integrals; the singular N x N system of Eq. 28 solved with B = 0 for
// absent phases and for the last present one (its equation dropped).  Eq. 4:
// face coefficient c_f = (c_a + c_b)/2, c = max(phi(1 - phi), 0); on each
// region that faces with c_f > 0 connect, the part D_i s_k (D_i = sum_faces
// c_f/dx^2, s_k = sum r / sum D over the region) is removed from the
// right-hand side, which makes the region's system consistent; it is solved
// by conjugate gradients preconditioned with D.  Only the face gradients on
// coupled faces are used (the Phase-Field flux takes G = 0 elsewhere).
#pragma once
#include <cuda_runtime.h>

#include "wenoc_device.cuh"

namespace wc {

// Fixed reduction grid: partial sums per block in a fixed order, summed in a
// fixed order, so every reduction is reproducible run to run.
constexpr int PF_BLOCKS = 148 * 4;
constexpr int PF_THREADS = 256;

struct PfGeom {
  int nx, ny, nz, dim;
  int per[3];        // periodic axis
  double idx2[3];    // 1/dx^2 per axis
  long ncell;
  int N, nv, a0;     // phases, variables, row of alpha_1
};

// Neighbour of cell i along axis ax in direction s (+1 / -1), or -1 where a
// reflective or outflow side mirrors the cell onto itself (no face).
__device__ __forceinline__ long pf_nbr(const PfGeom& g, long i, int ax, int s) {
  const long sx = 1, sy = g.nx, sz = (long)g.nx * g.ny;
  if (ax == 0) {
    const int x = (int)(i % g.nx);
    const int xn = x + s;
    if (xn < 0) return g.per[0] ? i + (g.nx - 1) * sx : -1;
    if (xn >= g.nx) return g.per[0] ? i - (g.nx - 1) * sx : -1;
    return i + s * sx;
  }
  if (ax == 1) {
    const int y = (int)((i / g.nx) % g.ny);
    const int yn = y + s;
    if (yn < 0) return g.per[1] ? i + (long)(g.ny - 1) * sy : -1;
    if (yn >= g.ny) return g.per[1] ? i - (long)(g.ny - 1) * sy : -1;
    return i + s * sy;
  }
  const int z = (int)(i / sz);
  const int zn = z + s;
  if (zn < 0) return g.per[2] ? i + (long)(g.nz - 1) * sz : -1;
  if (zn >= g.nz) return g.per[2] ? i - (long)(g.nz - 1) * sz : -1;
  return i + s * sz;
}

// Scratch of the mechanism, [N][ncell] each unless noted.
struct PfWork {
  double* R;        // [div J_p]^ (Eq. 28)
  double* c;        // max(phi (1 - phi), 0)
  double* D;        // coupling sum_faces c_f / dx^2
  int* lab;         // region label (smallest cell index of the region), -1: none
  double* sumR;     // per region (indexed by label): sum r
  double* sumD;     //                                 sum D
  double* r;        // conjugate-gradient residual
  double* z;        //                    preconditioned residual
  double* p;        //                    direction
  double* q;        //                    K p
  double* part;     // reduction partials [PF_BLOCKS][32] + [2][PF_BLOCKS][N] + [PF_BLOCKS][N]
  double* scal;     // [32]: M, B[0..N-1], rz0[N] ...
  int* flag;        // [8]: label change, converged per phase
};

// Launchers (wenoc_pf.cu), all asynchronous on st.
size_t pf_part_doubles();
// Eq. 28 into w.R (M into w.scal[0], B into w.scal[1..N]); M_in >= 0 fixes M.
cudaError_t pf_cac(const double* U, const PfGeom& g, const PfWork& w, double vol, double eta,
                   double M_in, cudaStream_t st);
// Eq. 4: coefficients, coupling D and initial labels.
cudaError_t pf_qmap_setup(const double* U, const PfGeom& g, const PfWork& w, cudaStream_t st);
// rounds of label propagation; w.flag[0] != 0 afterwards if any label moved.
cudaError_t pf_label_rounds(const PfGeom& g, const PfWork& w, int rounds, cudaStream_t st);
// region sums, the consistent right-hand side from R, and the CG start (Q = 0).
cudaError_t pf_qmap_project(const PfGeom& g, const PfWork& w, double* Q, cudaStream_t st);
// CG iterations it0 .. it0 + rounds - 1; w.flag[1 + p] set when phase p
// reached rz <= tol2 rz0; w.scal[24 + p] holds the last rz, w.scal[16 + p] rz0.
cudaError_t pf_cg_rounds(const PfGeom& g, const PfWork& w, double* Q, int it0, int rounds,
                         double tol2, cudaStream_t st);

}  // namespace wc
