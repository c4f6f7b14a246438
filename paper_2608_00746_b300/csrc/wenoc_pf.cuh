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

// The face neighbours of cell i (32-bit indices: the host requires ncell <
// 2^31): nb[ax][0] below and nb[ax][1] above along each used axis, -1 where a
// reflective or outflow side mirrors the cell onto itself (no face).
__device__ __forceinline__ void pf_stencil(const PfGeom& g, int i, int (&nb)[3][2]) {
  const unsigned ui = (unsigned)i, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
  const unsigned x = ui % nx, r = ui / nx;
  nb[0][0] = x > 0u ? i - 1 : (g.per[0] ? i + g.nx - 1 : -1);
  nb[0][1] = x + 1u < nx ? i + 1 : (g.per[0] ? i - (g.nx - 1) : -1);
  if (g.dim > 1) {
    const unsigned y = r % ny;
    const int sy = g.nx;
    nb[1][0] = y > 0u ? i - sy : (g.per[1] ? i + (g.ny - 1) * sy : -1);
    nb[1][1] = y + 1u < ny ? i + sy : (g.per[1] ? i - (g.ny - 1) * sy : -1);
  }
  if (g.dim > 2) {
    const unsigned z = r / ny;
    const int sz = g.nx * g.ny;
    nb[2][0] = z > 0u ? i - sz : (g.per[2] ? i + (g.nz - 1) * sz : -1);
    nb[2][1] = z + 1u < (unsigned)g.nz ? i + sz : (g.per[2] ? i - (g.nz - 1) * sz : -1);
  }
}

// Scratch of the mechanism, [N][ncell] each unless noted.
struct PfWork {
  double* R;        // [div J_p]^ (Eq. 28)
  double* c;        // max(phi (1 - phi), 0)
  double* w;        // face weights c_f / dx^2 of the face above, [3][N][ncell]
  double* D;        // coupling sum_faces c_f / dx^2
  double* Dinv;     // 1 / D, 0 where D = 0 (cells without a coupled face)
  int* lab;         // region label (smallest cell index of the region), -1: none
  double* sumR;     // per region (indexed by label): sum r
  double* sumD;     //                                 sum D
  double* x;        // Q on the grid (the conjugate gradients' start and result)
  double* r;        // conjugate gradients on the listed unknowns: residual,
  double* p;        //   u = r/D (read by the neighbours),
  double* q;        //   K u,
  double* xk;       //   iterate (position k of phase p at p ncell + k),
  double* pd;       //   direction and
  double* sd;       //   its product (the in-memory iteration)
  int* idx;         // the list: cell of unknown k of phase p
  int* pos;         // its inverse: position of cell i, -1 off the list
  double* part;     // reduction partials (offsets in wenoc_pf.cu)
  double* scal;     // [64]: M, B[0..N-1] | b.b/D at 16+p | r.r/D at 24+p
  int* flag;        // [64]: converged per phase at 1+p, grid barrier at
                    //       8..10 (arrivals, generation, error), iterations at 11,
                    //       unknowns per phase at 12+p, unknowns a thread keeps in
                    //       registers at 17 (0: the lists in memory), the
                    //       in-memory iteration deferred to its own launch at 18,
                    //       labelling: change words 20..22, rounds 23, error 24
};

// Launchers (wenoc_pf.cu), all asynchronous on st.
size_t pf_part_doubles();
// Eq. 28 into w.R (M into w.scal[0], B into w.scal[1..N]); M_in >= 0 fixes M.
cudaError_t pf_cac(const double* U, const PfGeom& g, const PfWork& w, double vol, double eta,
                   double M_in, cudaStream_t st);
// Eq. 4: coefficients, coupling D, 1/D and initial labels.
cudaError_t pf_qmap_setup(const double* U, const PfGeom& g, const PfWork& w, cudaStream_t st);
// The list of unknowns, region labels (rounds until one changes nothing:
// w.flag[23] rounds, w.flag[24] != 0 if they did not settle), region sums,
// the consistent right-hand side b from R, and conjugate gradients on the
// listed unknowns to r.r/D <= tol2 b.b/D per phase or maxit iterations, from
// 0 or (warm) the values in w.x; the result in w.x.
// One cooperative launch (one block per SM, grid barriers with bounded
// waits: w.flag[10] != 0 afterwards if a wait gave up), and for a band
// larger than the registers take a second one after reading w.flag[18]
// (this synchronizes st); w.flag[1 + p] set for the converged phases,
// w.flag[11] the iterations, w.scal[24 + p] the last r.r/D and
// w.scal[16 + p] the reference b.b/D.
cudaError_t pf_qmap_solve(const PfGeom& g, const PfWork& w, int warm, double tol2, int maxit,
                          cudaStream_t st);
// The Q-map's grid barrier on its own (words: 4 device ints, cleared here):
// rounds barriers of one block per SM; block skip >= 0 never arrives, so
// the others' waits run out and words[2] becomes nonzero.
cudaError_t pf_barrier_check(int* words, int skip, int rounds, cudaStream_t st);
// The preconditioner's neighbour barrier alone: words of pf_nbr_check_words()
// ints (0 if the device cannot be queried; cleared here), the error at [2].
size_t pf_nbr_check_words();
cudaError_t pf_nbr_check(int* words, int skip, int span, int rounds, cudaStream_t st);

}  // namespace wc
