// wenoc_pf.cu -- kernels of the Phase-Field mechanism (Eq. 28 and Eq. 4,
// readings in wenoc_pf.cuh).  All memory-bound stencil and reduction passes
// over [N][ncell] fields; grid-stride loops on a fixed grid of PF_BLOCKS
// blocks so that every reduction has one fixed order.
#include "wenoc_pf.cuh"

namespace wc {

// ------------------------------------------------------------------ helpers
template <int K>
__device__ __forceinline__ void block_sum_to(double (&v)[K], double* out) {
  // fixed-order block reduction: warp trees, then warps in order
  __shared__ double sm[PF_THREADS / 32][K > 0 ? K : 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sm[w][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int j = 0; j < PF_THREADS / 32; j++) s += sm[j][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double sm[PF_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int j = 0; j < PF_THREADS / 32; j++) m = fmax(m, sm[j]);
  __syncthreads();
  return m;
}

__device__ __forceinline__ double gprime(double f) { return 2.0 * f * (1.0 - f) * (1.0 - 2.0 * f); }

template <int N>
struct CacLayout {
  static constexpr int NW = N * (N + 1) / 2;  // W_pq, p <= q
  static constexpr int K = NW + N;           // + sums of g'_p - phi_p sum g'
};

// ------------------------------------------------------------------ Eq. 28
// Pass 1: per block, max |u|^2 and the sums of W_pq (p <= q) and of
// g'(phi_p) - phi_p sum_q g'(phi_q) over its cells.
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_cac_reduce(const double* __restrict__ U,
                                                           PfGeom g, double* part) {
  using L = CacLayout<N>;
  double acc[L::K];
#pragma unroll
  for (int k = 0; k < L::K; k++) acc[k] = 0.0;
  double umax = 0.0;
  const long n = g.ncell;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    double rho = 0.0;
#pragma unroll
    for (int p = 0; p < N; p++) rho += U[(long)p * n + i];
    double u2 = 0.0;
#pragma unroll
    for (int j = 0; j < 3; j++) {
      if (j >= g.dim) break;
      const double u = U[(long)(N + j) * n + i] / rho;
      u2 += u * u;
    }
    umax = fmax(umax, u2);
    double phi[N], gp[N], sg = 0.0;
#pragma unroll
    for (int p = 0; p < N; p++) {
      phi[p] = U[(long)(g.a0 + p) * n + i];
      gp[p] = gprime(phi[p]);
      sg += gp[p];
    }
    int k = 0;
#pragma unroll
    for (int p = 0; p < N; p++) {
#pragma unroll
      for (int q = p; q < N; q++) acc[k++] += p == q ? phi[p] * (1.0 - phi[p]) : -phi[p] * phi[q];
    }
#pragma unroll
    for (int p = 0; p < N; p++) acc[L::NW + p] += gp[p] - phi[p] * sg;
  }
  double* out = part + (long)blockIdx.x * 32;
  block_sum_to<L::K>(acc, out);
  const double m = block_max(umax);
  if (threadIdx.x == 0) out[31] = m;
}

// Pass 2 (one block): totals, M, the N x N system and its solution B.
template <int N>
__global__ void k_cac_solve(const double* part, double vol, double eta, double M_in, double* scal) {
  using L = CacLayout<N>;
  __shared__ double tot[32];
  const int t = threadIdx.x;
  if (t < L::K) {
    double s = 0.0;
    for (int b = 0; b < PF_BLOCKS; b++) s += part[(long)b * 32 + t];
    tot[t] = s;
  } else if (t == 31) {
    double m = 0.0;
    for (int b = 0; b < PF_BLOCKS; b++) m = fmax(m, part[(long)b * 32 + 31]);
    tot[31] = m;
  }
  __syncthreads();
  if (t != 0) return;
  const double M = M_in >= 0.0 ? M_in : 0.5 * eta * sqrt(tot[31]);
  double W[N][N], b[N], B[N];
  int k = 0;
  for (int p = 0; p < N; p++)
    for (int q = p; q < N; q++) {
      W[p][q] = W[q][p] = tot[k++] * vol;
    }
  for (int p = 0; p < N; p++) {
    b[p] = (M / (eta * eta)) * tot[L::NW + p] * vol;
    B[p] = 0.0;
  }
  // present phases (int W_pp > 0); the last one keeps B = 0, its equation
  // (implied by the others) is dropped
  int keep[N], m = 0;
  for (int p = 0; p < N; p++)
    if (W[p][p] > 0.0) keep[m++] = p;
  m -= 1;
  if (m >= 1) {
    double A[N][N + 1];
    for (int i = 0; i < m; i++) {
      for (int j = 0; j < m; j++) A[i][j] = W[keep[i]][keep[j]];
      A[i][m] = b[keep[i]];
    }
    // Gaussian elimination with partial pivoting
    for (int c = 0; c < m; c++) {
      int piv = c;
      for (int i = c + 1; i < m; i++)
        if (fabs(A[i][c]) > fabs(A[piv][c])) piv = i;
      if (piv != c)
        for (int j = c; j <= m; j++) {
          const double tmp = A[c][j];
          A[c][j] = A[piv][j];
          A[piv][j] = tmp;
        }
      for (int i = c + 1; i < m; i++) {
        const double f = A[i][c] / A[c][c];
        for (int j = c; j <= m; j++) A[i][j] -= f * A[c][j];
      }
    }
    for (int i = m - 1; i >= 0; i--) {
      double s = A[i][m];
      for (int j = i + 1; j < m; j++) s -= A[i][j] * B[keep[j]];
      B[keep[i]] = s / A[i][i];
    }
  }
  scal[0] = M;
  for (int p = 0; p < N; p++) scal[1 + p] = B[p];
}

// Pass 3: [div J_p]^ = M lap(phi_p) - (M/eta^2)(g'_p - phi_p sum g') + L^c_p.
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_cac_rhs(const double* __restrict__ U, PfGeom g,
                                                        const double* scal, double eta,
                                                        double* __restrict__ R) {
  const long n = g.ncell;
  const double M = scal[0];
  double B[N];
#pragma unroll
  for (int p = 0; p < N; p++) B[p] = scal[1 + p];
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    double phi[N], gp[N], sg = 0.0;
#pragma unroll
    for (int p = 0; p < N; p++) {
      phi[p] = U[(long)(g.a0 + p) * n + i];
      gp[p] = gprime(phi[p]);
      sg += gp[p];
    }
    int nb[3][2];
    pf_stencil(g, (int)i, nb);
#pragma unroll
    for (int p = 0; p < N; p++) {
      const double* f = U + (long)(g.a0 + p) * n;
      double lap = 0.0;
#pragma unroll
      for (int ax = 0; ax < 3; ax++) {
        if (ax >= g.dim) break;
        const double fm = nb[ax][0] >= 0 ? f[nb[ax][0]] : phi[p];
        const double fp = nb[ax][1] >= 0 ? f[nb[ax][1]] : phi[p];
        lap += (fp - 2.0 * phi[p] + fm) * g.idx2[ax];
      }
      const double S = (M / (eta * eta)) * (gp[p] - phi[p] * sg);
      double Lc = 0.0;
#pragma unroll
      for (int q = 0; q < N; q++) Lc += (p == q ? phi[p] * (1.0 - phi[q]) : -phi[p] * phi[q]) * B[q];
      R[(long)p * n + i] = M * lap - S + Lc;
    }
  }
}

// ------------------------------------------------------------------ Eq. 4
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_qm_coef(const double* __restrict__ U, PfGeom g,
                                                        double* __restrict__ c) {
  const long n = g.ncell;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      const double f = U[(long)(g.a0 + p) * n + i];
      c[(long)p * n + i] = fmax(f * (1.0 - f), 0.0);
    }
  }
}

// Face weights w_ax = c_f / dx^2 of the face above each cell along each
// axis (0 where a reflective or outflow side ends the axis), the coupling
// D_i = sum_faces c_f / dx^2 (the same weights summed), 1/D (0 where D = 0)
// and the initial labels (own index where D > 0).
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_qm_diag(PfGeom g, const double* __restrict__ c,
                                                        double* __restrict__ w,
                                                        double* __restrict__ D,
                                                        double* __restrict__ Dinv, int* lab) {
  const int n = (int)g.ncell;
  const long nn = (long)N * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int nb[3][2];
    pf_stencil(g, i, nb);
#pragma unroll
    for (int p = 0; p < N; p++) {
      const double* cp = c + (long)p * n;
      const double ci = cp[i];
      double d = 0.0;
#pragma unroll
      for (int ax = 0; ax < 3; ax++) {
        if (ax >= g.dim) break;
        const int jm = nb[ax][0], jp = nb[ax][1];
        const double wm = jm >= 0 ? 0.5 * (cp[jm] + ci) * g.idx2[ax] : 0.0;
        const double wp = jp >= 0 ? 0.5 * (ci + cp[jp]) * g.idx2[ax] : 0.0;
        w[ax * nn + (long)p * n + i] = wp;
        d += wm + wp;
      }
      D[(long)p * n + i] = d;
      Dinv[(long)p * n + i] = d > 0.0 ? 1.0 / d : 0.0;
      lab[(long)p * n + i] = d > 0.0 ? i : -1;
    }
  }
}

// (K v)_i = D_i v_i - sum_faces w_f v_nbr with K = -A (positive
// semi-definite), from the stored face weights.
template <int N>
__device__ __forceinline__ double k_apply(const PfGeom& g, const int (&nb)[3][2], int i, long o,
                                          long nn, const double* __restrict__ w,
                                          const double* __restrict__ D,
                                          const double* __restrict__ v) {
  double s = D[o + i] * v[o + i];
#pragma unroll
  for (int ax = 0; ax < 3; ax++) {
    if (ax >= g.dim) break;
    const double* wa = w + ax * nn + o;
    const int jm = nb[ax][0], jp = nb[ax][1];
    if (jp >= 0) s = fma(-wa[i], v[o + jp], s);
    if (jm >= 0) s = fma(-wa[jm], v[o + jm], s);
  }
  return s;
}

// One round of minimum-label propagation over coupled faces with pointer
// jumping.  Labels only decrease and always name a cell of the same region,
// so the rounds end (the host stops at a round without change) with every
// cell of a region labelled by the region's smallest cell index.
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_qm_label(PfGeom g, const double* __restrict__ c,
                                                         int* lab, int* flag) {
  const int n = (int)g.ncell;
  int changed = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int nb[3][2];
    pf_stencil(g, i, nb);
#pragma unroll
    for (int p = 0; p < N; p++) {
      int* lp = lab + (long)p * n;
      const int li = __ldcg(lp + i);
      if (li < 0) continue;
      const double* cp = c + (long)p * n;
      const double ci = cp[i];
      int m = li;
#pragma unroll
      for (int ax = 0; ax < 3; ax++) {
        if (ax >= g.dim) break;
#pragma unroll
        for (int s = 0; s < 2; s++) {
          const int j = nb[ax][s];
          if (j >= 0 && (ci > 0.0 || cp[j] > 0.0)) m = min(m, __ldcg(lp + j));
        }
      }
      m = min(m, __ldcg(lp + m));
      if (m < li) {
        atomicMin(lp + i, m);
        changed = 1;
      }
    }
  }
  if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(flag, 1);
}

template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_qm_sums(PfGeom g, const double* __restrict__ R,
                                                        const double* __restrict__ D,
                                                        const int* __restrict__ lab, double* sumR,
                                                        double* sumD) {
  const int n = (int)g.ncell;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      const int l = lab[(long)p * n + i];
      if (l < 0) continue;
      atomicAdd(sumR + (long)p * n + l, R[(long)p * n + i]);
      atomicAdd(sumD + (long)p * n + l, D[(long)p * n + i]);
    }
  }
}

// The conjugate-gradient kernels reduce over a fixed grid of PF_CG_BLOCKS
// blocks (8 per SM: the elementwise passes need many loads in flight).
// Partials: p . K p [PF_CG_BLOCKS][8]; r . r/D [2 parities][PF_CG_BLOCKS][8];
// b . b/D [PF_CG_BLOCKS][8], after the Eq. 28 totals [PF_BLOCKS][32].  The
// last block of a reducing kernel to finish (atomic ticket, no waiting)
// sums the partials in a fixed order and writes the scalars the next kernel
// reads: alpha after the matrix-vector pass, the convergence test and beta
// after the update.
constexpr int PF_CG_BLOCKS = 148 * 8;
constexpr long PART_CAC = 0;
constexpr long PART_PQ = (long)PF_BLOCKS * 32;
constexpr long PART_RZ = PART_PQ + (long)PF_CG_BLOCKS * 8;
constexpr long PART_REF = PART_RZ + 2L * PF_CG_BLOCKS * 8;
constexpr long PART_TOTAL = PART_REF + (long)PF_CG_BLOCKS * 8;
// scalars: scal[16 + p] b.b/D, [24 + p] r.r/D of the current iteration,
// [32 + p] beta, [40 + p] alpha; flags: [1 + p] converged, [6] and [7] the
// tickets of the matrix-vector and update passes (zero between launches)

// On B300 a warp's FP64 instruction occupies the FP64 pipe for the same time
// however few lanes are active, so the reductions here are written to issue
// few FP64 warp instructions.
//
// Block sum of N values per thread into out[0..N-1] (fixed order): a shared
// tree over the 256 threads down to one warp, then its shuffle tree.
template <int N>
__device__ __forceinline__ void block_sum_small(const double (&v)[N], double* out) {
  __shared__ double sm[N][PF_THREADS];
  const int t = threadIdx.x;
#pragma unroll
  for (int p = 0; p < N; p++) sm[p][t] = v[p];
  __syncthreads();
#pragma unroll
  for (int s = PF_THREADS / 2; s >= 32; s >>= 1) {
    if (t < s)
#pragma unroll
      for (int p = 0; p < N; p++) sm[p][t] += sm[p][t + s];
    __syncthreads();
  }
  if (t < 32) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      double x = sm[p][t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (t == 0) out[p] = x;
    }
  }
  __syncthreads();
}

// Sums of count per-block partial rows (8 doubles, N used) by the whole
// block, in a fixed order: thread t adds rows t, t + 256, ... (their loads
// in flight together), then block_sum_small; out[p] (shared) for every
// thread afterwards.
template <int N>
__device__ __forceinline__ void sum_partials_block(const double* part, long off, int count,
                                                   double* out) {
  constexpr int R = (PF_CG_BLOCKS + PF_THREADS - 1) / PF_THREADS;
  double t[R][N], v[N];
#pragma unroll
  for (int j = 0; j < R; j++) {
    const int b = threadIdx.x + PF_THREADS * j;
#pragma unroll
    for (int p = 0; p < N; p++) t[j][p] = b < count ? __ldcg(part + off + (long)b * 8 + p) : 0.0;
  }
#pragma unroll
  for (int p = 0; p < N; p++) {
    v[p] = 0.0;
#pragma unroll
    for (int j = 0; j < R; j++) v[p] += t[j][p];
  }
  block_sum_small<N>(v, out);
}

// True in the block that finishes last (after its partials are written);
// that block also resets the ticket for the next launch.
__device__ __forceinline__ bool last_block(int* ticket) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();
    const int t = atomicAdd(ticket, 1);
    last = t == (int)gridDim.x - 1;
    if (last) *ticket = 0;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// K Q = b with K = -A (positive semi-definite): b = -(r - D s_k) on cells
// with a label.  Start x0 = 0, or (warm) the x given; r0 = b - K x0.
// Partials of r0 . r0/D (parity 0) and of the reference b . b/D of the
// stopping test.
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_cg_init(PfGeom g, const double* __restrict__ R,
                                                        const double* __restrict__ w,
                                                        const double* __restrict__ D,
                                                        const double* __restrict__ Dinv,
                                                        const int* __restrict__ lab,
                                                        const double* __restrict__ sumR,
                                                        const double* __restrict__ sumD,
                                                        double* x, double* r, double* part,
                                                        int warm) {
  const int n = (int)g.ncell;
  const long nn = (long)N * n;
  double acc[N], ref[N];
#pragma unroll
  for (int p = 0; p < N; p++) acc[p] = ref[p] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int nb[3][2];
    pf_stencil(g, i, nb);
#pragma unroll
    for (int p = 0; p < N; p++) {
      const long o = (long)p * n, k = o + i;
      const int l = lab[k];
      double b = 0.0, rr = 0.0;
      if (l >= 0) {
        const double s = sumR[o + l] / sumD[o + l];
        b = -(R[k] - D[k] * s);
        rr = warm ? b - k_apply<N>(g, nb, i, o, nn, w, D, x) : b;
        ref[p] += b * (b * Dinv[k]);
      }
      r[k] = rr;
      acc[p] += rr * (rr * Dinv[k]);
    }
  }
  if (!warm) {
    // x0 = 0 (no block reads x when cold)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
      for (int p = 0; p < N; p++) x[(long)p * n + i] = 0.0;
  }
  block_sum_small<N>(acc, part + PART_RZ + (long)blockIdx.x * 8);  // parity 0
  block_sum_small<N>(ref, part + PART_REF + (long)blockIdx.x * 8);
}

// The reference b . b/D and r0 . r0/D per phase and tol^2 into scal (one
// warp); beta = 0 for the first directions; a phase whose start already
// meets the test is converged.
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_cg_start(const double* part, double* scal,
                                                         int* flag, double tol2) {
  __shared__ double rz[N], ref[N];
  sum_partials_block<N>(part, PART_RZ, PF_CG_BLOCKS, rz);
  sum_partials_block<N>(part, PART_REF, PF_CG_BLOCKS, ref);
  if (threadIdx.x != 0) return;
  scal[8] = tol2;
#pragma unroll
  for (int p = 0; p < N; p++) {
    scal[16 + p] = ref[p];
    scal[24 + p] = rz[p];
    scal[32 + p] = 0.0;
    flag[1 + p] = !(rz[p] > tol2 * ref[p]);
  }
}

__device__ __forceinline__ bool all_converged(const int* flag, int N) {
  int all = 1;
  for (int p = 0; p < N; p++) all &= flag[1 + p];
  return all;
}

// Step 1 (elementwise, any grid): p = r/D + beta p for the live phases
// (beta = 0 at the first iteration).
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_cg_dir(PfGeom g, const double* __restrict__ r,
                                                       const double* __restrict__ Dinv,
                                                       double* __restrict__ pv,
                                                       const double* __restrict__ scal,
                                                       const int* __restrict__ flag) {
  if (all_converged(flag, N)) return;
  const long n = g.ncell;
  for (int p = 0; p < N; p++) {
    if (flag[1 + p]) continue;
    const double beta = scal[32 + p];
    const long o = (long)p * n;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x)
      pv[o + i] = fma(beta, pv[o + i], r[o + i] * Dinv[o + i]);
  }
}

// Step 2: q = K p for the live phases and the partials of p . q; the last
// block forms alpha = r.r/D / p.q per live phase.
template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_cg_matvec(PfGeom g, const double* __restrict__ w,
                                                          const double* __restrict__ D,
                                                          const double* __restrict__ pv,
                                                          double* __restrict__ q, double* part,
                                                          double* scal, int* flag) {
  if (all_converged(flag, N)) return;
  bool live[N];
#pragma unroll
  for (int p = 0; p < N; p++) live[p] = !flag[1 + p];
  const int n = (int)g.ncell;
  const long nn = (long)N * n;
  double acc[N];
#pragma unroll
  for (int p = 0; p < N; p++) acc[p] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int nb[3][2];
    pf_stencil(g, i, nb);
#pragma unroll
    for (int p = 0; p < N; p++) {
      if (!live[p]) continue;
      const long o = (long)p * n;
      const double s = k_apply<N>(g, nb, i, o, nn, w, D, pv);
      q[o + i] = s;
      acc[p] = fma(pv[o + i], s, acc[p]);
    }
  }
  block_sum_small<N>(acc, part + PART_PQ + (long)blockIdx.x * 8);
  if (!last_block(flag + 6)) return;
  __shared__ double pq[N];
  sum_partials_block<N>(part, PART_PQ, (int)gridDim.x, pq);
  if (threadIdx.x == 0)
#pragma unroll
    for (int p = 0; p < N; p++)
      scal[40 + p] = (live[p] && pq[p] > 0.0) ? scal[24 + p] / pq[p] : 0.0;
}

// Step 3 (iteration it): x += alpha p, r -= alpha q for the live phases;
// partials of r . r/D into parity (it + 1) & 1 for every phase.  The last
// block sums them and sets, for the next iteration, r.r/D, the test
// (converged: r.r/D <= tol^2 b.b/D) and beta = new r.r/D / old.
template <int N>
__global__ void __launch_bounds__(PF_THREADS, 8) k_cg_update(PfGeom g,
                                                          const double* __restrict__ Dinv,
                                                          double* __restrict__ x,
                                                          double* __restrict__ r,
                                                          const double* __restrict__ pv,
                                                          const double* __restrict__ q,
                                                          double* part, double* scal, int* flag,
                                                          int it) {
  if (all_converged(flag, N)) return;
  bool live[N];
  double alpha[N];
#pragma unroll
  for (int p = 0; p < N; p++) {
    live[p] = !flag[1 + p];
    alpha[p] = scal[40 + p];
  }
  const int n = (int)g.ncell;
  double acc[N];
#pragma unroll
  for (int p = 0; p < N; p++) acc[p] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      const long k = (long)p * n + i;
      double rk = r[k];
      if (live[p]) {
        x[k] = fma(alpha[p], pv[k], x[k]);
        rk = fma(-alpha[p], q[k], rk);
        r[k] = rk;
      }
      acc[p] = fma(rk, rk * Dinv[k], acc[p]);
    }
  }
  const long onew = PART_RZ + (long)((it + 1) & 1) * PF_CG_BLOCKS * 8;
  block_sum_small<N>(acc, part + onew + (long)blockIdx.x * 8);
  if (!last_block(flag + 7)) return;
  __shared__ double rn[N];
  sum_partials_block<N>(part, onew, (int)gridDim.x, rn);
  if (threadIdx.x == 0) {
    const double tol2 = scal[8];
#pragma unroll
    for (int p = 0; p < N; p++) {
      const double ro = scal[24 + p];
      const bool conv = !(rn[p] > tol2 * scal[16 + p]);
      scal[32 + p] = ro > 0.0 ? rn[p] / ro : 0.0;
      scal[24 + p] = rn[p];
      // a phase that no longer moves (alpha = 0) stays where it is
      flag[1 + p] = flag[1 + p] || conv || !(scal[40 + p] > 0.0);
    }
  }
}

// ------------------------------------------------------------------ launchers
#define PF_DISPATCH(N, call)                       \
  switch (N) {                                     \
    case 1: { constexpr int N_ = 1; call; break; } \
    case 2: { constexpr int N_ = 2; call; break; } \
    case 3: { constexpr int N_ = 3; call; break; } \
    case 4: { constexpr int N_ = 4; call; break; } \
    case 5: { constexpr int N_ = 5; call; break; } \
    default: return cudaErrorInvalidValue;         \
  }

static int pf_grid(long n) {
  long b = (n + PF_THREADS - 1) / PF_THREADS;
  return (int)(b < PF_BLOCKS ? (b < 1 ? 1 : b) : PF_BLOCKS);
}

size_t pf_part_doubles() { return (size_t)PART_TOTAL; }

cudaError_t pf_cac(const double* U, const PfGeom& g, const PfWork& w, double vol, double eta,
                   double M_in, cudaStream_t st) {
  PF_DISPATCH(g.N, (k_cac_reduce<N_><<<PF_BLOCKS, PF_THREADS, 0, st>>>(U, g, w.part + PART_CAC)));
  PF_DISPATCH(g.N, (k_cac_solve<N_><<<1, 32, 0, st>>>(w.part + PART_CAC, vol, eta, M_in, w.scal)));
  PF_DISPATCH(g.N, (k_cac_rhs<N_><<<pf_grid(g.ncell), PF_THREADS, 0, st>>>(U, g, w.scal, eta, w.R)));
  return cudaGetLastError();
}

cudaError_t pf_qmap_setup(const double* U, const PfGeom& g, const PfWork& w, cudaStream_t st) {
  const int nb = pf_grid(g.ncell);
  PF_DISPATCH(g.N, (k_qm_coef<N_><<<nb, PF_THREADS, 0, st>>>(U, g, w.c)));
  PF_DISPATCH(g.N, (k_qm_diag<N_><<<nb, PF_THREADS, 0, st>>>(g, w.c, w.w, w.D, w.Dinv, w.lab)));
  return cudaGetLastError();
}

cudaError_t pf_label_rounds(const PfGeom& g, const PfWork& w, int rounds, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(w.flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int nb = pf_grid(g.ncell);
  for (int k = 0; k < rounds; k++)
    PF_DISPATCH(g.N, (k_qm_label<N_><<<nb, PF_THREADS, 0, st>>>(g, w.c, w.lab, w.flag)));
  return cudaGetLastError();
}

cudaError_t pf_qmap_project(const PfGeom& g, const PfWork& w, int warm, double tol2,
                            cudaStream_t st) {
  const size_t bytes = sizeof(double) * (size_t)g.N * g.ncell;
  cudaError_t e = cudaMemsetAsync(w.sumR, 0, bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.sumD, 0, bytes, st);
  if (e != cudaSuccess) return e;
  const int nb = pf_grid(g.ncell);
  PF_DISPATCH(g.N, (k_qm_sums<N_><<<nb, PF_THREADS, 0, st>>>(g, w.R, w.D, w.lab, w.sumR, w.sumD)));
  PF_DISPATCH(g.N, (k_cg_init<N_><<<PF_CG_BLOCKS, PF_THREADS, 0, st>>>(
                        g, w.R, w.w, w.D, w.Dinv, w.lab, w.sumR, w.sumD, w.x, w.r, w.part, warm)));
  PF_DISPATCH(g.N, (k_cg_start<N_><<<1, PF_THREADS, 0, st>>>(w.part, w.scal, w.flag, tol2)));
  return cudaGetLastError();
}

// Blocks of the matrix-vector pass: one wave of as many blocks as fit on
// the SMs (queried once per phase count), fewer on a small grid.
cudaError_t pf_cg_matvec_blocks(const PfGeom& g, int* blocks) {
  static int mv_per_sm[8] = {0};
  int& mps = mv_per_sm[g.N];
  if (mps == 0) {
    int k = 0;
    cudaError_t e = cudaSuccess;
    PF_DISPATCH(g.N, (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_cg_matvec<N_>,
                                                                       PF_THREADS, 0)));
    if (e != cudaSuccess) return e;
    mps = k < 1 ? 1 : (k > 8 ? 8 : k);
  }
  const long eb = (g.ncell + PF_THREADS - 1) / PF_THREADS;
  *blocks = (int)(eb < 148L * mps ? (eb < 1 ? 1 : eb) : 148L * mps);
  return *blocks > PF_CG_BLOCKS ? cudaErrorInvalidValue : cudaSuccess;  // partial rows
}

cudaError_t pf_cg_rounds(const PfGeom& g, const PfWork& w, int it0, int rounds, cudaStream_t st) {
  const long eb = (g.ncell + PF_THREADS - 1) / PF_THREADS;
  const int dir_blocks = (int)(eb < 148 * 16 ? (eb < 1 ? 1 : eb) : 148 * 16);
  // the update pass: PF_CG_BLOCKS blocks, fewer on a small grid (its last
  // block sums one partial per block launched)
  const int up_blocks = (int)(eb < PF_CG_BLOCKS ? (eb < 1 ? 1 : eb) : PF_CG_BLOCKS);
  int mv_blocks = 0;
  cudaError_t e = pf_cg_matvec_blocks(g, &mv_blocks);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < rounds; k++) {
    const int it = it0 + k;
    PF_DISPATCH(g.N, (k_cg_dir<N_><<<dir_blocks, PF_THREADS, 0, st>>>(g, w.r, w.Dinv, w.p,
                                                                       w.scal, w.flag)));
    PF_DISPATCH(g.N, (k_cg_matvec<N_><<<mv_blocks, PF_THREADS, 0, st>>>(
                          g, w.w, w.D, w.p, w.q, w.part, w.scal, w.flag)));
    PF_DISPATCH(g.N, (k_cg_update<N_><<<up_blocks, PF_THREADS, 0, st>>>(
                          g, w.Dinv, w.x, w.r, w.p, w.q, w.part, w.scal, w.flag, it)));
  }
  return cudaGetLastError();
}

// The launches of pf_cg_rounds(g, w, 0, rounds) recorded on `cap` (a stream
// of the caller's, not the legacy default stream) as one executable graph:
// replayed on any stream, it runs `rounds` iterations from any even
// iteration count (the kernels read the iteration only for the parity of
// the reduction buffer).  It holds the pointers of w and the geometry g.
cudaError_t pf_cg_graph(const PfGeom& g, const PfWork& w, int rounds, cudaStream_t cap,
                        cudaGraphExec_t* exec) {
  if (rounds % 2 != 0) return cudaErrorInvalidValue;
  int mv_blocks = 0;
  cudaError_t e = pf_cg_matvec_blocks(g, &mv_blocks);  // the query stays out of the capture
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t el = pf_cg_rounds(g, w, 0, rounds, cap);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  if (el != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return el != cudaSuccess ? el : e;
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

}  // namespace wc
