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
__global__ void __launch_bounds__(PF_THREADS) k_cac_solve(const double* part, double vol,
                                                          double eta, double M_in, double* scal) {
  using L = CacLayout<N>;
  __shared__ double red[32][PF_THREADS / 32], tot[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  // the PF_BLOCKS partial rows summed in a fixed order: rows t, t + 256, ...
  // by thread t, then a shuffle tree in each warp and the eight warp sums
  // (value 31 is a maximum)
  for (int j = 0; j < 32; j++) {
    if (j >= L::K && j != 31) continue;
    const bool mx = j == 31;
    double s = 0.0;
    for (int r = t; r < PF_BLOCKS; r += PF_THREADS) {
      const double v = part[(long)r * 32 + j];
      s = mx ? fmax(s, v) : s + v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, s, o);
      s = mx ? fmax(s, y) : s + y;
    }
    if (lane == 0) red[j][wid] = s;
  }
  __syncthreads();
  if (t < 32 && (t < L::K || t == 31)) {
    double s = red[t][0];
    for (int k = 1; k < PF_THREADS / 32; k++) s = t == 31 ? fmax(s, red[t][k]) : s + red[t][k];
    tot[t] = s;
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
      c[(long)p * n + i] = pf_active(f) ? f * (1.0 - f) : 0.0;
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


// The conjugate gradients of Eq. 4 run on the listed unknowns (the cells of
// some region, in cell order per phase) in one cooperative launch of at
// most PF_CG_BLOCKS blocks that meet at grid barriers.  Partials: the Eq. 28
// totals [PF_BLOCKS][32], the list counts [PF_CG_BLOCKS][8] and the
// iteration's sums [PF_CG_BLOCKS][PART_ROW] (up to four per phase).  Every
// block sums the partials itself, in the same fixed order, so all blocks
// hold the same scalars and take the same loop decisions.
constexpr int PF_CG_BLOCKS = 148 * 8;
constexpr int PART_ROW = 32;
constexpr long PART_CAC = 0;
constexpr long PART_LIST = (long)PF_BLOCKS * 32;
constexpr long PART_CG1 = PART_LIST + (long)PF_CG_BLOCKS * 8;
// the neighbour flags of the preconditioner's exchanges: one 32-byte word a block
constexpr long PART_NBR = PART_CG1 + (long)PF_CG_BLOCKS * PART_ROW;
constexpr long PART_TOTAL = PART_NBR + (long)PF_CG_BLOCKS * 4;
// results: scal[16 + p] b.b/D, [24 + p] r.r/D; flags: [1 + p] converged,
// [8] [9] [10] the grid barrier (arrivals, generation, error), [11] the
// iterations done

// On B300 a warp's FP64 instruction occupies the FP64 pipe for the same time
// however few lanes are active, so the reductions here are written to issue
// few FP64 warp instructions.
//
// Block sum of N values per thread into out[0..N-1] (fixed order).  In each
// warp a reduce-scatter: with the values padded to P = 2^k >= N, the lanes
// whose bit 16 is set keep the upper half, the others the lower half, each
// adding its partner's copy; then bit 8 halves again, and so on until a
// lane holds one value, which the remaining offsets sum as a butterfly.
// That is P - 1 + 5 - k FP64 adds a warp instead of 5 N (a warp's FP64
// instruction costs the same however few lanes it uses).  Lane v 32/P then
// holds the warp's sum of value v; warp 0 adds the eight warp sums.  out is
// written by thread 0 and read by the block after the closing barrier.
template <int N, int BT = PF_THREADS>
__device__ __forceinline__ void block_sum_small(const double (&v)[N], double* out,
                                                bool warp_zero = false) {
  constexpr int W = BT / 32;
  constexpr int P = N <= 1 ? 1 : (N <= 2 ? 2 : (N <= 4 ? 4 : (N <= 8 ? 8 : 16)));
  __shared__ double sm[N][W];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  // (warp_zero: the caller knows every value of this warp is +0; its sums
  // are +0 without the shuffles)
  if (warp_zero) {
    if (lane < N) sm[lane][wid] = 0.0;
  } else {
    double x[P];
#pragma unroll
    for (int j = 0; j < P; j++) x[j] = j < N ? v[j] : 0.0;
    int idx = 0;  // index of the first value this lane keeps
#pragma unroll
    for (int c = P, o = 16; c > 1; c >>= 1, o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < c / 2; i++) {
        const double mine = up ? x[c / 2 + i] : x[i];
        const double other = up ? x[i] : x[c / 2 + i];
        x[i] = mine + __shfl_xor_sync(0xffffffffu, other, o);
      }
      if (up) idx += c / 2;
    }
#pragma unroll
    for (int o = 16 / P; o > 0; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
    if (lane % (32 / P) == 0 && idx < N) sm[idx][wid] = x[0];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      double y = lane < W ? sm[p][lane] : 0.0;
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
      if (lane == 0) out[p] = y;
    }
  }
  __syncthreads();
}

// Grid barrier of the cooperative launch (every block resident): an arrival
// count and a generation word.  The last block to arrive resets the count
// and advances the generation; the others poll the generation, at most
// PF_SPIN_LIMIT times, and stop waiting when any block has set the error
// word (a timed-out wait sets it).  Returns false after an error: the
// caller leaves its iterations, and the host reports WC_ERR_TIMEOUT.
constexpr unsigned PF_SPIN_LIMIT = 1u << 22;
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // release of this block's writes with the arrival, acquire of the
    // others' with the generation (PTX memory model, gpu scope)
    volatile int* verr = err;
    unsigned g0, arrived;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(g0) : "l"(bar + 1) : "memory");
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      asm volatile("red.release.gpu.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
    } else {
      unsigned spins = 0;
      for (;;) {
        unsigned gv;
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(gv) : "l"(bar + 1) : "memory");
        if (gv != g0) break;
        if ((spins & 255u) == 0u && *verr) break;
        if (++spins > PF_SPIN_LIMIT) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    ok = *verr == 0;
  }
  __syncthreads();
  return ok;
}

// A barrier among neighbouring blocks only: this block publishes `epoch` in
// its flag (flags[8 b], one 32-byte word a block; release after the block's
// writes), then waits until every block of [lo, hi] has published it
// (acquire; bounded polls, the error word stops every waiter).  Used for the
// exchanges of the preconditioner, where a block reads the entries of the
// blocks that own its unknowns' neighbours: the coupling is symmetric, so
// the blocks it waits for are also the only ones that read its entries, and
// an entry is rewritten (two exchanges later, in the other buffer's turn)
// only after they have all published the exchange in between, that is,
// after they have read it.  Every block publishes every epoch.  Returns
// false after an error, as grid_sync.
__device__ __forceinline__ bool nbr_sync(unsigned* flags, int lo, int hi, unsigned epoch,
                                         int* err) {
  __shared__ int bad;
  __syncthreads();
  if (threadIdx.x == 0) {
    bad = 0;
    asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(flags + 8 * blockIdx.x), "r"(epoch)
                 : "memory");
  }
  __syncthreads();
  for (int q = lo + (int)threadIdx.x; q <= hi; q += (int)blockDim.x) {
    if (q == (int)blockIdx.x) continue;
    volatile int* verr = err;
    unsigned spins = 0;
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(flags + 8 * q) : "memory");
      if (v >= epoch) break;
      if ((spins & 255u) == 0u && *verr) {
        bad = 1;
        break;
      }
      if (++spins > PF_SPIN_LIMIT) {
        atomicExch(err, 1);
        bad = 1;
        break;
      }
    }
  }
  __syncthreads();
  return bad == 0;
}

// The unknowns of one phase taken by block b of G: [k0, k1) of m.
__device__ __forceinline__ void own_range(int m, int b, int G, int& k0, int& k1) {
  const int cp = (m + G - 1) / G;
  k0 = min(m, b * cp);
  k1 = min(m, k0 + cp);
}

// The grid sums and scalars of a conjugate-gradient iteration (Chronopoulos
// and Gear's form) for every phase, from the G block partials (rows of
// PART_ROW doubles: gamma = r.u at p, delta = w.u at N + p, with RHO the
// residual measure rho = r.D^-1 r at 2N + p -- else rho = gamma, the
// Jacobi-preconditioned case -- and at the start the reference b.D^-1 b
// after them).  Warp p alone takes phase p: lane l sums rows l, l + 32, ...
// in order, a fixed shuffle tree sums the lanes, and lane 0 computes the
// scalars and publishes them in shared memory, from which every thread takes
// its copy.  An FP64 warp instruction holds its sub-partition's FP64 unit as
// long with one active lane as with 32, so the sums and divisions are paid
// by one warp a phase, not by every warp of the block (an iteration on the
// shock-bubble's band, measured: 14.1 us with every warp summing all rows
// and dividing, 11.1 us with the divisions in one warp a phase, 9.8 us with
// the sums there too).  The reciprocals of gamma and alpha are carried from
// the previous iteration, two divisions a phase:
//   beta = gamma' (1/gamma),  s = delta - beta gamma' (1/alpha),
//   alpha' = gamma' / s,  1/alpha' = s (1/gamma'),  1/gamma' for the next;
// a phase has converged when rho <= tol2 b.D^-1 b (or alpha is not positive).
template <int N>
struct CgScal {
  double gam[N], igam[N], alpha[N], ialpha[N], beta[N], ref[N], rho[N];
  int conv[N];
};
template <int N, bool RHO>
__device__ __forceinline__ void cg_scalars(const double* part, int G, double tol2, bool start,
                                           double* alpha, double* beta, double* rho,
                                           double* ref, bool* conv) {
  static_assert(32 * N <= PF_THREADS, "one warp a phase");
  static_assert((RHO ? 4 : 3) * N <= PART_ROW, "partial row");
  constexpr int KREF = RHO ? 3 * N : 2 * N;  // reference b.D^-1 b at the start
  __shared__ CgScal<N> cs;
  const int t = (int)threadIdx.x, p = t >> 5, lane = t & 31;
  if (p < N) {
    double g = 0.0, d = 0.0, rh = 0.0, rf = 0.0;
    for (int r0 = 0; r0 < G; r0 += 8 * 32) {
      double vg[8], vd[8], vh[8], vr[8];  // loads of up to 8 rows issued together
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int r = r0 + lane + 32 * k;
        const double* row = part + (long)r * PART_ROW;
        vg[k] = r < G ? __ldcg(row + p) : 0.0;
        vd[k] = r < G ? __ldcg(row + N + p) : 0.0;
        vh[k] = RHO && r < G ? __ldcg(row + 2 * N + p) : 0.0;
        vr[k] = start && r < G ? __ldcg(row + KREF + p) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; k++) {
        if (r0 + lane + 32 * k >= G) break;
        g += vg[k];
        d += vd[k];
        if (RHO) rh += vh[k];
        rf += vr[k];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      g += __shfl_down_sync(0xffffffffu, g, o);
      d += __shfl_down_sync(0xffffffffu, d, o);
      if (RHO) rh += __shfl_down_sync(0xffffffffu, rh, o);
      if (start) rf += __shfl_down_sync(0xffffffffu, rf, o);
    }
    if (!RHO) rh = g;
    if (lane == 0) {
      if (start) {
        const double ig = g > 0.0 ? 1.0 / g : 0.0;
        const double a = d > 0.0 ? g / d : 0.0;
        cs.gam[p] = g;
        cs.igam[p] = ig;
        cs.ref[p] = rf;
        cs.rho[p] = rh;
        cs.alpha[p] = a;
        cs.ialpha[p] = d * ig;
        cs.beta[p] = 0.0;
        cs.conv[p] = !(rh > tol2 * rf) || !(a > 0.0);
      } else if (!cs.conv[p]) {
        const double bt = g * cs.igam[p];
        const double den = d - bt * g * cs.ialpha[p];
        const double ign = g > 0.0 ? 1.0 / g : 0.0;
        const double a = den > 0.0 ? g / den : 0.0;
        cs.beta[p] = bt;
        cs.gam[p] = g;
        cs.igam[p] = ign;
        cs.rho[p] = rh;
        cs.alpha[p] = a;
        cs.ialpha[p] = den * ign;
        cs.conv[p] = !(rh > tol2 * cs.ref[p]) || !(a > 0.0);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < N; q++) {
    alpha[q] = cs.alpha[q];
    beta[q] = cs.beta[q];
    rho[q] = cs.rho[q];
    ref[q] = cs.ref[q];
    conv[q] = cs.conv[q] != 0;
  }
}

// Chebyshev preconditioner of the register-resident iteration: z = p(A) r
// with A = D^-1 K and p the polynomial of the Chebyshev iteration of degree
// CHEB_M - 1 for A z = D^-1 r on [2 / CHEB_ALPHA, 2] (A's eigenvalues lie in
// [0, 2]: K = D - W with W >= 0 and D its row sums).  1 - lambda p(lambda)
// is T_m((theta - lambda)/delta) / T_m(theta/delta), so lambda p(lambda) > 0
// on (0, 2] and M^-1 = p(A) D^-1 is symmetric positive definite on K's range:
// a valid preconditioner for conjugate gradients.  It squeezes the spectrum
// on [2/alpha, 2] and leaves the smallest modes (the slow ones along a thin
// band) for the outer iteration: on the 1024 x 512 shock-bubble's band
// (oracle operator, CPU) 294 Jacobi iterations became 79 with CHEB_M = 4,
// CHEB_ALPHA = 30.  Recurrence (theta, delta the interval's centre and
// half-width, sigma = theta/delta, rho_0 = 1/sigma):
//   d_0 = D^-1 r / theta,  z = d_0,  s = D^-1 r - A d_0,
//   rho_j = 1/(2 sigma - rho_{j-1}),  d_j = rho_j rho_{j-1} d_{j-1}
//   + (2 rho_j / delta) s,  z += d_j,  s -= A d_j   (j = 1 .. CHEB_M - 1);
// the K d_j it forms give w = K z = sum_j K d_j for free.
constexpr int CHEB_M = 4;
constexpr double CHEB_ALPHA = 30.0;
struct ChebCoef {
  double c0, a[CHEB_M], b[CHEB_M];
};
constexpr ChebCoef cheb_coef() {
  const double lo = 2.0 / CHEB_ALPHA, hi = 2.0;
  const double th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sg = th / de;
  ChebCoef c{};
  c.c0 = 1.0 / th;
  double r0 = 1.0 / sg;
  for (int j = 1; j < CHEB_M; j++) {
    const double r1 = 1.0 / (2.0 * sg - r0);
    c.a[j] = r1 * r0;
    c.b[j] = 2.0 * r1 / de;
    r0 = r1;
  }
  return c;
}

// The iterations of k_qmap_cg when every phase has at most R unknowns per
// thread (R G 256 unknowns: interface bands): thread t of block b takes
// unknowns b 256 + t + j G 256, j < R, of each phase and keeps their state
// in registers (cell, D, 1/D, the neighbours' list positions and face
// weights, x, r, u, w, p, s and the preconditioner's d and s).  The
// iteration is Chronopoulos and Gear's form of preconditioned conjugate
// gradients (the same iterates as the textbook form in exact arithmetic),
// whose two inner products r . u and w . u (u = M^-1 r, w = K u) are summed
// together with the residual measure r . D^-1 r:
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M^-1 r,
//   w = K u, gamma' = r . u, delta = w . u, beta = gamma'/gamma,
//   alpha = gamma' / (delta - beta gamma' / alpha),
// with M^-1 the Chebyshev polynomial preconditioner above: CHEB_M products
// K d_j an iteration, each after a barrier among the neighbouring blocks
// (nbr_sync) that makes the neighbours' d_j visible (alternately in w.p and
// w.q: a buffer is rewritten only after the next exchange, when every block
// that reads it has read it), then one grid barrier before the sums.  Against Jacobi (u = D^-1 r: one product and two barriers an
// iteration) it trades the sums, scalars and barrier of about three
// iterations for three more products.
template <int N, int R>
__device__ __forceinline__ void cg_one(const PfGeom& g, const PfWork& w, double tol2, int warm,
                                       int maxit, const int* scnt, int c0, int c1, unsigned* bar,
                                       int* err) {
  constexpr int E = N * R;  // slot e: phase e / R, unknown k + (e % R) G 256
  constexpr ChebCoef CC = cheb_coef();
  const int n = (int)g.ncell;
  const long nn = (long)N * n;
  const int G = (int)gridDim.x, t = (int)threadIdx.x;
  const int k = (int)blockIdx.x * PF_THREADS + t;
  const int span = G * PF_THREADS;
  int maxm = 0;
#pragma unroll
  for (int p = 0; p < N; p++) maxm = max(maxm, scnt[p]);
  // a warp whose unknowns are all past the lists contributes zeros (the
  // blocks take consecutive runs of 256: spreading the lists evenly over
  // every block measured no faster, the product being latency-bound)
  const bool idle_warp = (int)blockIdx.x * PF_THREADS + (t & ~31) >= maxm;
  bool has[E];
  int cell[E], ke[E], nbk[E][6];
  double Dv[E], Di[E], wg[E][6], x[E], r[E], u[E], wv[E], pv[E], sv[E], dd[E], sr[E];
  double acc[4 * N];
#pragma unroll
  for (int j = 0; j < 4 * N; j++) acc[j] = 0.0;
  // start: b, x0, r0 = b - K x0
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int p = e / R;
    const long o = (long)p * n;
    ke[e] = k + (e % R) * span;
    has[e] = ke[e] < scnt[p];
    x[e] = r[e] = u[e] = wv[e] = pv[e] = sv[e] = dd[e] = sr[e] = 0.0;
    Dv[e] = Di[e] = 0.0;
    cell[e] = 0;
#pragma unroll
    for (int f = 0; f < 6; f++) {
      nbk[e][f] = -1;
      wg[e][f] = 0.0;
    }
    if (!has[e]) continue;
    const int i = __ldcg(w.idx + o + ke[e]);
    cell[e] = i;
    int nb[3][2];
    pf_stencil(g, i, nb);
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
      if (ax >= g.dim) break;
      const double* wa = w.w + ax * nn + o;
      const int jm = nb[ax][0], jp = nb[ax][1];
      // a neighbour off the list shares no coupled face (weight 0)
      if (jp >= 0) {
        nbk[e][2 * ax + 1] = __ldcg(w.pos + o + jp);
        wg[e][2 * ax + 1] = wa[i];
      }
      if (jm >= 0) {
        nbk[e][2 * ax] = __ldcg(w.pos + o + jm);
        wg[e][2 * ax] = wa[jm];
      }
    }
    const int l = __ldcg(w.lab + o + i);
    const double sk = __ldcg(w.sumR + o + l) / __ldcg(w.sumD + o + l);
    Dv[e] = w.D[o + i];
    Di[e] = w.Dinv[o + i];
    const double bv = -(w.R[o + i] - Dv[e] * sk);
    r[e] = bv;
    if (warm) {
      x[e] = w.x[o + i];
      r[e] = bv - k_apply<N>(g, nb, i, o, nn, w.w, w.D, w.x);
    }
    acc[3 * N + p] = fma(bv, bv * Di[e], acc[3 * N + p]);
  }
  bool conv[N];
#pragma unroll
  for (int p = 0; p < N; p++) conv[p] = false;
  // the blocks owning this block's neighbours (list position k of a phase
  // belongs to block (k mod G 256) / 256): the preconditioner's exchanges
  // wait for them only (nbr_sync)
  int lo, hi;
  {
    __shared__ int s_lo, s_hi;
    if (t == 0) s_lo = s_hi = (int)blockIdx.x;
    __syncthreads();
    int ml = (int)blockIdx.x, mh = (int)blockIdx.x;
#pragma unroll
    for (int e = 0; e < E; e++) {
      if (!has[e]) continue;
#pragma unroll
      for (int f = 0; f < 6; f++) {
        if (nbk[e][f] < 0) continue;
        const int q = (nbk[e][f] % span) / PF_THREADS;
        ml = min(ml, q);
        mh = max(mh, q);
      }
    }
    atomicMin(&s_lo, ml);
    atomicMax(&s_hi, mh);
    __syncthreads();
    lo = s_lo;
    hi = s_hi;
  }
  unsigned* nflag = reinterpret_cast<unsigned*>(w.part + PART_NBR);
  unsigned epoch = 0u;
  // u = M^-1 r and w = K u for the phases not yet converged (CHEB_M
  // neighbour exchanges), then gamma = r.u, delta = w.u and rho = r.D^-1 r
  // into acc
  auto precondition = [&]() -> bool {
#pragma unroll
    for (int e = 0; e < E; e++) {
      const int p = e / R;
      if (conv[p] || !has[e]) continue;
      const double rr = r[e] * Di[e];
      dd[e] = rr * CC.c0;
      u[e] = dd[e];
      wv[e] = 0.0;
      sr[e] = rr;
    }
#pragma unroll
    for (int j = 0; j < CHEB_M; j++) {
      double* xb = (j & 1) ? w.q : w.p;
#pragma unroll
      for (int e = 0; e < E; e++) {
        const int p = e / R;
        if (conv[p] || !has[e]) continue;
        xb[(long)p * n + ke[e]] = dd[e];
      }
      if (!nbr_sync(nflag, lo, hi, ++epoch, err)) return false;
#pragma unroll
      for (int e = 0; e < E; e++) {
        const int p = e / R;
        if (conv[p] || !has[e]) continue;
        const long o = (long)p * n;
        double q = Dv[e] * dd[e];  // K d_j
#pragma unroll
        for (int f = 0; f < 6; f++)
          if (nbk[e][f] >= 0) q = fma(-wg[e][f], __ldcg(xb + o + nbk[e][f]), q);
        wv[e] += q;
        if (j + 1 < CHEB_M) {
          sr[e] = fma(-Di[e], q, sr[e]);
          dd[e] = fma(CC.a[j + 1], dd[e], CC.b[j + 1] * sr[e]);
          u[e] += dd[e];
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 3 * N; p++) acc[p] = 0.0;
#pragma unroll
    for (int e = 0; e < E; e++) {
      const int p = e / R;
      if (conv[p] || !has[e]) continue;
      acc[p] = fma(r[e], u[e], acc[p]);
      acc[N + p] = fma(wv[e], u[e], acc[N + p]);
      acc[2 * N + p] = fma(r[e], r[e] * Di[e], acc[2 * N + p]);
    }
    return true;
  };
  double rho[N], alpha[N], beta[N], ref[N];
  int it = 0;
  bool ok = precondition();
  if (ok) {
    double v4[4 * N];
#pragma unroll
    for (int j = 0; j < 4 * N; j++) v4[j] = acc[j];
    block_sum_small<4 * N>(v4, w.part + PART_CG1 + (long)blockIdx.x * PART_ROW, idle_warp);
    ok = grid_sync(bar, err);
  }
  if (ok) {
    cg_scalars<N, true>(w.part + PART_CG1, G, tol2, true, alpha, beta, rho, ref, conv);
    // the start may meet the test already; the others iterate
    while (it < maxit) {
      bool all = true;
#pragma unroll
      for (int p = 0; p < N; p++) all = all && conv[p];
      if (all) break;
#pragma unroll
      for (int e = 0; e < E; e++) {
        const int p = e / R;
        if (conv[p] || !has[e]) continue;
        pv[e] = fma(beta[p], pv[e], u[e]);
        sv[e] = fma(beta[p], sv[e], wv[e]);
        x[e] = fma(alpha[p], pv[e], x[e]);
        r[e] = fma(-alpha[p], sv[e], r[e]);
      }
      if (!(ok = precondition())) break;
      double v3[3 * N];
#pragma unroll
      for (int j = 0; j < 3 * N; j++) v3[j] = acc[j];
      block_sum_small<3 * N>(v3, w.part + PART_CG1 + (long)blockIdx.x * PART_ROW, idle_warp);
      if (!(ok = grid_sync(bar, err))) break;
      cg_scalars<N, true>(w.part + PART_CG1, G, tol2, false, alpha, beta, rho, ref, conv);
      it++;
    }
  }
  if (ok) {
#pragma unroll
    for (int e = 0; e < E; e++)
      if (has[e]) w.x[(long)(e / R) * n + cell[e]] = x[e];
    if (!warm)
#pragma unroll
      for (int p = 0; p < N; p++) {
        const long o = (long)p * n;
        for (int i = c0 + t; i < c1; i += PF_THREADS)
          if (w.pos[o + i] < 0) w.x[o + i] = 0.0;
      }
  }
  if (blockIdx.x == 0 && t == 0 && ok) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      w.scal[16 + p] = ref[p];
      w.scal[24 + p] = rho[p];
      w.flag[1 + p] = conv[p] ? 1 : 0;
    }
    w.flag[11] = it;
  }
}

// The same iteration with the state in memory, for bands larger than the
// registers take: block b takes a contiguous range of each phase's list
// (own_range: position k of a phase of m unknowns belongs to block
// k / ceil(m / G)), its threads the same unknowns every iteration, in the
// workspace's list layout (p ncell + k): x (xk), r, the directions p (pd)
// and s (sd), u (p) and w = K u (q), and for the Chebyshev preconditioner
// its residual (c, whose coefficients the set-up has consumed) and d_j,
// exchanged among neighbouring blocks (nbr_sync) alternately in sumR and
// sumD (read only to form the right-hand side, before the grid barrier that
// follows the start).  Same preconditioner and form as the register path.
template <int N, int BT, int MB>
__device__ __forceinline__ void cg_mem(const PfGeom& g, const PfWork& w, double tol2, int warm,
                                       int maxit, const int* scnt, int c0, int c1, unsigned* bar,
                                       int* err) {
  static_assert(32 * N <= BT, "cg_scalars takes one warp a phase");
  constexpr ChebCoef CC = cheb_coef();
  const int n = (int)g.ncell;
  const long nn = (long)N * n;
  const int G = (int)gridDim.x, b = (int)blockIdx.x, t = (int)threadIdx.x;
  double* const xbuf[2] = {w.sumR, w.sumD};
  double acc[4 * N];
#pragma unroll
  for (int j = 0; j < 4 * N; j++) acc[j] = 0.0;
  // start: b, x0, r0 = b - K x0; the neighbour blocks' range
  int ml = b, mh = b;
#pragma unroll
  for (int p = 0; p < N; p++) {
    const long o = (long)p * n;
    int k0, k1;
    own_range(scnt[p], b, G, k0, k1);
    const int cp = (scnt[p] + G - 1) / G;
    for (int k = k0 + t; k < k1; k += BT) {
      const int i = __ldcg(w.idx + o + k);
      const int l = __ldcg(w.lab + o + i);
      const double sk = __ldcg(w.sumR + o + l) / __ldcg(w.sumD + o + l);
      const double bv = -(w.R[o + i] - w.D[o + i] * sk);
      int nb[3][2];
      pf_stencil(g, i, nb);
      double x0 = 0.0, r0 = bv;
      if (warm) {
        x0 = w.x[o + i];
        r0 = bv - k_apply<N>(g, nb, i, o, nn, w.w, w.D, w.x);
      }
#pragma unroll
      for (int ax = 0; ax < 3; ax++) {
        if (ax >= g.dim) break;
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
          const int j = nb[ax][sd];
          if (j < 0) continue;
          const int kq = __ldcg(w.pos + o + j);
          if (kq < 0) continue;
          ml = min(ml, kq / cp);
          mh = max(mh, kq / cp);
        }
      }
      w.xk[o + k] = x0;
      w.r[o + k] = r0;
      acc[3 * N + p] = fma(bv, bv * w.Dinv[o + i], acc[3 * N + p]);
    }
  }
  int lo, hi;
  {
    __shared__ int s_lo, s_hi;
    if (t == 0) s_lo = s_hi = b;
    __syncthreads();
    atomicMin(&s_lo, ml);
    atomicMax(&s_hi, mh);
    __syncthreads();
    lo = s_lo;
    hi = s_hi;
  }
  unsigned* nflag = reinterpret_cast<unsigned*>(w.part + PART_NBR);
  unsigned epoch = 0u;
  bool conv[N];
#pragma unroll
  for (int p = 0; p < N; p++) conv[p] = false;
  // (the right-hand side has read sumR and sumD: they become the exchange
  // buffers after this barrier)
  bool ok = grid_sync(bar, err);
  // u = M^-1 r, w = K u for the phases not yet converged, then r.u, w.u and
  // r.D^-1 r into acc; the unknowns of a thread in batches of MB, their
  // loads issued together
  auto precondition = [&]() -> bool {
#pragma unroll 1
    for (int p = 0; p < N; p++) {
      if (conv[p]) continue;
      const long o = (long)p * n;
      int k0, k1;
      own_range(scnt[p], b, G, k0, k1);
      for (int k = k0 + t; k < k1; k += BT) {
        const double rr = w.r[o + k] * w.Dinv[o + __ldcg(w.idx + o + k)];
        const double d0 = rr * CC.c0;
        xbuf[0][o + k] = d0;
        w.p[o + k] = d0;
        w.q[o + k] = 0.0;
        w.c[o + k] = rr;
      }
    }
#pragma unroll
    for (int j = 0; j < CHEB_M; j++) {
      const double* xb = xbuf[j & 1];
      double* xn = xbuf[(j + 1) & 1];
      if (!nbr_sync(nflag, lo, hi, ++epoch, err)) return false;
#pragma unroll 1
      for (int p = 0; p < N; p++) {
        if (conv[p]) continue;
        const long o = (long)p * n;
        int k0, k1;
        own_range(scnt[p], b, G, k0, k1);
        for (int kb = k0 + t; kb < k1; kb += MB * BT) {
          int ii[MB], kn[MB][6];
          double wt[MB][6], un[MB][6];
#pragma unroll
          for (int m = 0; m < MB; m++) {
            const int k = kb + m * BT;
            ii[m] = k < k1 ? __ldcg(w.idx + o + k) : -1;
          }
#pragma unroll
          for (int m = 0; m < MB; m++) {
#pragma unroll
            for (int f = 0; f < 6; f++) {
              kn[m][f] = -1;
              wt[m][f] = 0.0;
            }
            if (ii[m] < 0) continue;
            const int i = ii[m];
            int nb[3][2];
            pf_stencil(g, i, nb);
#pragma unroll
            for (int ax = 0; ax < 3; ax++) {
              if (ax >= g.dim) break;
              const double* wa = w.w + ax * nn + o;
              const int jm = nb[ax][0], jp = nb[ax][1];
              // a neighbour off the list shares no coupled face (weight 0)
              if (jp >= 0) {
                kn[m][2 * ax] = __ldcg(w.pos + o + jp);
                wt[m][2 * ax] = wa[i];
              }
              if (jm >= 0) {
                kn[m][2 * ax + 1] = __ldcg(w.pos + o + jm);
                wt[m][2 * ax + 1] = wa[jm];
              }
            }
          }
#pragma unroll
          for (int m = 0; m < MB; m++)
#pragma unroll
            for (int f = 0; f < 6; f++)
              un[m][f] = kn[m][f] >= 0 ? __ldcg(xb + o + kn[m][f]) : 0.0;
#pragma unroll
          for (int m = 0; m < MB; m++) {
            if (ii[m] < 0) continue;
            const int k = kb + m * BT, i = ii[m];
            const double dk = __ldcg(xb + o + k);
            double q = w.D[o + i] * dk;  // K d_j
#pragma unroll
            for (int f = 0; f < 6; f++)
              if (kn[m][f] >= 0) q = fma(-wt[m][f], un[m][f], q);
            w.q[o + k] += q;
            if (j + 1 < CHEB_M) {
              const double sr = fma(-w.Dinv[o + i], q, w.c[o + k]);
              w.c[o + k] = sr;
              const double dn = fma(CC.a[j + 1], dk, CC.b[j + 1] * sr);
              xn[o + k] = dn;
              w.p[o + k] += dn;
            }
          }
        }
      }
    }
#pragma unroll 1
    for (int p = 0; p < N; p++) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      if (!conv[p]) {
        const long o = (long)p * n;
        int k0, k1;
        own_range(scnt[p], b, G, k0, k1);
        for (int k = k0 + t; k < k1; k += BT) {
          const double rk = w.r[o + k], uk = w.p[o + k];
          s0 = fma(rk, uk, s0);
          s1 = fma(w.q[o + k], uk, s1);
          s2 = fma(rk, rk * w.Dinv[o + __ldcg(w.idx + o + k)], s2);
        }
      }
      acc[p] = s0;
      acc[N + p] = s1;
      acc[2 * N + p] = s2;
    }
    return true;
  };
  double rho[N], alpha[N], beta[N], ref[N];
  int it = 0;
  if (ok) ok = precondition();
  if (ok) {
    double v4[4 * N];
#pragma unroll
    for (int j = 0; j < 4 * N; j++) v4[j] = acc[j];
    block_sum_small<4 * N, BT>(v4, w.part + PART_CG1 + (long)b * PART_ROW);
    ok = grid_sync(bar, err);
  }
  if (ok) {
    cg_scalars<N, true>(w.part + PART_CG1, G, tol2, true, alpha, beta, rho, ref, conv);
    while (it < maxit) {
      bool all = true;
#pragma unroll
      for (int p = 0; p < N; p++) all = all && conv[p];
      if (all) break;
#pragma unroll
      for (int p = 0; p < N; p++) {
        if (conv[p]) continue;
        const long o = (long)p * n;
        int k0, k1;
        own_range(scnt[p], b, G, k0, k1);
        for (int k = k0 + t; k < k1; k += BT) {
          const double uk = w.p[o + k], qk = w.q[o + k];
          // (the first directions are u and K u themselves)
          const double pk = it == 0 ? uk : fma(beta[p], w.pd[o + k], uk);
          const double sk = it == 0 ? qk : fma(beta[p], w.sd[o + k], qk);
          w.pd[o + k] = pk;
          w.sd[o + k] = sk;
          w.xk[o + k] = fma(alpha[p], pk, w.xk[o + k]);
          w.r[o + k] = fma(-alpha[p], sk, w.r[o + k]);
        }
      }
      if (!(ok = precondition())) break;
      double v3[3 * N];
#pragma unroll
      for (int j = 0; j < 3 * N; j++) v3[j] = acc[j];
      block_sum_small<3 * N, BT>(v3, w.part + PART_CG1 + (long)b * PART_ROW);
      if (!(ok = grid_sync(bar, err))) break;
      cg_scalars<N, true>(w.part + PART_CG1, G, tol2, false, alpha, beta, rho, ref, conv);
      it++;
    }
  }
  if (ok) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      const long o = (long)p * n;
      int k0, k1;
      own_range(scnt[p], b, G, k0, k1);
      for (int k = k0 + t; k < k1; k += BT) w.x[o + __ldcg(w.idx + o + k)] = w.xk[o + k];
      if (!warm)
        for (int i = c0 + t; i < c1; i += BT)
          if (w.pos[o + i] < 0) w.x[o + i] = 0.0;
    }
  }
  if (b == 0 && t == 0 && ok) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      w.scal[16 + p] = ref[p];
      w.scal[24 + p] = rho[p];
      w.flag[1 + p] = conv[p] ? 1 : 0;
    }
    w.flag[11] = it;
  }
}

// x 2^k for |k| <= 2000 as two exact power-of-two factors (each in
// [-1000, 1000], a normal double): exact unless the result leaves the
// normal range.
__device__ __forceinline__ double pf_pow2(int j) {
  return __longlong_as_double((long long)(j + 1023) << 52);
}
__device__ __forceinline__ double pf_scale2(double x, int k) {
  const int k1 = k / 2;
  return (x * pf_pow2(k1)) * pf_pow2(k - k1);
}

// Exponent E of a positive finite double given by its bits: 2^E <= M < 2^(E+1).
__device__ __forceinline__ int pf_exponent(unsigned long long bits) {
  const int ef = (int)(bits >> 52);
  return ef > 0 ? ef - 1023 : -1074 + (63 - __clzll((long long)bits));
}

// Region sums of R and D (the right-hand side's consistency shift of Eq. 4:
// sum_region R / sum_region D), the same bit for bit whatever the order in
// which threads add.  Per region and quantity the largest magnitude M,
// 2^E <= M < 2^(E+1), fixes a scale; each value x becomes y = x 2^(31-E),
// |y| < 2^32, split into hi = floor(y) and lo = floor((y - hi) 2^32) in
// [0, 2^32) (both exact), and hi and lo are summed as 64-bit integers,
// whose addition is associative and cannot overflow below 2^30 cells a
// region.  The sum is then (sum hi 2^32 + sum lo) 2^(E-63): each value is
// cut at 2^(E-63), below the 2^(E-53) rounding of one FP64 addition at
// the region's scale.  Scratch: the iteration's vectors, which are written
// before they are read once the sums are taken (maxima in r and xk, hi and
// lo in p, q, pd and sd), at the region's label (a listed cell).  Three
// grid barriers; false if one gave up.
template <int N>
__device__ __forceinline__ bool region_sums(const PfWork& w, int n, const int* scnt, int b, int G,
                                            int t, unsigned* bar, int* err) {
  typedef unsigned long long u64;
  u64* mR = reinterpret_cast<u64*>(w.r);
  u64* mD = reinterpret_cast<u64*>(w.xk);
  u64* hR = reinterpret_cast<u64*>(w.p);
  u64* lR = reinterpret_cast<u64*>(w.q);
  u64* hD = reinterpret_cast<u64*>(w.pd);
  u64* lD = reinterpret_cast<u64*>(w.sd);
  // (i) clear, and the magnitudes of the region's values
#pragma unroll
  for (int p = 0; p < N; p++) {
    const long o = (long)p * n;
    int k0, k1;
    own_range(scnt[p], b, G, k0, k1);
    for (int k = k0 + t; k < k1; k += PF_THREADS) {
      const long a = o + __ldcg(w.idx + o + k);
      mR[a] = mD[a] = hR[a] = lR[a] = hD[a] = lD[a] = 0ull;
    }
  }
  if (!grid_sync(bar, err)) return false;
#pragma unroll
  for (int p = 0; p < N; p++) {
    const long o = (long)p * n;
    int k0, k1;
    own_range(scnt[p], b, G, k0, k1);
    for (int k = k0 + t; k < k1; k += PF_THREADS) {
      const int i = __ldcg(w.idx + o + k);
      const long l = o + __ldcg(w.lab + o + i);
      // the bits of |x| order as |x| does
      atomicMax(mR + l, (u64)__double_as_longlong(fabs(w.R[o + i])));
      atomicMax(mD + l, (u64)__double_as_longlong(fabs(w.D[o + i])));
    }
  }
  if (!grid_sync(bar, err)) return false;
  // (ii) the fixed-point parts, added as integers (two's complement wraps
  // to the signed sum)
  auto split = [](double x, u64 mbits, u64& hi, u64& lo) {
    if (mbits == 0ull || mbits >= 0x7ff0000000000000ull) {
      hi = lo = 0ull;
      return;
    }
    const double y = pf_scale2(x, 31 - pf_exponent(mbits));
    const double f = floor(y);
    hi = (u64)(long long)f;
    lo = (u64)(long long)floor((y - f) * 4294967296.0);
  };
#pragma unroll
  for (int p = 0; p < N; p++) {
    const long o = (long)p * n;
    int k0, k1;
    own_range(scnt[p], b, G, k0, k1);
    for (int k = k0 + t; k < k1; k += PF_THREADS) {
      const int i = __ldcg(w.idx + o + k);
      const long l = o + __ldcg(w.lab + o + i);
      u64 hi, lo;
      split(w.R[o + i], __ldcg(mR + l), hi, lo);
      atomicAdd(hR + l, hi);
      atomicAdd(lR + l, lo);
      split(w.D[o + i], __ldcg(mD + l), hi, lo);
      atomicAdd(hD + l, hi);
      atomicAdd(lD + l, lo);
    }
  }
  if (!grid_sync(bar, err)) return false;
  // (iii) back to FP64 at each region's label; a region holding a value
  // that is not finite sums to NaN
  auto join = [](u64 mbits, u64 hs, u64 ls) {
    if (mbits == 0ull) return 0.0;
    if (mbits >= 0x7ff0000000000000ull) return __longlong_as_double(0x7ff8000000000000ll);
    const long long h = (long long)hs + (long long)(ls >> 32);
    const double v = fma((double)h, 4294967296.0, (double)(long long)(ls & 0xffffffffull));
    return pf_scale2(v, pf_exponent(mbits) - 63);
  };
#pragma unroll
  for (int p = 0; p < N; p++) {
    const long o = (long)p * n;
    int k0, k1;
    own_range(scnt[p], b, G, k0, k1);
    for (int k = k0 + t; k < k1; k += PF_THREADS) {
      const int i = __ldcg(w.idx + o + k);
      if (__ldcg(w.lab + o + i) != i) continue;
      const long a = o + i;
      w.sumR[a] = join(__ldcg(mR + a), __ldcg(hR + a), __ldcg(lR + a));
      w.sumD[a] = join(__ldcg(mD + a), __ldcg(hD + a), __ldcg(lD + a));
    }
  }
  return grid_sync(bar, err);
}

template <int N>
__global__ void __launch_bounds__(PF_THREADS) k_qmap_cg(PfGeom g, PfWork w, double tol2, int warm,
                                                        int maxit) {
  const int n = (int)g.ncell;
  const long nn = (long)N * n;
  const int G = (int)gridDim.x, b = (int)blockIdx.x, t = (int)threadIdx.x;
  unsigned* bar = reinterpret_cast<unsigned*>(w.flag + 8);
  int* err = w.flag + 10;
  __shared__ int wtot[PF_THREADS / 32], soff[N], scnt[N];
  // the preconditioner's neighbour flags start at epoch 0 (published by the
  // grid barriers before the iteration)
  if (t == 0) reinterpret_cast<unsigned*>(w.part + PART_NBR)[8 * b] = 0u;

  // 1. list
  const int cc = (n + G - 1) / G, c0 = min(n, b * cc), c1 = min(n, c0 + cc);
  for (int p = 0; p < N; p++) {
    int cnt = 0;
    for (int i = c0 + t; i < c1; i += PF_THREADS) cnt += w.lab[(long)p * n + i] >= 0 ? 1 : 0;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((t & 31) == 0) wtot[t >> 5] = cnt;
    __syncthreads();
    if (t == 0) {
      int sum = 0;
      for (int k = 0; k < PF_THREADS / 32; k++) sum += wtot[k];
      w.part[PART_LIST + (long)b * 8 + p] = (double)sum;
    }
    __syncthreads();
  }
  if (!grid_sync(bar, err)) return;
  if (t < 32) {
    for (int p = 0; p < N; p++) {
      int o = 0, m = 0;
      for (int bb = t; bb < G; bb += 32) {
        const int c = (int)__ldcg(w.part + PART_LIST + (long)bb * 8 + p);
        m += c;
        if (bb < b) o += c;
      }
      o = __reduce_add_sync(0xffffffffu, o);
      m = __reduce_add_sync(0xffffffffu, m);
      if (t == 0) {
        soff[p] = o;
        scnt[p] = m;
      }
    }
  }
  __syncthreads();
  for (int p = 0; p < N; p++) {
    const long o = (long)p * n;
    int base = soff[p];
    for (int i0 = c0; i0 < c1; i0 += PF_THREADS) {
      const int i = i0 + t;
      const bool act = i < c1 && w.lab[o + i] >= 0;
      const unsigned bal = __ballot_sync(0xffffffffu, act);
      if ((t & 31) == 0) wtot[t >> 5] = __popc(bal);
      __syncthreads();
      int before = 0, tot = 0;
      for (int k = 0; k < PF_THREADS / 32; k++) {
        const int v = wtot[k];
        tot += v;
        if (k < (t >> 5)) before += v;
      }
      const int k = base + before + __popc(bal & ((1u << (t & 31)) - 1u));
      if (i < c1) w.pos[o + i] = act ? k : -1;
      if (act) w.idx[o + k] = i;
      base += tot;
      __syncthreads();
    }
  }
  if (!grid_sync(bar, err)) return;

  // 1b. region labels: rounds of minimum-label propagation over coupled
  // faces with pointer jumping, on the listed cells, until a round changes
  // nothing.  Labels only decrease and always name a listed cell of the
  // same region, so the rounds end with every cell of a region labelled by
  // the region's smallest cell index.  A round's change word is one of
  // three: it was last read two barriers before and is cleared a round
  // ahead by block 0, so every block reads the same value.
  int rounds = 0;
  for (;;) {
    int* chg = w.flag + 20 + rounds % 3;
    if (b == 0 && t == 0) w.flag[20 + (rounds + 1) % 3] = 0;
    int changed = 0;
#pragma unroll
    for (int p = 0; p < N; p++) {
      const long o = (long)p * n;
      int* lp = w.lab + o;
      int k0, k1;
      own_range(scnt[p], b, G, k0, k1);
      for (int k = k0 + t; k < k1; k += PF_THREADS) {
        const int i = __ldcg(w.idx + o + k);
        const int li = __ldcg(lp + i);
        int nb[3][2];
        pf_stencil(g, i, nb);
        int m = li;
        // a face couples its cells when the operator's weight on it is
        // positive (the test k_qm_diag lists cells by): then both cells
        // are listed and carry labels >= 0.  (c_a + c_b)/2 of a denormal
        // c next to c = 0 rounds to a zero weight, and such a neighbour
        // is not listed.
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
          if (ax >= g.dim) break;
          const double* wa = w.w + ax * nn + o;
#pragma unroll
          for (int sd = 0; sd < 2; sd++) {
            const int j = nb[ax][sd];
            if (j >= 0 && wa[sd ? i : j] > 0.0) m = min(m, __ldcg(lp + j));
          }
        }
        m = min(m, __ldcg(lp + m));
        if (m < li) {
          atomicMin(lp + i, m);
          changed = 1;
        }
      }
    }
    if (__syncthreads_or(changed) && t == 0) atomicOr(chg, 1);
    if (!grid_sync(bar, err)) return;
    rounds++;
    if (__ldcg(chg) == 0) break;
    if (rounds > n + 1) {  // cannot happen: a changing round lowers a label
      if (b == 0 && t == 0) w.flag[24] = 1;
      return;
    }
  }
  if (b == 0 && t == 0) w.flag[23] = rounds;
  // 1c. region sums of R and D over the listed cells, in fixed point so
  // that the order of the additions does not matter (region_sums)
  if (!region_sums<N>(w, n, scnt, b, G, t, bar, err)) return;

  // unknowns a thread keeps in registers: one, two (N <= 2), else the
  // iteration on the lists in memory below
  int maxm = 0;
#pragma unroll
  for (int p = 0; p < N; p++) maxm = max(maxm, scnt[p]);
  const int per_thread = maxm <= G * PF_THREADS ? 1 : (N <= 2 && maxm <= 2 * G * PF_THREADS ? 2 : 0);
  if (b == 0 && t == 0) {
#pragma unroll
    for (int p = 0; p < N; p++) w.flag[12 + p] = scnt[p];
    w.flag[17] = per_thread;
  }
  if (per_thread == 1) {
    cg_one<N, 1>(g, w, tol2, warm, maxit, scnt, c0, c1, bar, err);
    return;
  }
  if constexpr (N <= 2) {
    if (per_thread == 2) {
      cg_one<N, 2>(g, w, tol2, warm, maxit, scnt, c0, c1, bar, err);
      return;
    }
  }

  // larger bands: k_qmap_cg_mem, launched next with more threads an SM
  if (b == 0 && t == 0) w.flag[18] = 1;
}

// The iteration on the lists in memory (bands of more than two unknowns a
// thread of k_qmap_cg): a cooperative launch of one 256-thread block per SM
// after k_qmap_cg has listed the unknowns (their counts in w.flag[12 + p]).
// Its own launch keeps k_qmap_cg's register-resident paths free of this
// code (they run faster so).  1024-thread blocks with one unknown a thread
// measured slower (35 against 24 us an iteration: 32 warps' reductions and
// register spills).
template <int N>
__global__ void __launch_bounds__(PF_THREADS, 1) k_qmap_cg_mem(PfGeom g, PfWork w, double tol2,
                                                               int warm, int maxit) {
  __shared__ int scnt[N];
  if (threadIdx.x < N) scnt[threadIdx.x] = __ldcg(w.flag + 12 + threadIdx.x);
  // the neighbour flags start at epoch 0 (published by cg_mem's first grid
  // barrier, before the first exchange)
  if (threadIdx.x == 0) reinterpret_cast<unsigned*>(w.part + PART_NBR)[8 * blockIdx.x] = 0u;
  __syncthreads();
  const int n = (int)g.ncell, G = (int)gridDim.x, b = (int)blockIdx.x;
  const int cc = (n + G - 1) / G, c0 = min(n, b * cc), c1 = min(n, c0 + cc);
  cg_mem<N, PF_THREADS, 4>(g, w, tol2, warm, maxit, scnt, c0, c1,
                     reinterpret_cast<unsigned*>(w.flag + 8), w.flag + 10);
}

// The grid barrier alone, for its test: rounds barriers, except that block
// skip (>= 0) leaves before the first, so every other block's wait runs
// out and sets the error word.
__global__ void __launch_bounds__(PF_THREADS) k_barrier_check(unsigned* bar, int* err, int skip,
                                                              int rounds) {
  if ((int)blockIdx.x == skip) return;
  for (int r = 0; r < rounds; r++)
    if (!grid_sync(bar, err)) return;
}

// The neighbour barrier alone, for its test: blocks on a line, block b
// waiting for the blocks within span of it, rounds exchanges; block skip
// (>= 0) leaves before the first, so its neighbours' waits run out and set
// the error word, and the others stop waiting when they see it.
__global__ void __launch_bounds__(PF_THREADS) k_nbr_check(unsigned* flags, int* err, int skip,
                                                          int span, int rounds) {
  const int b = (int)blockIdx.x, G = (int)gridDim.x;
  if (b == skip) return;
  const int lo = max(0, b - span), hi = min(G - 1, b + span);
  for (int r = 0; r < rounds; r++)
    if (!nbr_sync(flags, lo, hi, (unsigned)(r + 1), err)) return;
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
  PF_DISPATCH(g.N, (k_cac_solve<N_><<<1, PF_THREADS, 0, st>>>(w.part + PART_CAC, vol, eta, M_in,
                                                              w.scal)));
  PF_DISPATCH(g.N, (k_cac_rhs<N_><<<pf_grid(g.ncell), PF_THREADS, 0, st>>>(U, g, w.scal, eta, w.R)));
  return cudaGetLastError();
}

cudaError_t pf_qmap_setup(const double* U, const PfGeom& g, const PfWork& w, cudaStream_t st) {
  const int nb = pf_grid(g.ncell);
  PF_DISPATCH(g.N, (k_qm_coef<N_><<<nb, PF_THREADS, 0, st>>>(U, g, w.c)));
  PF_DISPATCH(g.N, (k_qm_diag<N_><<<nb, PF_THREADS, 0, st>>>(g, w.c, w.w, w.D, w.Dinv, w.lab)));
  return cudaGetLastError();
}


cudaError_t pf_qmap_solve(const PfGeom& g, const PfWork& w, int warm, double tol2, int maxit,
                          cudaStream_t st) {
  // the grid barrier's arrival count, generation and error word; the
  // deferral word; the labelling's change words, rounds and error word
  cudaError_t e = cudaMemsetAsync(w.flag + 8, 0, 3 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.flag + 18, 0, 7 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  // one block per SM, all resident (a cooperative launch fails otherwise);
  // the register-resident iteration takes up to 256 unknowns a block and
  // phase.  (Two blocks per SM, where registers allow, measured slower: 25
  // against 15 us an iteration on the shock-bubble bands.)
  // SM count of the current device, queried per call (a process may drive
  // devices of different sizes)
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms < 1 ? 1 : (sms > 4 * PF_THREADS ? 4 * PF_THREADS : sms);
  PfGeom gg = g;
  PfWork ww = w;
  void* args[] = {&gg, &ww, &tol2, &warm, &maxit};
  PF_DISPATCH(g.N, (e = cudaLaunchCooperativeKernel((const void*)k_qmap_cg<N_>, dim3(blocks),
                                                    dim3(PF_THREADS), args, 0, st)));
  if (e != cudaSuccess) return e;
  // a band too large for the registers: the in-memory iteration follows
  int deferred = 0, errw = 0;
  e = cudaMemcpyAsync(&deferred, w.flag + 18, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&errw, w.flag + 10, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || !deferred || errw) return e;
  e = cudaMemsetAsync(w.flag + 8, 0, 3 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  PF_DISPATCH(g.N, (e = cudaLaunchCooperativeKernel((const void*)k_qmap_cg_mem<N_>,
                                                    dim3(blocks), dim3(PF_THREADS), args, 0, st)));
  return e;
}

cudaError_t pf_barrier_check(int* words, int skip, int rounds, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(words, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  unsigned* bar = reinterpret_cast<unsigned*>(words);
  int* err = words + 2;
  void* args[] = {&bar, &err, &skip, &rounds};
  return cudaLaunchCooperativeKernel((const void*)k_barrier_check, dim3(sms < 1 ? 1 : sms),
                                     dim3(PF_THREADS), args, 0, st);
}

size_t pf_nbr_check_words() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return 0;
  return 8 + 8 * (size_t)sms;
}

cudaError_t pf_nbr_check(int* words, int skip, int span, int rounds, cudaStream_t st) {
  const size_t nw = pf_nbr_check_words();
  if (nw == 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(words, 0, nw * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const unsigned sms = (unsigned)((nw - 8) / 8);
  int* err = words + 2;
  unsigned* flags = reinterpret_cast<unsigned*>(words + 8);
  void* args[] = {&flags, &err, &skip, &span, &rounds};
  return cudaLaunchCooperativeKernel((const void*)k_nbr_check, dim3(sms), dim3(PF_THREADS), args,
                                     0, st);
}

}  // namespace wc
