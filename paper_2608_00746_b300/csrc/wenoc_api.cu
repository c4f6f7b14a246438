// wenoc_api.cu -- host side of the C ABI declared in include/wenoc.h.
// Argument checks, grid descriptors, Runge-Kutta stage orchestration and
// kernel dispatch.  The library allocates no device memory: the caller binds
// its state array and a workspace.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/wenoc.h"
#include "wenoc_kernels.cuh"
#include "wenoc_mlp.cuh"
#include "wenoc_pf.cuh"
#include "wenoc_window.cuh"

using namespace wc;

struct wc_grid {
  wc_grid_desc d;
  Mat mat;
  int nv;
  long ncell;
  double* U = nullptr;       // bound state (caller's device memory)
  char* ws = nullptr;        // bound workspace
  size_t ws_bytes = 0;
  double* B1 = nullptr;      // stage buffers
  double* B2 = nullptr;
  double* Lacc = nullptr;    // direction accumulator
  unsigned* status = nullptr;
  unsigned long long* rate = nullptr;
  double* dt = nullptr;
  unsigned* ticket = nullptr;  // window queue (two words, zero between launches)
  // learned precision: the surrogate's parameter block (caller's device
  // memory), acceptance threshold, optional counters and the weight buffer
  // (in the workspace, after its 256-byte tail)
  const void* mlp = nullptr;
  float tau = 1e-4f;
  unsigned long long* lcount = nullptr;
  float* Wbuf = nullptr;
  // window schedule: the primitive slots of a stage's input (in the
  // workspace, after the learned weights); null: each sweep converts its cells
  double* vbuf = nullptr;
  // reduced precision: the split sweep's face buffer (in the workspace,
  // after the primitive slots); null: the single-pass sweep
  double* fbuf = nullptr;
  char err[256];
  // sweep timing (wc_sweep_timing_begin / _read)
  std::vector<cudaEvent_t> tev;
  std::vector<char> tprim;     // event pair k times a primitive-slot pass
  int tmax = 0, tcount = 0;    // sweeps to time; event pairs used
  int tsweeps = 0;             // sweeps timed
  // Phase-Field mechanism (wc_set_pf_workspace): scratch, geometry, the
  // auxiliary fields Q of the last wc_step, statistics of the last Q-map
  bool pf_bound = false;
  PfWork pw;
  PfGeom pg;
  int pf_iters = 0, pf_label_rounds = 0, pf_have_q = 0;
  double pf_resid = 0.0;
  int pf_unknowns[8] = {0};  // listed unknowns per phase of the last Q-map
  int pf_per_thread = 0;     // and the unknowns a thread kept in registers
  // host-buffer step (wc_rk_step_host): its copy stream and band events
  cudaStream_t cstream = nullptr;
  std::vector<cudaEvent_t> hev;
};

static wc_status fail(wc_grid* g, wc_status s, const char* msg) {
  if (g) snprintf(g->err, sizeof(g->err), "%s", msg);
  return s;
}

static wc_status cuda_fail(wc_grid* g, cudaError_t e, const char* where) {
  if (g) snprintf(g->err, sizeof(g->err), "%s: %s", where, cudaGetErrorString(e));
  return WC_ERR_CUDA;
}

static inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------ dispatch
#define WC_DISPATCH(N, D, EXPR)                                        \
  switch ((N) * 4 + (D)) {                                             \
    case 1 * 4 + 1: { constexpr int N_ = 1, D_ = 1; EXPR; } break;     \
    case 1 * 4 + 2: { constexpr int N_ = 1, D_ = 2; EXPR; } break;     \
    case 1 * 4 + 3: { constexpr int N_ = 1, D_ = 3; EXPR; } break;     \
    case 2 * 4 + 1: { constexpr int N_ = 2, D_ = 1; EXPR; } break;     \
    case 2 * 4 + 2: { constexpr int N_ = 2, D_ = 2; EXPR; } break;     \
    case 2 * 4 + 3: { constexpr int N_ = 2, D_ = 3; EXPR; } break;     \
    case 3 * 4 + 1: { constexpr int N_ = 3, D_ = 1; EXPR; } break;     \
    case 3 * 4 + 2: { constexpr int N_ = 3, D_ = 2; EXPR; } break;     \
    case 3 * 4 + 3: { constexpr int N_ = 3, D_ = 3; EXPR; } break;     \
    case 4 * 4 + 1: { constexpr int N_ = 4, D_ = 1; EXPR; } break;     \
    case 4 * 4 + 2: { constexpr int N_ = 4, D_ = 2; EXPR; } break;     \
    case 4 * 4 + 3: { constexpr int N_ = 4, D_ = 3; EXPR; } break;     \
    case 5 * 4 + 1: { constexpr int N_ = 5, D_ = 1; EXPR; } break;     \
    case 5 * 4 + 2: { constexpr int N_ = 5, D_ = 2; EXPR; } break;     \
    case 5 * 4 + 3: { constexpr int N_ = 5, D_ = 3; EXPR; } break;     \
    default: break;                                                    \
  }

static int grid_blocks(long n, int threads) {
  long b = (n + threads - 1) / threads;
  if (b > 148L * 64) b = 148L * 64;
  return (int)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------ init
extern "C" wc_status wc_init_grid(const wc_grid_desc* desc, wc_grid** out) {
  if (!desc || !out) return WC_ERR_ARG;
  *out = nullptr;
  const wc_grid_desc& d = *desc;
  if (d.dim < 1 || d.dim > 3) return WC_ERR_ARG;
  if (d.nphase < 1 || d.nphase > 5) return WC_ERR_UNSUPPORTED;
  for (int a = 0; a < 3; a++) {
    if (a < d.dim && (d.n[a] < 3 || !(d.dx[a] > 0.0))) return WC_ERR_ARG;
    if (a >= d.dim && d.n[a] != 1) return WC_ERR_ARG;
  }
  for (int k = 0; k < 2 * d.dim; k++)
    if (d.bc[k] < 0 || d.bc[k] > 2) return WC_ERR_ARG;
  for (int a = 0; a < d.dim; a++)
    if ((d.bc[2 * a] == WC_BC_PERIODIC) != (d.bc[2 * a + 1] == WC_BC_PERIODIC)) return WC_ERR_ARG;
  if (d.flux != WC_FLUX_HLL && d.flux != WC_FLUX_HLLC) return WC_ERR_ARG;
  if (d.precision != WC_PREC_FP64 && d.precision != WC_PREC_MIXED &&
      d.precision != WC_PREC_LEARNED)
    return WC_ERR_UNSUPPORTED;
  if (d.precision == WC_PREC_LEARNED && d.nphase > 3) return WC_ERR_UNSUPPORTED;
  if (d.seg < 0 || d.block < 0 || d.block > 128 || (d.block % 32) != 0) return WC_ERR_ARG;
  if (d.blocks_per_sm < 0 || d.blocks_per_sm > 32) return WC_ERR_ARG;
  if (d.scheme < WC_SCHEME_C || d.scheme > WC_SCHEME_JS) return WC_ERR_ARG;
  const bool comparison = d.scheme == WC_SCHEME_W || d.scheme == WC_SCHEME_JS;
  if (comparison && d.precision != WC_PREC_FP64) return WC_ERR_UNSUPPORTED;
  if (d.scheme == WC_SCHEME_JS && d.js_eps < 0.0) return WC_ERR_ARG;
  if (d.kmodel != WC_KMODEL_ALLAIRE && d.kmodel != WC_KMODEL_KAPILA) return WC_ERR_ARG;
  for (int p = 0; p < d.nphase; p++)
    if (!(d.gamma[p] > 1.0) || !(d.pinf[p] >= 0.0)) return WC_ERR_ARG;
  wc_grid* g = new (std::nothrow) wc_grid();
  if (!g) return WC_ERR_ARG;
  g->d = d;
  if (comparison) g->d.energy_limiter = 0;
  if (d.scheme == WC_SCHEME_JS && !(d.js_eps > 0.0)) g->d.js_eps = 1e-6;
  g->nv = 2 * d.nphase + d.dim + 1;
  g->ncell = (long)d.n[0] * d.n[1] * d.n[2];
  Mat& m = g->mat;
  memset(&m, 0, sizeof(m));
  m.N = d.nphase;
  m.cl = d.scheme == WC_SCHEME_CL;
  m.kapila = d.kmodel == WC_KMODEL_KAPILA;
  m.cmp = d.scheme == WC_SCHEME_W ? CMP_W : (d.scheme == WC_SCHEME_JS ? CMP_JS : CMP_NONE);
  m.js_eps = g->d.js_eps;
  for (int p = 0; p < d.nphase; p++) {
    m.A[p] = 1.0 / (d.gamma[p] - 1.0);
    m.B[p] = d.gamma[p] * d.pinf[p] / (d.gamma[p] - 1.0);
    m.D[p] = d.D[p];
    m.pinf[p] = d.pinf[p];
    m.gam[p] = d.gamma[p];
    m.Ag[p] = m.A[p] * d.gamma[p];
    m.Apmin[p] = m.A[p] * d.pmin[p];
    m.Cmin[p] = m.A[p] * d.pmin[p] + m.B[p];
    if (d.D[p] != 0.0) m.hasD = 1;
  }
  m.psi_floor = psi_face_floor(m);
  g->err[0] = 0;
  *out = g;
  return WC_OK;
}

extern "C" void wc_destroy(wc_grid* g) {
  if (!g) return;
  for (cudaEvent_t ev : g->tev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : g->hev) cudaEventDestroy(ev);
  if (g->cstream) cudaStreamDestroy(g->cstream);
  delete g;
}
extern "C" int wc_nvar(const wc_grid* g) { return g ? g->nv : 0; }
extern "C" long wc_ncell(const wc_grid* g) { return g ? g->ncell : 0; }

// Bytes of the learned weights and of the split sweep's face buffer (the
// largest direction's) in the workspace.
static size_t learned_bytes(const wc_grid* g) {
  if (g->d.precision != WC_PREC_LEARNED) return 0;
  return ((size_t)2 * MLP_NW * g->ncell * sizeof(float) + 255) / 256 * 256;
}
static size_t face_buffer_bytes(const wc_grid* g) {
  if (g->d.precision == WC_PREC_FP64 || g->d.seg > 0) return 0;
  const int K = g->nv;  // FaceBuf<N, D, float>::K: masses, fractions, velocity, pressure
  long most = 0;
  for (int d = 0; d < g->d.dim; d++) {
    const long n = g->d.n[d];
    const long b = fbuf_doubles(K, g->ncell / n, (int)n);
    if (b > most) most = b;
  }
  return ((size_t)most * sizeof(double) + 255) / 256 * 256;
}

// The primitive slots of the window schedule: Ring<N, D, double>::SLOTD = 1 +
// NV words a cell (the FP64 slot; the reduced precision's is smaller, and a
// learned grid's Phase-Field sweeps take FP64 slots).
static size_t prim_buffer_bytes(const wc_grid* g) {
  // (the segment schedule converts in its ring; a 1-D stage has one sweep,
  // whose own conversions a separate pass would not save, only relaunch)
  if (g->d.seg > 0 || g->d.dim == 1) return 0;
  return ((size_t)(1 + g->nv) * g->ncell * sizeof(double) + 255) / 256 * 256;
}
// The part of the workspace every step needs: two stage buffers, the
// direction accumulator, 256 bytes of words and the learned weights.
static size_t base_workspace_bytes(const wc_grid* g) {
  size_t state = (size_t)g->nv * g->ncell * sizeof(double);
  state = (state + 255) / 256 * 256;
  return 3 * state + 256 + learned_bytes(g);
}

extern "C" size_t wc_workspace_bytes(const wc_grid* g) {
  if (!g) return 0;
  return base_workspace_bytes(g) + prim_buffer_bytes(g) + face_buffer_bytes(g);
}

extern "C" size_t wc_prim_buffer_bytes(const wc_grid* g) { return g ? prim_buffer_bytes(g) : 0; }

extern "C" size_t wc_face_buffer_bytes(const wc_grid* g) { return g ? face_buffer_bytes(g) : 0; }

extern "C" wc_status wc_set_state(wc_grid* g, double* U_dev, void* ws, size_t ws_bytes) {
  if (!g || !U_dev) return WC_ERR_ARG;
  const bool with_faces = ws_bytes >= wc_workspace_bytes(g);
  const bool with_prim = ws_bytes >= base_workspace_bytes(g) + prim_buffer_bytes(g);
  if (ws && ws_bytes < base_workspace_bytes(g))
    return fail(g, WC_ERR_ARG, "workspace too small");
  if (ws && (reinterpret_cast<uintptr_t>(ws) & 255)) return fail(g, WC_ERR_ARG, "workspace not 256-byte aligned");
  if (reinterpret_cast<uintptr_t>(U_dev) & 7) return fail(g, WC_ERR_ARG, "state not 8-byte aligned");
  g->U = U_dev;
  g->ws = (char*)ws;
  g->ws_bytes = ws_bytes;
  if (ws) {
    size_t state = (size_t)g->nv * g->ncell * sizeof(double);
    state = (state + 255) / 256 * 256;
    g->B1 = (double*)(g->ws);
    g->B2 = (double*)(g->ws + state);
    g->Lacc = (double*)(g->ws + 2 * state);
    char* tail = g->ws + 3 * state;
    g->rate = (unsigned long long*)tail;
    g->dt = (double*)(tail + 8);
    g->status = (unsigned*)(tail + 16);
    g->ticket = (unsigned*)(tail + 32);
    g->Wbuf = g->d.precision == WC_PREC_LEARNED ? (float*)(tail + 256) : nullptr;
    g->vbuf = prim_buffer_bytes(g) && with_prim ? (double*)(tail + 256 + learned_bytes(g))
                                                : nullptr;
    g->fbuf = face_buffer_bytes(g) && with_faces
                  ? (double*)(tail + 256 + learned_bytes(g) + prim_buffer_bytes(g))
                  : nullptr;
    // the workspace comes uninitialised: clear rate, dt and the status word
    cudaError_t e = cudaMemset(tail, 0, 256);
    if (e != cudaSuccess) return cuda_fail(g, e, "workspace clear");
  } else {
    g->B1 = g->B2 = g->Lacc = nullptr;
    g->rate = nullptr;
    g->dt = nullptr;
    g->status = nullptr;
    g->ticket = nullptr;
    g->Wbuf = nullptr;
    g->vbuf = nullptr;
    g->fbuf = nullptr;
  }
  return WC_OK;
}

extern "C" wc_status wc_check_state(wc_grid* g, const double* U_dev, double sum_tol,
                                    long* nbad, long* first_bad, void* stream) {
  if (!g || !U_dev || !(sum_tol >= 0.0)) return WC_ERR_ARG;
  if (!g->ws) return fail(g, WC_ERR_STATE, "wc_check_state needs a bound workspace");
  // two counters in the workspace tail (bytes 64..79, unused by the steps)
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(g->ws + 3 * ((g->nv * g->ncell * 8 + 255) / 256 * 256) + 64);
  const unsigned long long init[2] = {0ull, ~0ull};
  cudaStream_t st = S(stream);
  cudaError_t e = cudaMemcpyAsync(bad, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(g, e, "check init");
  int blocks = grid_blocks(g->ncell, 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  WC_DISPATCH(g->d.nphase, g->d.dim,
              (k_check_state<N_, D_><<<blocks, 256, 0, st>>>(U_dev, g->ncell, g->mat, sum_tol, bad)));
  unsigned long long out[2] = {0ull, 0ull};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, bad, sizeof(out), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(g, e, "check");
  if (nbad) *nbad = (long)out[0];
  if (first_bad) *first_bad = out[0] ? (long)out[1] : -1;
  if (out[0]) {
    snprintf(g->err, sizeof(g->err), "%llu cell(s) outside the admissible set, first %llu",
             out[0], out[1]);
    return WC_ERR_INADMISSIBLE;
  }
  return WC_OK;
}

extern "C" wc_status wc_upload_state(wc_grid* g, const double* U_host, void* stream) {
  if (!g || !U_host) return WC_ERR_ARG;
  if (!g->U) return fail(g, WC_ERR_STATE, "no state bound");
  cudaError_t e = cudaMemcpyAsync(g->U, U_host, (size_t)g->nv * g->ncell * sizeof(double),
                                  cudaMemcpyHostToDevice, S(stream));
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "upload");
}

extern "C" wc_status wc_download_state(const wc_grid* g, double* U_host, void* stream) {
  if (!g || !U_host) return WC_ERR_ARG;
  if (!g->U) return WC_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(U_host, g->U, (size_t)g->nv * g->ncell * sizeof(double),
                                  cudaMemcpyDeviceToHost, S(stream));
  return e == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

extern "C" wc_status wc_prim_to_cons(const wc_grid* gc, const double* V, double* U, void* stream) {
  wc_grid* g = const_cast<wc_grid*>(gc);
  if (!g || !V || !U) return WC_ERR_ARG;
  int blocks = grid_blocks(g->ncell, 256);
  WC_DISPATCH(g->d.nphase, g->d.dim,
              (k_prim_to_cons<N_, D_><<<blocks, 256, 0, S(stream)>>>(V, U, g->ncell, g->mat)));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "prim_to_cons");
}

extern "C" wc_status wc_cons_to_prim(const wc_grid* gc, const double* U, double* V, void* stream) {
  wc_grid* g = const_cast<wc_grid*>(gc);
  if (!g || !V || !U) return WC_ERR_ARG;
  int blocks = grid_blocks(g->ncell, 256);
  WC_DISPATCH(g->d.nphase, g->d.dim,
              (k_cons_to_prim<N_, D_><<<blocks, 256, 0, S(stream)>>>(U, V, g->ncell, g->mat)));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "cons_to_prim");
}

extern "C" wc_status wc_temperature(const wc_grid* gc, const double* U, const double* cT,
                                    double* T, void* stream) {
  wc_grid* g = const_cast<wc_grid*>(gc);
  if (!g || !U || !cT || !T) return WC_ERR_ARG;
  HeatCap h;
  memset(&h, 0, sizeof(h));
  for (int p = 0; p < g->d.nphase; p++) {
    if (!(cT[p] > 0.0)) return fail(g, WC_ERR_ARG, "heat capacities must be positive");
    h.cT[p] = cT[p];
  }
  int blocks = grid_blocks(g->ncell, 256);
  WC_DISPATCH(g->d.nphase, g->d.dim,
              (k_temperature<N_, D_><<<blocks, 256, 0, S(stream)>>>(U, T, g->ncell, g->mat, h)));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "temperature");
}

// ------------------------------------------------------------------ sweeps
// Threads per sweep block: as given, else 128 for the segment march and
// WIN_BLOCK for the window sweep.
static int sweep_block(const wc_grid* g) {
  if (g->d.block > 0) return g->d.block;
  return g->d.seg > 0 ? 128 : WIN_BLOCK;
}

// Threads of one sweep launch: a whole number of blocks per SM on all 148
// SMs, so every SM sub-partition gets the same number of warps (the sweep is
// FP64-pipe bound, and the pipe is per sub-partition).
static long sweep_threads(const wc_grid* g) {
  int block = sweep_block(g);
  int bps = g->d.blocks_per_sm > 0 ? g->d.blocks_per_sm : 2;  // blocks per SM
  if (g->d.blocks_per_sm <= 0 && g->d.precision != WC_PREC_FP64) bps = 3;
  return 148L * bps * block;
}

static SweepArgs make_args(const wc_grid* g, int dir, const double* U, double* L) {
  SweepArgs a;
  memset(&a, 0, sizeof(a));
  a.U = U;
  a.L = L;
  a.ncell = g->ncell;
  a.nx = g->d.n[0];
  a.ny = g->d.n[1];
  a.nz = g->d.n[2];
  a.dir = dir;
  a.n = g->d.n[dir];
  a.stride = dir == 0 ? 1 : (dir == 1 ? (long)a.nx : (long)a.nx * a.ny);
  a.npencil = g->ncell / a.n;
  if (g->d.seg > 0) {
    // per-thread segment march of seg cells
    a.seg = g->d.seg;
    a.nseg = (a.n + a.seg - 1) / a.seg;
  } else {
    // one cell per lane, windows of WIN cells from a dynamic queue
    a.nwin = (a.n + WIN - 1) / WIN;
    a.ticket = g->ticket;
    const WinPlan w = win_plan(a.n, a.npencil);
    a.wfull = w.wfull;
    a.wtail = w.wtail;
    a.wgrp = w.wgrp;
    a.wslots = w.slots;
    a.nitems = w.nitems;
  }
  // window schedule: blocks_per_sm when given, else the occupancy limit
  a.max_threads = (g->d.seg > 0 || g->d.blocks_per_sm > 0) ? sweep_threads(g) : 0;
  a.inv_dx = 1.0 / g->d.dx[dir];
  a.bclo = g->d.bc[2 * dir];
  a.bchi = g->d.bc[2 * dir + 1];
  a.hllc = g->d.flux == WC_FLUX_HLLC;
  a.energy_limiter = g->d.energy_limiter;
  a.status = g->status;
  return a;
}

static MlpGeom mlp_geom(const wc_grid* g, int dir, const double* U) {
  MlpGeom mg;
  mg.U = U;
  mg.ncell = g->ncell;
  mg.nx = g->d.n[0];
  mg.ny = g->d.n[1];
  mg.nz = g->d.n[2];
  mg.dir = dir;
  mg.n = g->d.n[dir];
  mg.stride = dir == 0 ? 1 : (dir == 1 ? (long)mg.nx : (long)mg.nx * mg.ny);
  mg.bclo = g->d.bc[2 * dir];
  mg.bchi = g->d.bc[2 * dir + 1];
  mg.N = g->d.nphase;
  mg.nv = g->nv;
  return mg;
}

static cudaError_t launch(const wc_grid* gc, const SweepArgs& a0, cudaStream_t st) {
  wc_grid* g = const_cast<wc_grid*>(gc);
  const bool timed = g->tsweeps < g->tmax && g->tcount < 2 * g->tmax;
  if (timed) cudaEventRecord(g->tev[2 * g->tcount], st);
  cudaError_t e;
  SweepArgs a = a0;
  // the split sweep where the workspace holds its face buffer (not for the
  // comparison schemes, which are FP64)
  if (g->mat.cmp == CMP_NONE && g->d.seg == 0) a.fbuf = g->fbuf;
  if (g->d.precision == WC_PREC_LEARNED && a.kind == 0) {
    // weights of this direction from the surrogate, then the sweep
    e = launch_mlp_infer(mlp_geom(g, a.dir, a.U), g->mlp, g->Wbuf, g->status, st);
    if (e == cudaSuccess) {
      a.Wm = g->Wbuf;
      a.tau = g->tau;
      a.lcount = g->lcount;
      e = launch_sweep_learned(g->d.nphase, g->d.dim, a, g->mat, sweep_block(g), st);
    }
  } else if (g->mat.cmp != CMP_NONE)
    e = launch_sweep_compare(g->d.nphase, g->d.dim, a, g->mat, sweep_block(g), st);
  else if (g->d.precision == WC_PREC_MIXED)
    e = launch_sweep_mixed(g->d.nphase, g->d.dim, a, g->mat, sweep_block(g), st);
  else
    e = launch_sweep_fp64(g->d.nphase, g->d.dim, a, g->mat, sweep_block(g), st);
  if (timed) {
    cudaEventRecord(g->tev[2 * g->tcount + 1], st);
    g->tprim[g->tcount] = 0;
    g->tcount++;
    g->tsweeps++;
  }
  return e;
}

// The primitive slots of cells c0 .. c1 - 1 of U into the workspace, in the
// format of the sweep that reads them (kind as in launch: the FP64 and
// comparison sweeps, and a learned grid's Phase-Field sweeps, hold FP64
// slots).  Returns the slots, or null when the workspace has none (the
// sweeps then convert their cells themselves).  rate: the pass also reduces
// the CFL rate of U into g->rate (cleared by the caller), as k_max_rate does.
static const double* launch_prim(wc_grid* g, const double* U, int kind, long c0, long c1,
                                 cudaStream_t st, cudaError_t& e, bool rate = false) {
  e = cudaSuccess;
  if (!g->vbuf || g->d.seg > 0) return nullptr;
  const double i0 = 1.0 / g->d.dx[0];
  const double i1 = g->d.dim > 1 ? 1.0 / g->d.dx[1] : 0.0;
  const double i2 = g->d.dim > 2 ? 1.0 / g->d.dx[2] : 0.0;
  const bool fp64 = g->d.precision == WC_PREC_FP64 || g->mat.cmp != CMP_NONE ||
                    (g->d.precision == WC_PREC_LEARNED && kind == 1);
  const int blocks = grid_blocks(c1 - c0, 256);
  // (timed with the sweeps: their per-launch time includes each direction's
  // share of the pass)
  const bool timed = g->tsweeps < g->tmax && g->tcount < 2 * g->tmax;
  if (timed) cudaEventRecord(g->tev[2 * g->tcount], st);
  if (fp64 && rate) {
    WC_DISPATCH(g->d.nphase, g->d.dim,
                (k_prim_slots<N_, D_, double, true>
                 <<<blocks, 256, 256 * Ring<N_, D_, double>::SLOTD * 8, st>>>(
                     U, g->vbuf, g->ncell, c0, c1, g->mat, i0, i1, i2, g->rate, g->status)));
  } else if (fp64) {
    WC_DISPATCH(g->d.nphase, g->d.dim,
                (k_prim_slots<N_, D_, double><<<blocks, 256,
                                               256 * Ring<N_, D_, double>::SLOTD * 8, st>>>(
                    U, g->vbuf, g->ncell, c0, c1, g->mat)));
  } else if (rate) {
    WC_DISPATCH(g->d.nphase, g->d.dim,
                (k_prim_slots<N_, D_, float, true>
                 <<<blocks, 256, 256 * Ring<N_, D_, float>::SLOTD * 8, st>>>(
                     U, g->vbuf, g->ncell, c0, c1, g->mat, i0, i1, i2, g->rate, g->status)));
  } else {
    WC_DISPATCH(g->d.nphase, g->d.dim,
                (k_prim_slots<N_, D_, float><<<blocks, 256,
                                              256 * Ring<N_, D_, float>::SLOTD * 8, st>>>(
                    U, g->vbuf, g->ncell, c0, c1, g->mat)));
  }
  e = cudaGetLastError();
  if (timed) {
    cudaEventRecord(g->tev[2 * g->tcount + 1], st);
    g->tprim[g->tcount] = 1;
    g->tcount++;
  }
  return e == cudaSuccess ? g->vbuf : nullptr;
}

extern "C" wc_status wc_sweep_timing_begin(wc_grid* g, int max_launches) {
  if (!g || max_launches < 0 || max_launches > 100000) return WC_ERR_ARG;
  // pairs for the sweeps and as many primitive-slot passes
  while ((int)g->tev.size() < 4 * max_launches) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail(g, e, "event create");
    g->tev.push_back(ev);
  }
  g->tprim.assign(2 * (size_t)max_launches, 0);
  g->tmax = max_launches;
  g->tcount = 0;
  g->tsweeps = 0;
  return WC_OK;
}

extern "C" wc_status wc_sweep_timing_read(wc_grid* g, int* launches, double* total_ms,
                                          double* max_ms) {
  if (!g) return WC_ERR_ARG;
  int n = g->tcount;
  double tot = 0.0, mx = 0.0;
  if (n > 0) {
    cudaError_t e = cudaEventSynchronize(g->tev[2 * n - 1]);
    if (e != cudaSuccess) return cuda_fail(g, e, "event sync");
  }
  int sweeps = 0;
  for (int k = 0; k < n; k++) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, g->tev[2 * k], g->tev[2 * k + 1]);
    if (e != cudaSuccess) return cuda_fail(g, e, "event time");
    tot += ms;
    if (!g->tprim[k]) {
      sweeps++;
      if (ms > mx) mx = ms;
    }
  }
  if (launches) *launches = sweeps;
  if (total_ms) *total_ms = tot;
  if (max_ms) *max_ms = mx;
  g->tmax = 0;
  g->tcount = 0;
  g->tsweeps = 0;
  return WC_OK;
}

extern "C" wc_status wc_rhs(wc_grid* g, const double* U, double* L, void* stream) {
  if (!g || !U || !L) return WC_ERR_ARG;
  if (!g->status) return fail(g, WC_ERR_STATE, "wc_rhs needs a bound workspace (status word)");
  if (g->d.precision == WC_PREC_LEARNED && !g->mlp)
    return fail(g, WC_ERR_STATE, "learned precision needs wc_set_mlp");
  cudaError_t e;
  const double* Vs = launch_prim(g, U, 0, 0, g->ncell, S(stream), e);
  if (e != cudaSuccess) return cuda_fail(g, e, "primitive slots");
  for (int dir = 0; dir < g->d.dim; dir++) {
    SweepArgs a = make_args(g, dir, U, L);
    a.mode = dir == 0 ? 0 : 1;
    a.Vs = Vs;
    e = launch(g, a, S(stream));
    if (e != cudaSuccess) return cuda_fail(g, e, "sweep");
  }
  return WC_OK;
}

extern "C" wc_status wc_faces(wc_grid* g, int dir, const double* U, double* UL, double* UR,
                              void* stream) {
  if (!g || !U || !UL || !UR) return WC_ERR_ARG;
  if (dir < 0 || dir >= g->d.dim) return fail(g, WC_ERR_ARG, "bad direction");
  if (!g->status || !g->Lacc)
    return fail(g, WC_ERR_STATE, "wc_faces needs a bound workspace (its rhs goes there)");
  if (g->d.seg > 0) return fail(g, WC_ERR_UNSUPPORTED, "wc_faces needs the window schedule (seg = 0)");
  if (g->d.precision == WC_PREC_LEARNED && !g->mlp)
    return fail(g, WC_ERR_STATE, "learned precision needs wc_set_mlp");
  SweepArgs a = make_args(g, dir, U, g->Lacc);
  a.mode = 0;
  a.faceL = UL;
  a.faceR = UR;
  cudaError_t e = launch(g, a, S(stream));
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "face sweep");
}

extern "C" wc_status wc_rhs_pf(wc_grid* g, const double* U, const double* Q, double dt_limit,
                               double* L, void* stream) {
  if (!g || !U || !Q || !L || dt_limit < 0.0) return WC_ERR_ARG;
  if (!g->status) return fail(g, WC_ERR_STATE, "wc_rhs_pf needs a bound workspace (status word)");
  cudaError_t e0;
  const double* Vs = launch_prim(g, U, 1, 0, g->ncell, S(stream), e0);
  if (e0 != cudaSuccess) return cuda_fail(g, e0, "primitive slots");
  for (int dir = 0; dir < g->d.dim; dir++) {
    SweepArgs a = make_args(g, dir, U, L);
    a.mode = dir == 0 ? 0 : 1;
    a.Vs = Vs;
    a.kind = 1;
    a.Q = Q;
    a.gmax = dt_limit > 0.0 ? g->d.dx[dir] / (12.0 * g->d.dim * dt_limit) : 0.0;
    cudaError_t e = launch(g, a, S(stream));
    if (e != cudaSuccess) return cuda_fail(g, e, "pf sweep");
  }
  return WC_OK;
}

static wc_status clear_rate(wc_grid* g, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g->rate, 0, sizeof(unsigned long long), st);
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "memset");
}

static wc_status launch_rate(wc_grid* g, const double* U, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g->rate, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(g, e, "memset");
  int blocks = grid_blocks(g->ncell, 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  double i0 = 1.0 / g->d.dx[0];
  double i1 = g->d.dim > 1 ? 1.0 / g->d.dx[1] : 0.0;
  double i2 = g->d.dim > 2 ? 1.0 / g->d.dx[2] : 0.0;
  WC_DISPATCH(g->d.nphase, g->d.dim,
              (k_max_rate<N_, D_><<<blocks, 256, 0, st>>>(U, g->ncell, g->mat, i0, i1, i2,
                                                          g->rate, g->status)));
  e = cudaGetLastError();
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "max_rate");
}

extern "C" wc_status wc_compute_dt(wc_grid* g, double cfl, double* dt_dev, void* stream) {
  if (!g || !dt_dev || !(cfl > 0.0)) return WC_ERR_ARG;
  if (!g->U || !g->ws) return fail(g, WC_ERR_STATE, "state/workspace not bound");
  wc_status s = launch_rate(g, g->U, S(stream));
  if (s) return s;
  k_dt_from_rate<<<1, 32, 0, S(stream)>>>((const double*)g->rate, cfl, dt_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "dt");
}

// Band hooks of the host-buffer step (wc_rk_step_host): the first
// direction's sweep runs as nb launches over consecutive pencils, band b
// after the copy stream's event up[b] (its rows uploaded), then the time
// step's rate from the whole state; or the last direction's sweep runs as nb
// launches, event done[b] recorded after band b (its cells final).
struct HostBands {
  int nb = 0;
  const cudaEvent_t* up = nullptr;
  cudaEvent_t* done = nullptr;
};

// Pencils t0 .. t1 - 1 of band b of nb over np pencils.  The band whose copy
// nothing hides is small (np / 32): the first one of an upload (small < 0;
// the sweep waits for it) and the last one of a download (small > 0; the
// step ends with it); the others share the rest evenly.
static long band_edge(long np, int nb, int e, int small) {
  if (nb < 2) return e == 0 ? 0 : np;
  long s = np / 32;
  if (s < 1) s = 1;
  if (small < 0) return e == 0 ? 0 : s + (np - s) * (e - 1) / (nb - 1);
  return e == nb ? np : (np - s) * e / (nb - 1);
}
static void band_range(long np, int nb, int b, int small, long& t0, long& t1) {
  t0 = band_edge(np, nb, b, small);
  t1 = band_edge(np, nb, b + 1, small);
}

// One SSP-RK3 stage: dst = r0 U0 + r1 src + r2 dt L(src); L of Eq. 3, or of
// Eq. 5 with the auxiliary fields Q (kind 1; face gradients limited to
// dx / (12 d dt), reading R17).
static wc_status stage(wc_grid* g, const double* src, double* dst, double r0, double r1,
                       double r2, double cfl, double dt_fixed, cudaStream_t st, int kind = 0,
                       const double* Q = nullptr, const HostBands* hb = nullptr,
                       bool rate = false) {
  int D = g->d.dim;
  // directions x, y, z; a 2-D stage whose last sweep is banded for the
  // download takes y first, so that the banded sweep runs over rows (x
  // pencils, contiguous in every field): L_y + L_x is L_x + L_y bit for bit
  const bool swap = hb && hb->done && D == 2;
  // the primitive slots of src, once for the stage's directions (band by
  // band with the first direction when the upload is still arriving)
  const double* Vs = nullptr;
  const bool banded_up = hb && hb->up;
  if (!banded_up) {
    cudaError_t e;
    Vs = launch_prim(g, src, kind, 0, g->ncell, st, e, rate);
    if (e != cudaSuccess) return cuda_fail(g, e, "primitive slots");
  }
  for (int k = 0; k < D; k++) {
    const int dir = swap ? 1 - k : k;
    SweepArgs a = make_args(g, dir, src, g->Lacc);
    a.Vs = Vs;
    if (kind == 1) {
      a.kind = 1;
      a.Q = Q;
      a.gcoef = g->d.dx[dir] / (12.0 * g->d.dim);
    }
    a.U0 = g->U;
    a.Uout = dst;
    a.rate = (const double*)g->rate;
    a.cfl = cfl;
    a.dt_fixed = dt_fixed;
    a.rk0 = r0;
    a.rk1 = r1;
    a.rk2 = r2;
    if (D == 1) a.mode = 3;
    else a.mode = k == 0 ? 0 : (k < D - 1 ? 1 : 2);
    const bool up = hb && hb->up && k == 0, down = hb && hb->done && k == D - 1;
    if (!up && !down) {
      cudaError_t e = launch(g, a, st);
      if (e != cudaSuccess) return cuda_fail(g, e, "sweep");
      continue;
    }
    // (band launches: the window plan of each band's pencils; the split
    // sweep's face buffer is indexed by the band's own pencils in both passes)
    // An upload band (rows of x-pencils, cells t0 nx .. t1 nx - 1, whose
    // stencils stay in their rows) takes its rows' primitive slots, and the
    // CFL rate over them, once they have arrived; the first direction (mode
    // 0) needs no time step, the others read the rate of the whole state.
    const bool band_rate = up && g->vbuf && !(dt_fixed > 0.0);
    if (band_rate) {
      wc_status r = clear_rate(g, st);
      if (r) return r;
    }
    for (int b = 0; b < hb->nb; b++) {
      long t0, t1;
      band_range(a.npencil, hb->nb, b, up ? -1 : 1, t0, t1);
      SweepArgs ab = a;
      ab.tr0 = t0;
      ab.npencil = t1 - t0;
      const WinPlan w = win_plan(ab.n, ab.npencil);
      ab.nitems = w.nitems;
      ab.wslots = w.slots;
      cudaError_t e = up ? cudaStreamWaitEvent(st, hb->up[b], 0) : cudaSuccess;
      if (e == cudaSuccess && up)
        ab.Vs = launch_prim(g, src, kind, t0 * (long)ab.n, t1 * (long)ab.n, st, e, band_rate);
      if (e == cudaSuccess) e = launch(g, ab, st);
      if (e == cudaSuccess && down) e = cudaEventRecord(hb->done[b], st);
      if (e != cudaSuccess) return cuda_fail(g, e, "band sweep");
    }
    if (up && !g->vbuf && !(dt_fixed > 0.0)) {
      wc_status r = launch_rate(g, g->U, st);
      if (r) return r;
    }
    if (up) Vs = g->vbuf && g->d.seg == 0 ? g->vbuf : nullptr;
  }
  return WC_OK;
}

extern "C" wc_status wc_rk_step(wc_grid* g, double cfl, double dt_fixed, int nsteps,
                                double* dt_host, void* stream) {
  if (!g || nsteps < 0) return WC_ERR_ARG;
  if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(g, WC_ERR_ARG, "need cfl > 0 or dt > 0");
  if (!g->U || !g->ws) return fail(g, WC_ERR_STATE, "state/workspace not bound");
  if (g->d.precision == WC_PREC_LEARNED && !g->mlp)
    return fail(g, WC_ERR_STATE, "learned precision needs wc_set_mlp");
  cudaStream_t st = S(stream);
  // the CFL rate of U^n: in the first stage's primitive-slot pass when the
  // workspace holds the slots (the state is read and converted once), else
  // by k_max_rate
  const bool fuse = !(dt_fixed > 0.0) && g->vbuf;
  for (int s = 0; s < nsteps; s++) {
    if (!(dt_fixed > 0.0)) {
      wc_status r = fuse ? clear_rate(g, st) : launch_rate(g, g->U, st);
      if (r) return r;
    }
    wc_status r;
    if ((r = stage(g, g->U, g->B1, 0.0, 1.0, 1.0, cfl, dt_fixed, st, 0, nullptr, nullptr, fuse)))
      return r;
    if ((r = stage(g, g->B1, g->B2, 0.75, 0.25, 0.25, cfl, dt_fixed, st))) return r;
    if ((r = stage(g, g->B2, g->U, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, cfl, dt_fixed, st))) return r;
  }
  if (dt_host) {
    if (dt_fixed > 0.0) {
      *dt_host = dt_fixed;
    } else {
      double rate = 0.0;
      cudaError_t e = cudaMemcpyAsync(&rate, g->rate, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(g, e, "dt readback");
      *dt_host = cfl / rate;
    }
  }
  return WC_OK;
}

// ------------------------------------------------------------------ host buffers
// Bands of the host-buffer step's overlapped sweeps.
static constexpr int kHostBands = 8;

static wc_status host_resources(wc_grid* g) {
  if (!g->cstream) {
    cudaError_t e = cudaStreamCreateWithFlags(&g->cstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      g->cstream = nullptr;
      return cuda_fail(g, e, "copy stream");
    }
  }
  while ((int)g->hev.size() < 2 * kHostBands + 2) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(g, e, "event");
    g->hev.push_back(ev);
  }
  return WC_OK;
}

extern "C" wc_status wc_rk_step_host(wc_grid* g, const double* U_in_host, double* U_out_host,
                                     double cfl, double dt_fixed, int nsteps, void* stream) {
  if (!g || !U_in_host || !U_out_host || nsteps < 1) return WC_ERR_ARG;
  if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(g, WC_ERR_ARG, "need cfl > 0 or dt > 0");
  if (!g->U || !g->ws) return fail(g, WC_ERR_STATE, "state/workspace not bound");
  if (g->d.precision == WC_PREC_LEARNED && !g->mlp)
    return fail(g, WC_ERR_STATE, "learned precision needs wc_set_mlp");
  cudaStream_t st = S(stream);
  const size_t nv = (size_t)g->nv, nc = (size_t)g->ncell;
  const int D = g->d.dim;
  // overlap needs a second direction after the banded first one and the
  // window schedule; the learned weights come from one inference over the
  // whole state per direction, so that precision runs the steps unbanded
  if (D == 1 || g->d.seg > 0 || g->d.precision == WC_PREC_LEARNED) {
    wc_status r = wc_upload_state(g, U_in_host, stream);
    if (!r) r = wc_rk_step(g, cfl, dt_fixed, nsteps, nullptr, stream);
    if (!r) r = wc_download_state(g, U_out_host, stream);
    return r;
  }
  wc_status r = host_resources(g);
  if (r) return r;
  cudaStream_t cs = g->cstream;
  cudaEvent_t* up = g->hev.data();
  cudaEvent_t* done = up + kHostBands;
  cudaEvent_t start = up[2 * kHostBands], fin = up[2 * kHostBands + 1];
  // first-direction bands: rows of x-pencils, contiguous in every field
  const int n0 = g->d.n[0];
  const long np0 = g->ncell / n0;
  const int nb0 = np0 < kHostBands ? (int)np0 : kHostBands;
  // last-sweep bands: rows of x-pencils in 2-D (the last stage takes y
  // first); in 3-D z-pencils tr0 .. tr1 - 1, which hold the cells tr + k P
  // (k < nz, P = nx ny), a strided block of rows of (tr1 - tr0) values
  const int dl = D == 2 ? 0 : D - 1;
  const int nl = g->d.n[dl];
  const long npl = g->ncell / nl;
  const int nbl = npl < kHostBands ? (int)npl : kHostBands;
  // the upload waits for the work already on the caller's stream
  cudaError_t e = cudaEventRecord(start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, start, 0);
  for (int b = 0; b < nb0 && e == cudaSuccess; b++) {
    long t0, t1;
    band_range(np0, nb0, b, -1, t0, t1);
    const size_t off = (size_t)t0 * n0, cnt = (size_t)(t1 - t0) * n0;
    for (size_t v = 0; v < nv && e == cudaSuccess; v++)
      e = cudaMemcpyAsync(g->U + v * nc + off, U_in_host + v * nc + off, cnt * sizeof(double),
                          cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(up[b], cs);
  }
  if (e != cudaSuccess) return cuda_fail(g, e, "band upload");
  HostBands hu, hd;
  hu.nb = nb0;
  hu.up = up;
  hd.nb = nbl;
  hd.done = done;
  const bool fuse = !(dt_fixed > 0.0) && g->vbuf;
  for (int s = 0; s < nsteps; s++) {
    const bool first = s == 0, last = s == nsteps - 1;
    // (the first step's rate comes with its banded upload; later steps take
    // it in the first stage's slot pass, as wc_rk_step does)
    if (!first && !(dt_fixed > 0.0)) {
      r = fuse ? clear_rate(g, st) : launch_rate(g, g->U, st);
      if (r) return r;
    }
    if ((r = stage(g, g->U, g->B1, 0.0, 1.0, 1.0, cfl, dt_fixed, st, 0, nullptr,
                   first ? &hu : nullptr, fuse && !first)))
      return r;
    if ((r = stage(g, g->B1, g->B2, 0.75, 0.25, 0.25, cfl, dt_fixed, st))) return r;
    if ((r = stage(g, g->B2, g->U, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, cfl, dt_fixed, st, 0,
                   nullptr, last ? &hd : nullptr)))
      return r;
  }
  for (int b = 0; b < nbl && e == cudaSuccess; b++) {
    long t0, t1;
    band_range(npl, nbl, b, 1, t0, t1);
    e = cudaStreamWaitEvent(cs, done[b], 0);
    if (dl == 0) {
      const size_t off = (size_t)t0 * nl, cnt = (size_t)(t1 - t0) * nl;
      for (size_t v = 0; v < nv && e == cudaSuccess; v++)
        e = cudaMemcpyAsync(U_out_host + v * nc + off, g->U + v * nc + off,
                            cnt * sizeof(double), cudaMemcpyDeviceToHost, cs);
    } else {
      const size_t pitch = (size_t)npl * sizeof(double);
      for (size_t v = 0; v < nv && e == cudaSuccess; v++)
        e = cudaMemcpy2DAsync(U_out_host + v * nc + t0, pitch, g->U + v * nc + t0, pitch,
                              (size_t)(t1 - t0) * sizeof(double), (size_t)nl,
                              cudaMemcpyDeviceToHost, cs);
    }
  }
  // the caller's stream covers the downloads
  if (e == cudaSuccess) e = cudaEventRecord(fin, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fin, 0);
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "band download");
}

// ------------------------------------------------------------------ Phase-Field mechanism
static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

extern "C" size_t wc_pf_workspace_bytes(const wc_grid* g) {
  if (!g) return 0;
  const size_t f = align256(sizeof(double) * (size_t)g->d.nphase * g->ncell);
  const size_t li = align256(sizeof(int) * (size_t)g->d.nphase * g->ncell);
  // R c D 1/D sumR sumD x r p q xk pd sd, three face-weight fields, labels,
  // the unknowns' list and its inverse, partials, scalars, flags
  return 16 * f + 3 * li + align256(sizeof(double) * pf_part_doubles()) + 512 + 256;
}

extern "C" wc_status wc_set_pf_workspace(wc_grid* g, void* ws_dev, size_t bytes) {
  if (!g || !ws_dev) return WC_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(ws_dev) & 255) != 0) return fail(g, WC_ERR_ARG, "workspace not 256-byte aligned");
  if (bytes < wc_pf_workspace_bytes(g)) return fail(g, WC_ERR_ARG, "pf workspace too small");
  if (g->ncell > 2147483647L / 2) return fail(g, WC_ERR_UNSUPPORTED, "pf mechanism: grid too large");
  const size_t f = align256(sizeof(double) * (size_t)g->d.nphase * g->ncell);
  const size_t li = align256(sizeof(int) * (size_t)g->d.nphase * g->ncell);
  char* w = static_cast<char*>(ws_dev);
  double** fields[] = {&g->pw.R, &g->pw.c, &g->pw.D, &g->pw.Dinv, &g->pw.sumR, &g->pw.sumD,
                       &g->pw.x, &g->pw.r, &g->pw.p, &g->pw.q, &g->pw.xk, &g->pw.pd,
                       &g->pw.sd};
  for (double** d : fields) {
    *d = reinterpret_cast<double*>(w);
    w += f;
  }
  g->pw.w = reinterpret_cast<double*>(w);  // [3][N][ncell]
  w += 3 * f;
  g->pw.lab = reinterpret_cast<int*>(w);
  w += li;
  g->pw.idx = reinterpret_cast<int*>(w);
  w += li;
  g->pw.pos = reinterpret_cast<int*>(w);
  w += li;
  g->pw.part = reinterpret_cast<double*>(w);
  w += align256(sizeof(double) * pf_part_doubles());
  g->pw.scal = reinterpret_cast<double*>(w);  // 64 doubles
  w += 512;
  g->pw.flag = reinterpret_cast<int*>(w);
  // the tickets of the reducing CG kernels start at zero (and return to it)
  cudaError_t e0 = cudaMemset(g->pw.flag, 0, 256);
  if (e0 != cudaSuccess) return cuda_fail(g, e0, "pf workspace flags");
  PfGeom& pg = g->pg;
  pg.nx = g->d.n[0];
  pg.ny = g->d.n[1];
  pg.nz = g->d.n[2];
  pg.dim = g->d.dim;
  for (int a = 0; a < 3; a++) {
    pg.per[a] = a < g->d.dim && g->d.bc[2 * a] == WC_BC_PERIODIC;
    pg.idx2[a] = a < g->d.dim ? 1.0 / (g->d.dx[a] * g->d.dx[a]) : 0.0;
  }
  pg.ncell = g->ncell;
  pg.N = g->d.nphase;
  pg.nv = g->nv;
  pg.a0 = g->d.nphase + g->d.dim + 1;
  g->pf_bound = true;
  g->pf_have_q = 0;
  return WC_OK;
}

static double cell_volume(const wc_grid* g) {
  double v = 1.0;
  for (int a = 0; a < g->d.dim; a++) v *= g->d.dx[a];
  return v;
}

extern "C" wc_status wc_cac_rhs(wc_grid* g, const double* U, double eta, double M, double* R,
                                void* stream) {
  if (!g || !U) return WC_ERR_ARG;
  if (!g->pf_bound) return fail(g, WC_ERR_STATE, "wc_cac_rhs needs wc_set_pf_workspace");
  const double et = eta > 0.0 ? eta : g->d.dx[0];
  cudaStream_t st = S(stream);
  cudaError_t e = pf_cac(U, g->pg, g->pw, cell_volume(g), et, M, st);
  if (e == cudaSuccess && R && R != g->pw.R)
    e = cudaMemcpyAsync(R, g->pw.R, sizeof(double) * (size_t)g->d.nphase * g->ncell,
                        cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "cac_rhs");
}

// Eq. 4 for the fractions of U and the right-hand sides R ([N][ncell];
// null: those of the last wc_cac_rhs); Q receives the solution (and holds
// the start when warm); Q may be the iterate buffer itself.
static wc_status qmap(wc_grid* g, const double* U, const double* R, double* Q, double tol,
                      int maxit, int warm, cudaStream_t st) {
  const size_t fb = sizeof(double) * (size_t)g->d.nphase * g->ncell;
  cudaError_t e = cudaSuccess;
  if (R && R != g->pw.R) e = cudaMemcpyAsync(g->pw.R, R, fb, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && warm && Q != g->pw.x)
    e = cudaMemcpyAsync(g->pw.x, Q, fb, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = pf_qmap_setup(U, g->pg, g->pw, st);
  if (e != cudaSuccess) return cuda_fail(g, e, "qmap setup");
  e = pf_qmap_solve(g->pg, g->pw, warm, tol * tol, maxit, st);
  if (e != cudaSuccess) return cuda_fail(g, e, "qmap cg");
  const int N = g->d.nphase;
  int flags[32] = {0};
  double sc[32];
  e = cudaMemcpyAsync(flags, g->pw.flag, sizeof(flags), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc, g->pw.scal, sizeof(sc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(g, e, "qmap residual");
  if (flags[10]) return fail(g, WC_ERR_TIMEOUT, "qmap: a grid barrier wait gave up");
  if (flags[24]) return fail(g, WC_ERR_STATE, "qmap labels did not settle");
  g->pf_label_rounds = flags[23];
  if (Q != g->pw.x) {
    e = cudaMemcpyAsync(Q, g->pw.x, fb, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(g, e, "qmap result");
  }
  double res = 0.0;  // sqrt(r.r/D / b.b/D): the D-weighted residual relative to b
  for (int p = 0; p < N; p++)
    if (sc[16 + p] > 0.0) res = fmax(res, sqrt(fmax(sc[24 + p], 0.0) / sc[16 + p]));
  const int it = flags[11];
  for (int p = 0; p < N; p++) g->pf_unknowns[p] = flags[12 + p];
  g->pf_per_thread = flags[17];
  g->pf_iters = it;
  g->pf_resid = res;
  return WC_OK;
}

extern "C" wc_status wc_qmap(wc_grid* g, const double* U, const double* R, double* Q, double tol,
                             int maxit, int warm, int* iters, double* resid, void* stream) {
  if (!g || !U || !Q || !(tol > 0.0) || maxit < 1) return WC_ERR_ARG;
  if (!g->pf_bound) return fail(g, WC_ERR_STATE, "wc_qmap needs wc_set_pf_workspace");
  wc_status s = qmap(g, U, R, Q, tol, maxit, warm, S(stream));
  if (s) return s;
  if (iters) *iters = g->pf_iters;
  if (resid) *resid = g->pf_resid;
  return WC_OK;
}

// SSP-RK3 of Eq. 5 on the bound state with Q fixed (time step dt_fixed, or
// cfl over the rate of the last hyperbolic step on the device).
static wc_status pf_stages(wc_grid* g, const double* Q, double cfl, double dt_fixed,
                           cudaStream_t st) {
  wc_status r;
  if ((r = stage(g, g->U, g->B1, 0.0, 1.0, 1.0, cfl, dt_fixed, st, 1, Q))) return r;
  if ((r = stage(g, g->B1, g->B2, 0.75, 0.25, 0.25, cfl, dt_fixed, st, 1, Q))) return r;
  return stage(g, g->B2, g->U, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, cfl, dt_fixed, st, 1, Q);
}

extern "C" wc_status wc_pf_step(wc_grid* g, const double* Q, double dt, void* stream) {
  if (!g || !Q || !(dt > 0.0)) return WC_ERR_ARG;
  if (!g->U || !g->ws) return fail(g, WC_ERR_STATE, "state/workspace not bound");
  return pf_stages(g, Q, 0.0, dt, S(stream));
}

extern "C" wc_status wc_step(wc_grid* g, double cfl, double dt_fixed, int nsteps, double tol,
                             int maxit, double* dt_host, void* stream) {
  if (!g || nsteps < 0 || !(tol > 0.0) || maxit < 1) return WC_ERR_ARG;
  if (!g->pf_bound) return fail(g, WC_ERR_STATE, "wc_step needs wc_set_pf_workspace");
  cudaStream_t st = S(stream);
  for (int s = 0; s < nsteps; s++) {
    wc_status r = wc_rk_step(g, cfl, dt_fixed, 1, nullptr, stream);
    if (r) return r;
    cudaError_t e = pf_cac(g->U, g->pg, g->pw, cell_volume(g), g->d.dx[0], -1.0, st);
    if (e != cudaSuccess) return cuda_fail(g, e, "cac_rhs");
    // Q in the iterate buffer, started from the previous step's Q
    if ((r = qmap(g, g->U, nullptr, g->pw.x, tol, maxit, g->pf_have_q, st))) return r;
    g->pf_have_q = 1;
    if ((r = pf_stages(g, g->pw.x, cfl, dt_fixed, st))) return r;
  }
  if (dt_host) {
    if (dt_fixed > 0.0) {
      *dt_host = dt_fixed;
    } else {
      double rate = 0.0;
      cudaError_t e = cudaMemcpyAsync(&rate, g->rate, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(g, e, "dt readback");
      *dt_host = cfl / rate;
    }
  }
  return WC_OK;
}

extern "C" wc_status wc_pf_stats(const wc_grid* g, int* cg_iters, int* label_rounds,
                                 double* resid) {
  if (!g) return WC_ERR_ARG;
  if (cg_iters) *cg_iters = g->pf_iters;
  if (label_rounds) *label_rounds = g->pf_label_rounds;
  if (resid) *resid = g->pf_resid;
  return WC_OK;
}

extern "C" wc_status wc_pf_band(const wc_grid* g, int* unknowns, int* per_thread) {
  if (!g) return WC_ERR_ARG;
  if (unknowns)
    for (int p = 0; p < g->d.nphase; p++) unknowns[p] = g->pf_unknowns[p];
  if (per_thread) *per_thread = g->pf_per_thread;
  return WC_OK;
}

extern "C" const double* wc_pf_q(const wc_grid* g) { return g && g->pf_bound ? g->pw.x : nullptr; }

extern "C" wc_status wc_limit(const wc_grid* gc, int dir, long ncell, const double* Ubar,
                              const double* VL, const double* VR, double* UL, double* UR,
                              double* theta, void* stream) {
  wc_grid* g = const_cast<wc_grid*>(gc);
  if (!g || !Ubar || !VL || !VR || !UL || !UR || ncell < 0) return WC_ERR_ARG;
  if (dir < 0 || dir >= g->d.dim) return fail(g, WC_ERR_ARG, "bad direction");
  if (ncell == 0) return WC_OK;
  int blocks = grid_blocks(ncell, 128);
  WC_DISPATCH(g->d.nphase, g->d.dim,
              (k_limit<N_, D_><<<blocks, 128, 0, S(stream)>>>(Ubar, VL, VR, UL, UR, theta, ncell,
                                                              g->mat, g->d.energy_limiter)));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "limit");
}

extern "C" wc_status wc_sync_status(wc_grid* g, void* stream) {
  if (!g) return WC_ERR_ARG;
  if (!g->status) return WC_ERR_STATE;
  unsigned st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, g->status, sizeof(unsigned), cudaMemcpyDeviceToHost, S(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
  if (e == cudaSuccess) e = cudaMemsetAsync(g->status, 0, sizeof(unsigned), S(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
  if (e != cudaSuccess) return cuda_fail(g, e, "status");
  if (st & ST_INADMISSIBLE) return fail(g, WC_ERR_INADMISSIBLE, "inadmissible state met by a kernel");
  if (st & ST_NAN) return fail(g, WC_ERR_NAN, "non-finite value produced by a kernel");
  if (st & 4u) return fail(g, WC_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel ran out");
  return WC_OK;
}

extern "C" void wc_last_error(const wc_grid* g, char* buf, size_t n) {
  if (!buf || n == 0) return;
  snprintf(buf, n, "%s", g ? g->err : "null grid");
}

// ------------------------------------------------------------------ learned weights
extern "C" wc_status wc_set_mlp(wc_grid* g, const void* params_dev, float tau,
                                unsigned long long* counters_dev) {
  if (!g) return WC_ERR_ARG;
  if (g->d.precision != WC_PREC_LEARNED)
    return fail(g, WC_ERR_STATE, "wc_set_mlp needs a grid of precision WC_PREC_LEARNED");
  if (params_dev && (reinterpret_cast<uintptr_t>(params_dev) & 15))
    return fail(g, WC_ERR_ARG, "parameter block not 16-byte aligned");
  if (!(tau >= 0.0f) || !(tau <= 1.0f)) return fail(g, WC_ERR_ARG, "tau outside [0, 1]");
  g->mlp = params_dev;
  g->tau = tau;
  g->lcount = counters_dev;
  return WC_OK;
}

extern "C" wc_status wc_mlp_infer(const wc_grid* gc, const double* U_dev, int dir,
                                  const void* params_dev, float* W_dev, unsigned* status_dev,
                                  void* stream) {
  wc_grid* g = const_cast<wc_grid*>(gc);
  if (!g || !U_dev || !params_dev || !W_dev || !status_dev) return WC_ERR_ARG;
  if (dir < 0 || dir >= g->d.dim) return fail(g, WC_ERR_ARG, "bad direction");
  if (g->d.nphase > 3) return fail(g, WC_ERR_UNSUPPORTED, "the surrogate takes N <= 3");
  if (reinterpret_cast<uintptr_t>(params_dev) & 15)
    return fail(g, WC_ERR_ARG, "parameter block not 16-byte aligned");
  cudaError_t e = launch_mlp_infer(mlp_geom(g, dir, U_dev), params_dev, W_dev, status_dev,
                                   S(stream));
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "mlp infer");
}

extern "C" wc_status wc_mlp_features(const wc_grid* gc, const double* U_dev, int dir, long row0,
                                     void* X_dev, float* T_dev, long* list_dev,
                                     unsigned long long* count_dev, long list_cap,
                                     void* stream) {
  wc_grid* g = const_cast<wc_grid*>(gc);
  if (!g || !U_dev || !X_dev || row0 < 0 || list_cap < 0) return WC_ERR_ARG;
  if (list_dev && !count_dev) return fail(g, WC_ERR_ARG, "list needs a counter");
  if (dir < 0 || dir >= g->d.dim) return fail(g, WC_ERR_ARG, "bad direction");
  if (g->d.nphase > 3) return fail(g, WC_ERR_UNSUPPORTED, "the surrogate takes N <= 3");
  if (reinterpret_cast<uintptr_t>(X_dev) & 15) return fail(g, WC_ERR_ARG, "X not 16-byte aligned");
  cudaError_t e = launch_mlp_features(mlp_geom(g, dir, U_dev), row0,
                                      reinterpret_cast<__nv_bfloat16*>(X_dev), T_dev, list_dev,
                                      count_dev, list_cap, S(stream));
  return e == cudaSuccess ? WC_OK : cuda_fail(g, e, "mlp features");
}

// ------------------------------------------------------------------ FP64 peak probe
__global__ void k_fp64_peak(int iters, double* sink) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  const double a = 0.999999, b = 1e-7;
  for (int i = 0; i < iters; i++) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 12345.678) sink[0] = s;  // keeps the loop alive
}

extern "C" wc_status wc_fp64_peak_kernel(int blocks, int threads, int iters, double* sink,
                                         double* flops, void* stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !sink) return WC_ERR_ARG;
  k_fp64_peak<<<blocks, threads, 0, S(stream)>>>(iters, sink);
  if (flops) *flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  return cudaGetLastError() == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

// ------------------------------------------------------------------ grid barrier check
extern "C" wc_status wc_grid_barrier_check(int* words, int skip_block, int rounds, void* stream) {
  if (!words || rounds < 1 || skip_block < -1) return WC_ERR_ARG;
  cudaStream_t st = S(stream);
  cudaError_t e = pf_barrier_check(words, skip_block, rounds, st);
  int h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, words, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return WC_ERR_CUDA;
  return h[2] ? WC_ERR_TIMEOUT : WC_OK;
}

extern "C" size_t wc_neighbour_barrier_words(void) { return pf_nbr_check_words(); }

extern "C" wc_status wc_neighbour_barrier_check(int* words, size_t nwords, int skip_block,
                                                int span, int rounds, void* stream) {
  if (!words || rounds < 1 || skip_block < -1 || span < 1) return WC_ERR_ARG;
  const size_t need = pf_nbr_check_words();
  if (need == 0) return WC_ERR_CUDA;
  if (nwords < need) return WC_ERR_ARG;
  cudaStream_t st = S(stream);
  cudaError_t e = pf_nbr_check(words, skip_block, span, rounds, st);
  int h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, words, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return WC_ERR_CUDA;
  return h[2] ? WC_ERR_TIMEOUT : WC_OK;
}

// ------------------------------------------------------------------ conversion check
__global__ void k_convert_f32(const double* x, float* f, double* back, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const float v = f64_to_f32(x[i]);
    f[i] = v;
    back[i] = f32_to_f64(v);
  }
}

extern "C" wc_status wc_convert_f32(const double* x, float* f, double* back, long n,
                                    void* stream) {
  if (n < 0 || (n > 0 && (!x || !f || !back))) return WC_ERR_ARG;
  if (n == 0) return WC_OK;
  const long blocks = (n + 255) / 256 < 148L * 8 ? (n + 255) / 256 : 148L * 8;
  k_convert_f32<<<(unsigned)blocks, 256, 0, S(stream)>>>(x, f, back, n);
  return cudaGetLastError() == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

// ------------------------------------------------------------------ fixed-scratch stepping
// Used by wc_rk_step_noalloc (wenoc_noalloc.cu): runs wc_rk_step on state U
// with the stage buffers, accumulator, rate and status words placed in the
// given scratch area (same layout as the bound workspace), then restores the
// grid's own bindings.  Returns the device address of the status word used.
wc_status wc_internal_scratch_supported(wc_grid* g) {
  if (g->d.precision == WC_PREC_LEARNED)
    return fail(g, WC_ERR_UNSUPPORTED, "the fixed scratch holds no learned-weight buffer");
  return WC_OK;
}

wc_status wc_internal_rk_with_scratch(wc_grid* g, double* U, char* scratch, double cfl,
                                      double dt_fixed, int nsteps, cudaStream_t st,
                                      unsigned** status_out) {
  const wc_status sup = wc_internal_scratch_supported(g);
  if (sup != WC_OK) return sup;
  // save and restore only the bindings (the grid also owns timing events)
  struct Bind {
    double* U; char* ws; size_t ws_bytes; double *B1, *B2, *Lacc;
    unsigned long long* rate; double* dt; unsigned* status; unsigned* ticket; double* vbuf;
    double* fbuf;
  } saved{g->U,    g->ws, g->ws_bytes, g->B1,     g->B2,   g->Lacc,
          g->rate, g->dt, g->status,   g->ticket, g->vbuf, g->fbuf};
  size_t state = (size_t)g->nv * g->ncell * sizeof(double);
  state = (state + 255) / 256 * 256;
  char* tail = scratch + 3 * state;
  cudaError_t e = cudaMemsetAsync(tail, 0, 256, st);
  if (e != cudaSuccess) return cuda_fail(g, e, "scratch clear");
  g->U = U;
  g->ws = scratch;
  g->ws_bytes = 3 * state + 256;
  g->B1 = (double*)scratch;
  g->B2 = (double*)(scratch + state);
  g->Lacc = (double*)(scratch + 2 * state);
  g->rate = (unsigned long long*)tail;
  g->dt = (double*)(tail + 8);
  g->status = (unsigned*)(tail + 16);
  g->ticket = (unsigned*)(tail + 32);
  g->vbuf = nullptr;  // the sweeps convert their cells (no primitive slots in the scratch)
  g->fbuf = nullptr;  // the single-pass sweep (no face buffer in the scratch)
  wc_status r = wc_rk_step(g, cfl, dt_fixed, nsteps, nullptr, reinterpret_cast<void*>(st));
  if (status_out) *status_out = g->status;
  g->U = saved.U;
  g->ws = saved.ws;
  g->ws_bytes = saved.ws_bytes;
  g->B1 = saved.B1;
  g->B2 = saved.B2;
  g->Lacc = saved.Lacc;
  g->rate = saved.rate;
  g->dt = saved.dt;
  g->status = saved.status;
  g->ticket = saved.ticket;
  g->vbuf = saved.vbuf;
  g->fbuf = saved.fbuf;
  return r;
}

void wc_internal_set_error(wc_grid* g, const char* msg) { fail(g, WC_ERR_ARG, msg); }
