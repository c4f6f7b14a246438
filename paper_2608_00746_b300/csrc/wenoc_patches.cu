// wenoc_patches.cu -- host side of the batched-patch executor: patch table,
// one persistent launch per Runge-Kutta stage, CUDA-graph capture of a whole
// step, and the schedule autotuner.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/wenoc.h"
#include "wenoc_kernels.cuh"
#include "wenoc_patches.cuh"
#include "wenoc_window.cuh"

using namespace wc;

namespace wc {

template <int N, typename T, typename TF>
static cudaError_t go_stage(const PatchArgs& pa, const Mat& m, int block, int grid,
                           cudaStream_t st) {
  const int smem = Ring<N, 3, T>::BYTES * block;
  auto k = k_patch_stage<N, T, TF>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, block, smem, st>>>(pa, m);
  return cudaGetLastError();
}

cudaError_t launch_patch_stage(int N, int mixed, const PatchArgs& pa, const Mat& m, int block,
                               int grid, cudaStream_t st) {
#define PS_(NN)                                                                     \
  if (N == NN) {                                                                    \
    if (mixed) return go_stage<NN, float, float>(pa, m, block, grid, st);           \
    return go_stage<NN, double, double>(pa, m, block, grid, st);                    \
  }
  PS_(1) PS_(2) PS_(3) PS_(4) PS_(5)
#undef PS_
  return cudaErrorInvalidValue;
}

cudaError_t launch_patch_rate(int N, const double* U, long ncell, const int* edge,
                              const long* off, int npatch, const Mat& m,
                              unsigned long long* rate_bits, unsigned* status, cudaStream_t st) {
  int grid = std::min(npatch, 148 * 16);
#define PR_(NN)                                                                       \
  if (N == NN) {                                                                      \
    k_patch_rate<NN><<<grid, 256, 0, st>>>(U, ncell, edge, off, npatch, m, rate_bits, \
                                           status);                                   \
    return cudaGetLastError();                                                        \
  }
  PR_(1) PR_(2) PR_(3) PR_(4) PR_(5)
#undef PR_
  return cudaErrorInvalidValue;
}

}  // namespace wc

// The patches of one edge e, for the window schedule: their first cells in
// the pooled state at gpoff[first .. first + count).
struct PatchGroup {
  int e, first, count;
};

struct wc_patches {
  wc_patches_desc d;
  Mat mat;
  int nv = 0;
  std::vector<int> edge;
  std::vector<long> off;
  std::vector<int> order;
  std::vector<PatchGroup> groups;  // by decreasing edge
  std::vector<long> gpoff;
  long ncell = 0;
  // bindings
  double* U = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double *B1 = nullptr, *B2 = nullptr, *Lacc = nullptr, *backup = nullptr;
  int* d_edge = nullptr;
  long* d_off = nullptr;
  int* d_order = nullptr;
  long* d_gpoff = nullptr;
  double* vbuf = nullptr;    // primitive slots of a stage's input (window schedule)
  double* fbuf = nullptr;    // face buffer of the split window sweep (mixed)
  unsigned* d_ticket = nullptr;  // window queue (next window, warps finished)
  int* d_counter = nullptr;  // 3 queue heads (one per stage)
  unsigned long long* d_rate = nullptr;
  unsigned* d_status = nullptr;
  // schedule (dynamic: 1 queue of patches, 0 round-robin, 2 window sweeps)
  int block = 64, ctas_per_sm = 4, dynamic = 1;
  // captured step
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gstream = nullptr;
  double gcfl = 0.0, gdt = 0.0;
  char err[256];
};

static wc_status pfail(wc_patches* g, wc_status s, const char* msg) {
  if (g) snprintf(g->err, sizeof(g->err), "%s", msg);
  return s;
}
static wc_status pcuda(wc_patches* g, cudaError_t e, const char* where) {
  if (g) snprintf(g->err, sizeof(g->err), "%s: %s", where, cudaGetErrorString(e));
  return WC_ERR_CUDA;
}
static inline cudaStream_t PS(void* s) { return reinterpret_cast<cudaStream_t>(s); }
static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

extern "C" wc_status wc_patches_init(const wc_patches_desc* desc, const int* edges,
                                     wc_patches** out) {
  if (!desc || !edges || !out) return WC_ERR_ARG;
  *out = nullptr;
  const wc_patches_desc& d = *desc;
  if (d.nphase < 1 || d.nphase > 5) return WC_ERR_UNSUPPORTED;
  if (d.npatch < 1) return WC_ERR_ARG;
  if (d.flux != WC_FLUX_HLL && d.flux != WC_FLUX_HLLC) return WC_ERR_ARG;
  if (d.precision != WC_PREC_FP64 && d.precision != WC_PREC_MIXED) return WC_ERR_UNSUPPORTED;
  if (d.kmodel != WC_KMODEL_ALLAIRE && d.kmodel != WC_KMODEL_KAPILA) return WC_ERR_ARG;
  for (int p = 0; p < d.nphase; p++)
    if (!(d.gamma[p] > 1.0) || !(d.pinf[p] >= 0.0)) return WC_ERR_ARG;
  for (int i = 0; i < d.npatch; i++)
    if (edges[i] < 3 || edges[i] > 1024) return WC_ERR_ARG;
  wc_patches* g = new (std::nothrow) wc_patches();
  if (!g) return WC_ERR_ARG;
  g->d = d;
  g->nv = 2 * d.nphase + 3 + 1;
  Mat& m = g->mat;
  memset(&m, 0, sizeof(m));
  m.N = d.nphase;
  m.kapila = d.kmodel == WC_KMODEL_KAPILA;
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
  g->edge.assign(edges, edges + d.npatch);
  g->off.resize(d.npatch);
  long o = 0;
  for (int i = 0; i < d.npatch; i++) {
    g->off[i] = o;
    o += (long)edges[i] * edges[i] * edges[i];
  }
  g->ncell = o;
  g->order.resize(d.npatch);
  std::iota(g->order.begin(), g->order.end(), 0);
  // largest patch first (longest processing time first), ties by index
  std::stable_sort(g->order.begin(), g->order.end(),
                   [&](int a, int b) { return edges[a] > edges[b]; });
  // window schedule: the patches of each edge, largest edge first, each
  // group in patch order
  for (int i : g->order) {
    if (g->groups.empty() || g->groups.back().e != edges[i])
      g->groups.push_back(PatchGroup{edges[i], (int)g->gpoff.size(), 0});
    g->groups.back().count++;
    g->gpoff.push_back(g->off[i]);
  }
  for (PatchGroup& gr : g->groups)
    std::sort(g->gpoff.begin() + gr.first, g->gpoff.begin() + gr.first + gr.count);
  g->err[0] = 0;
  *out = g;
  return WC_OK;
}

extern "C" void wc_patches_destroy(wc_patches* g) {
  if (!g) return;
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  delete g;
}

extern "C" long wc_patches_ncell(const wc_patches* g) { return g ? g->ncell : 0; }
extern "C" long wc_patches_offset(const wc_patches* g, int p) {
  return (g && p >= 0 && p < (int)g->off.size()) ? g->off[p] : -1;
}

static size_t table_bytes(const wc_patches* g) {
  size_t np = g->edge.size();
  return round256(np * sizeof(int)) + round256(np * sizeof(long)) + round256(np * sizeof(int)) +
         round256(np * sizeof(long)) + 256;
}

// The split window sweep's face buffer (mixed precision): room for the
// largest group of patches, whose sweeps run one group at a time.
static size_t face_buffer_bytes(const wc_patches* g) {
  if (g->d.precision != WC_PREC_MIXED) return 0;
  long most = 0;
  for (const PatchGroup& gr : g->groups)
    most = std::max(most, fbuf_doubles(g->nv, (long)gr.count * gr.e * gr.e, gr.e));
  return round256((size_t)most * sizeof(double));
}

// The primitive slots of the window schedule: 1 + NV words a cell (the FP64
// slot; the mixed precision's is smaller).
static size_t prim_buffer_bytes(const wc_patches* g) {
  return round256((size_t)(1 + g->nv) * g->ncell * sizeof(double));
}

static size_t base_bytes(const wc_patches* g) {
  size_t state = round256((size_t)g->nv * g->ncell * sizeof(double));
  return 4 * state + table_bytes(g);
}

extern "C" size_t wc_patches_face_buffer_bytes(const wc_patches* g) {
  return g ? face_buffer_bytes(g) : 0;
}

extern "C" size_t wc_patches_prim_buffer_bytes(const wc_patches* g) {
  return g ? prim_buffer_bytes(g) : 0;
}

extern "C" size_t wc_patches_workspace_bytes(const wc_patches* g) {
  if (!g) return 0;
  return base_bytes(g) + prim_buffer_bytes(g) + face_buffer_bytes(g);
}

extern "C" wc_status wc_patches_set_state(wc_patches* g, double* U_dev, void* ws, size_t bytes,
                                          void* stream) {
  if (!g || !U_dev || !ws) return WC_ERR_ARG;
  if (bytes < base_bytes(g)) return pfail(g, WC_ERR_ARG, "workspace too small");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return pfail(g, WC_ERR_ARG, "workspace alignment");
  size_t state = round256((size_t)g->nv * g->ncell * sizeof(double));
  size_t np = g->edge.size();
  g->U = U_dev;
  g->ws = (char*)ws;
  g->ws_bytes = bytes;
  g->B1 = (double*)g->ws;
  g->B2 = (double*)(g->ws + state);
  g->Lacc = (double*)(g->ws + 2 * state);
  g->backup = (double*)(g->ws + 3 * state);
  char* t = g->ws + 4 * state;
  g->d_edge = (int*)t;
  t += round256(np * sizeof(int));
  g->d_off = (long*)t;
  t += round256(np * sizeof(long));
  g->d_order = (int*)t;
  t += round256(np * sizeof(int));
  g->d_gpoff = (long*)t;
  t += round256(np * sizeof(long));
  g->d_counter = (int*)t;                 // 3 ints
  g->d_rate = (unsigned long long*)(t + 64);
  g->d_status = (unsigned*)(t + 128);
  g->d_ticket = (unsigned*)(t + 192);     // 2 unsigned
  // without room for the primitive slots the window sweeps convert their
  // cells themselves; without the face buffer the mixed one runs in one pass
  g->vbuf = bytes >= base_bytes(g) + prim_buffer_bytes(g) ? (double*)(g->ws + base_bytes(g))
                                                          : nullptr;
  g->fbuf = bytes >= wc_patches_workspace_bytes(g) && face_buffer_bytes(g)
                ? (double*)(g->ws + base_bytes(g) + prim_buffer_bytes(g))
                : nullptr;
  cudaStream_t st = PS(stream);
  cudaError_t e = cudaMemcpyAsync(g->d_edge, g->edge.data(), np * sizeof(int),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_off, g->off.data(), np * sizeof(long), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_order, g->order.data(), np * sizeof(int), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_gpoff, g->gpoff.data(), np * sizeof(long), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t, 0, 256, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return pcuda(g, e, "patch table upload");
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  return WC_OK;
}

extern "C" wc_status wc_patches_set_schedule(wc_patches* g, int block, int ctas_per_sm,
                                             int dynamic) {
  if (!g || (block != 32 && block != 64 && block != 96 && block != 128) || ctas_per_sm < 1 ||
      ctas_per_sm > 16 || dynamic < 0 || dynamic > 2)
    return WC_ERR_ARG;
  g->block = block;
  g->ctas_per_sm = ctas_per_sm;
  g->dynamic = dynamic;
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  return WC_OK;
}

static PatchArgs patch_args(wc_patches* g, const double* src, double* dst, double r0, double r1,
                            double r2, double cfl, double dt, int stage, int rhs_only,
                            double* L) {
  PatchArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.U = src;
  pa.L = L;
  pa.U0 = g->U;
  pa.Uout = dst;
  pa.rate = (const double*)g->d_rate;
  pa.cfl = cfl;
  pa.dt_fixed = dt;
  pa.rk0 = r0;
  pa.rk1 = r1;
  pa.rk2 = r2;
  pa.ncell = g->ncell;
  pa.edge = g->d_edge;
  pa.off = g->d_off;
  pa.order = g->d_order;
  pa.npatch = (int)g->edge.size();
  pa.counter = g->d_counter + stage;
  pa.dynamic = g->dynamic;
  pa.rhs_only = rhs_only;
  pa.hllc = g->d.flux == WC_FLUX_HLLC;
  pa.energy_limiter = g->d.energy_limiter;
  pa.status = g->d_status;
  return pa;
}

static int patch_grid(const wc_patches* g) { return 148 * g->ctas_per_sm; }

// The window schedule: for each direction, the window sweep over the pencils
// of each group of equal patches (pencil tr of a group in its patch
// tr / e^2, at the offset table gpoff), outflow boundary cells at both ends
// of every pencil; mixed precision splits each sweep into the face and the
// flux pass when the workspace holds the face buffer.  Directions run in
// order over all patches, so the accumulator modes are those of a grid:
// L = x part, L += y part, then the stage (or L += z part for the rhs).
template <typename T>
static cudaError_t launch_prim_patches(const wc_patches* g, const double* src, cudaStream_t st) {
  long b = (g->ncell + 255) / 256;
  if (b > 148L * 64) b = 148L * 64;
  const int blocks = (int)(b < 1 ? 1 : b);
  switch (g->d.nphase) {
#define WC_PRIM_CASE(NP)                                                                   \
  case NP:                                                                                 \
    k_prim_slots<NP, 3, T><<<blocks, 256, 256 * Ring<NP, 3, T>::SLOTD * 8, st>>>(          \
        src, g->vbuf, g->ncell, 0, g->ncell, g->mat);                                      \
    break;
    WC_PRIM_CASE(1)
    WC_PRIM_CASE(2)
    WC_PRIM_CASE(3)
    WC_PRIM_CASE(4)
    WC_PRIM_CASE(5)
#undef WC_PRIM_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

static cudaError_t enqueue_windows(wc_patches* g, const double* src, double* dst, double* L,
                                   double r0, double r1, double r2, double cfl, double dt,
                                   int rhs_only, cudaStream_t st) {
  const int mixed = g->d.precision == WC_PREC_MIXED;
  // the primitive slots of src, once for the stage's three directions
  if (g->vbuf) {
    const cudaError_t e = mixed ? launch_prim_patches<float>(g, src, st)
                                : launch_prim_patches<double>(g, src, st);
    if (e != cudaSuccess) return e;
  }
  for (int dir = 0; dir < 3; dir++) {
    for (const PatchGroup& gr : g->groups) {
      SweepArgs a;
      memset(&a, 0, sizeof(a));
      a.U = src;
      a.L = L;
      a.U0 = g->U;
      a.Uout = dst;
      a.rate = (const double*)g->d_rate;
      a.cfl = cfl;
      a.dt_fixed = dt;
      a.rk0 = r0;
      a.rk1 = r1;
      a.rk2 = r2;
      a.ncell = g->ncell;
      a.nx = a.ny = a.nz = gr.e;
      a.dir = dir;
      a.n = gr.e;
      a.stride = dir == 0 ? 1 : (dir == 1 ? (long)gr.e : (long)gr.e * gr.e);
      a.npencil = (long)gr.count * gr.e * gr.e;
      a.nwin = (gr.e + WIN - 1) / WIN;
      a.ticket = g->d_ticket;
      const WinPlan w = win_plan(gr.e, a.npencil);
      a.wfull = w.wfull;
      a.wtail = w.wtail;
      a.wgrp = w.wgrp;
      a.wslots = w.slots;
      a.nitems = w.nitems;
      a.max_threads = 148L * g->ctas_per_sm * g->block;  // ctas_per_sm resident blocks
      a.inv_dx = (double)gr.e;  // unit-cube patch: dx = 1/e
      a.bclo = a.bchi = BC_OUTFLOW;
      a.mode = rhs_only ? (dir == 0 ? 0 : 1) : (dir == 0 ? 0 : (dir == 1 ? 1 : 2));
      a.hllc = g->d.flux == WC_FLUX_HLLC;
      a.energy_limiter = g->d.energy_limiter;
      a.status = g->d_status;
      a.poff = g->d_gpoff + gr.first;
      a.Vs = g->vbuf;
      a.fbuf = mixed ? g->fbuf : nullptr;
      cudaError_t e = mixed ? launch_sweep_mixed(g->d.nphase, 3, a, g->mat, g->block, st)
                            : launch_sweep_fp64(g->d.nphase, 3, a, g->mat, g->block, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// One SSP-RK3 step: rate reduction (unless dt is fixed), queue reset, three
// persistent stage launches.
static cudaError_t enqueue_step(wc_patches* g, double cfl, double dt, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (!(dt > 0.0)) {
    e = cudaMemsetAsync(g->d_rate, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess)
      e = launch_patch_rate(g->d.nphase, g->U, g->ncell, g->d_edge, g->d_off,
                            (int)g->edge.size(), g->mat, g->d_rate, g->d_status, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(g->d_counter, 0, 3 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int mixed = g->d.precision == WC_PREC_MIXED;
  PatchArgs a1 = patch_args(g, g->U, g->B1, 0.0, 1.0, 1.0, cfl, dt, 0, 0, g->Lacc);
  PatchArgs a2 = patch_args(g, g->B1, g->B2, 0.75, 0.25, 0.25, cfl, dt, 1, 0, g->Lacc);
  PatchArgs a3 = patch_args(g, g->B2, g->U, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, cfl, dt, 2, 0,
                            g->Lacc);
  for (const PatchArgs* a : {&a1, &a2, &a3}) {
    if (g->dynamic == 2)
      e = enqueue_windows(g, a->U, a->Uout, a->L, a->rk0, a->rk1, a->rk2, cfl, dt, 0, st);
    else
      e = launch_patch_stage(g->d.nphase, mixed, *a, g->mat, g->block, patch_grid(g), st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

extern "C" wc_status wc_patches_rk_step(wc_patches* g, double cfl, double dt_fixed, int nsteps,
                                        int use_graph, void* stream) {
  if (!g || nsteps < 0) return WC_ERR_ARG;
  if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return pfail(g, WC_ERR_ARG, "need cfl or dt");
  if (!g->U) return pfail(g, WC_ERR_STATE, "state not bound");
  cudaStream_t st = PS(stream);
  if (!use_graph) {
    for (int s = 0; s < nsteps; s++) {
      cudaError_t e = enqueue_step(g, cfl, dt_fixed, st);
      if (e != cudaSuccess) return pcuda(g, e, "patch step");
    }
    return WC_OK;
  }
  if (st == nullptr) return pfail(g, WC_ERR_ARG, "graph capture needs a non-default stream");
  if (!g->gexec || g->gstream != st || g->gcfl != cfl || g->gdt != dt_fixed) {
    if (g->gexec) {
      cudaGraphExecDestroy(g->gexec);
      g->gexec = nullptr;
    }
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return pcuda(g, e, "begin capture");
    cudaError_t e2 = enqueue_step(g, cfl, dt_fixed, st);
    e = cudaStreamEndCapture(st, &graph);
    if (e2 != cudaSuccess) return pcuda(g, e2, "captured step");
    if (e != cudaSuccess) return pcuda(g, e, "end capture");
    e = cudaGraphInstantiate(&g->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return pcuda(g, e, "graph instantiate");
    g->gstream = st;
    g->gcfl = cfl;
    g->gdt = dt_fixed;
  }
  for (int s = 0; s < nsteps; s++) {
    cudaError_t e = cudaGraphLaunch(g->gexec, st);
    if (e != cudaSuccess) return pcuda(g, e, "graph launch");
  }
  return WC_OK;
}

extern "C" wc_status wc_patches_rhs(wc_patches* g, const double* U, double* L, void* stream) {
  if (!g || !U || !L) return WC_ERR_ARG;
  if (!g->d_counter) return pfail(g, WC_ERR_STATE, "state/workspace not bound");
  cudaStream_t st = PS(stream);
  cudaError_t e = cudaMemsetAsync(g->d_counter, 0, 3 * sizeof(int), st);
  if (e != cudaSuccess) return pcuda(g, e, "counter reset");
  if (g->dynamic == 2) {
    e = enqueue_windows(g, U, nullptr, L, 0.0, 0.0, 0.0, 0.0, 0.0, 1, st);
    return e == cudaSuccess ? WC_OK : pcuda(g, e, "patch rhs");
  }
  PatchArgs a = patch_args(g, U, nullptr, 0, 0, 0, 0, 0, 0, 1, L);
  e = launch_patch_stage(g->d.nphase, g->d.precision == WC_PREC_MIXED, a, g->mat, g->block,
                         patch_grid(g), st);
  return e == cudaSuccess ? WC_OK : pcuda(g, e, "patch rhs");
}

extern "C" wc_status wc_patches_sync_status(wc_patches* g, void* stream) {
  if (!g || !g->d_status) return WC_ERR_STATE;
  unsigned s = 0;
  cudaStream_t st = PS(stream);
  cudaError_t e = cudaMemcpyAsync(&s, g->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return pcuda(g, e, "status");
  if (s & ST_INADMISSIBLE) return pfail(g, WC_ERR_INADMISSIBLE, "inadmissible state");
  if (s & ST_NAN) return pfail(g, WC_ERR_NAN, "non-finite value");
  return WC_OK;
}

extern "C" wc_status wc_patches_autotune(wc_patches* g, double cfl, int steps, void* stream,
                                         int* best_block, int* best_ctas, int* best_dynamic,
                                         double* best_ms) {
  if (!g || steps < 1 || !(cfl > 0.0)) return WC_ERR_ARG;
  if (!g->U) return pfail(g, WC_ERR_STATE, "state not bound");
  cudaStream_t st = PS(stream);
  size_t bytes = (size_t)g->nv * g->ncell * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(g->backup, g->U, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return pcuda(g, e, "backup");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks[] = {64, 128};
  const int ctas[] = {2, 3, 4, 6};
  const int dyn[] = {1, 0, 2};
  double best = -1.0;
  int bb = g->block, bc = g->ctas_per_sm, bd = g->dynamic;
  for (int b : blocks)
    for (int c : ctas)
      for (int d : dyn) {
        // skip schedules whose resident CTAs cannot fit; the window sweep
        // with 128-thread blocks at 2-4 per SM (its registers admit no more)
        if (b * c > 768) continue;
        if (d == 2 && (b != 128 || c > 4)) continue;
        g->block = b;
        g->ctas_per_sm = c;
        g->dynamic = d;
        e = cudaMemcpyAsync(g->U, g->backup, bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = enqueue_step(g, cfl, 0.0, st);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int s = 0; s < steps && e == cudaSuccess; s++) e = enqueue_step(g, cfl, 0.0, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        double per = ms / steps;
        if (best < 0 || per < best) {
          best = per;
          bb = b;
          bc = c;
          bd = d;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return pcuda(g, e, "autotune");
  e = cudaMemcpyAsync(g->U, g->backup, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return pcuda(g, e, "restore");
  wc_status s = wc_patches_set_schedule(g, bb, bc, bd);
  if (best_block) *best_block = bb;
  if (best_ctas) *best_ctas = bc;
  if (best_dynamic) *best_dynamic = bd;
  if (best_ms) *best_ms = best;
  return s;
}

extern "C" void wc_patches_last_error(const wc_patches* g, char* buf, size_t n) {
  if (!buf || n == 0) return;
  snprintf(buf, n, "%s", g ? g->err : "null");
}

extern "C" wc_status wc_patches_prim_to_cons(const wc_patches* gc, const double* V, double* U,
                                             void* stream) {
  wc_patches* g = const_cast<wc_patches*>(gc);
  if (!g || !V || !U) return WC_ERR_ARG;
  long n = g->ncell;
  int blocks = (int)std::min<long>((n + 255) / 256, 148L * 64);
  cudaStream_t st = PS(stream);
  switch (g->d.nphase) {
    case 1: k_prim_to_cons<1, 3><<<blocks, 256, 0, st>>>(V, U, n, g->mat); break;
    case 2: k_prim_to_cons<2, 3><<<blocks, 256, 0, st>>>(V, U, n, g->mat); break;
    case 3: k_prim_to_cons<3, 3><<<blocks, 256, 0, st>>>(V, U, n, g->mat); break;
    case 4: k_prim_to_cons<4, 3><<<blocks, 256, 0, st>>>(V, U, n, g->mat); break;
    case 5: k_prim_to_cons<5, 3><<<blocks, 256, 0, st>>>(V, U, n, g->mat); break;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WC_OK : pcuda(g, e, "prim_to_cons");
}
