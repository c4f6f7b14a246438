/*
 * wenoc.h -- C ABI of the B300 WENO-C finite-volume operator.
 *
 * The operator is the hyperbolic step of the N-phase Euler/Phase-Field model
 * of Huang, "Consistent and bound-preserving finite-volume WENO scheme for
 * compressible two-/N-phase flows with Phase-Field mechanism":
 *     dU/dt + div F^HB(U^L, U^R) = H^HB(U) div u_hat            (Eq. 3)
 * with fifth-order WENO-C reconstruction (Eq. 15-21), an HLL or HLLC flux with
 * the consistent face velocity u_hat (Sec. 2.2.1), and third-order SSP
 * Runge-Kutta time stepping (Sec. 4).
 *
 * State layout (every array in this header): structure of arrays, FP64,
 *     U[v * ncell + cell],  cell = (k * ny + j) * nx + i   (x fastest)
 * with v over U = [(alpha rho)_1..N, (rho u)_1..d, rho E, alpha_1..N] (Eq. 1)
 * or V = [(alpha rho)_1..N, u_1..d, P, alpha_1..N] (primitive, Sec. 2.2.2).
 * Only interior cells are stored; boundary cells are produced on the fly
 * from the boundary condition of each side.
 *
 * Memory and ownership: the library allocates no device memory.  Every
 * device pointer belongs to the caller and must stay valid for the calls
 * that use it; host pointers are read or written only during the call.
 * All device work is enqueued on the caller's CUDA stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream); calls return as soon as
 * the work is enqueued unless stated otherwise.
 *
 * Errors: every entry point returns a wc_status and never aborts.  Argument
 * errors are detected on the host before any launch.  Problems found by the
 * kernels (an inadmissible state: non-positive density, non-finite pressure)
 * set bits in a device status word that wc_sync_status() reads.
 */
#ifndef WENOC_H
#define WENOC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WC_MAX_PHASE 8

typedef enum {
  WC_OK = 0,
  WC_ERR_ARG = 1,          /* invalid argument (checked on the host) */
  WC_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  WC_ERR_INADMISSIBLE = 3, /* a kernel met a state outside the admissible set */
  WC_ERR_NAN = 4,          /* a kernel produced a non-finite value */
  WC_ERR_UNSUPPORTED = 5,  /* combination not built (e.g. phase count) */
  WC_ERR_STATE = 6,        /* call order: state or workspace not bound */
  WC_ERR_TIMEOUT = 7       /* a bounded wait inside a tensor-core kernel ran out */
} wc_status;

enum { WC_BC_PERIODIC = 0, WC_BC_REFLECTIVE = 1, WC_BC_OUTFLOW = 2 };
enum { WC_FLUX_HLL = 0, WC_FLUX_HLLC = 1 };
enum { WC_PREC_FP64 = 0, WC_PREC_MIXED = 1, WC_PREC_LEARNED = 2 };
enum { WC_SCHEME_C = 0, WC_SCHEME_CL = 1, WC_SCHEME_W = 2, WC_SCHEME_JS = 3 };
enum { WC_KMODEL_ALLAIRE = 0, WC_KMODEL_KAPILA = 1 };

/* Grid, materials and scheme options.  Materials follow the stiffened-gas
 * equation of state of Eq. 26: A_p = 1/(gamma_p-1), B_p = gamma_p Pinf_p /
 * (gamma_p-1), D_p; pmin[p] is the phasic minimum pressure of the energy
 * constraint psi (Eq. 9). */
typedef struct {
  int dim;                    /* 1, 2 or 3 */
  int n[3];                   /* interior cells per axis; 1 on unused axes */
  double dx[3];               /* uniform cell size per axis (Sec. 3.5) */
  int nphase;                 /* N, 1..5 built */
  double gamma[WC_MAX_PHASE];
  double pinf[WC_MAX_PHASE];
  double D[WC_MAX_PHASE];
  double pmin[WC_MAX_PHASE];
  int flux;                   /* WC_FLUX_HLL (Sec. 4.2) or WC_FLUX_HLLC (Sec. 4.1) */
  int precision;              /* WC_PREC_FP64; WC_PREC_MIXED (FP32 smoothness
                                 indicators, reconstruction and flux; FP64
                                 pressure, limiter factors, unity sum, update);
                                 WC_PREC_LEARNED (as mixed, with the mass and
                                 fraction weights of Eq. 16 from the learned
                                 surrogate where accepted, N <= 3; see
                                 wc_set_mlp) */
  int energy_limiter;         /* 1: Eq. 21 applied (default); 0: skipped */
  int bc[6];                  /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi: WC_BC_* */
  int seg;                    /* sweep schedule.  0 (default): one cell per
                                 lane, each warp takes windows of 32 cells of
                                 a pencil (30 updated) from a dynamic queue;
                                 > 0: each thread marches segments of seg
                                 cells of one pencil */
  int block;                  /* threads per sweep block, a multiple of 32
                                 in 32..128; 0 = automatic (128) */
  int blocks_per_sm;          /* resident sweep blocks per SM (1..32); 0 =
                                 automatic (the window sweep: as many as
                                 fit) */
  int scheme;                 /* WC_SCHEME_C: unity sum by Eq. 19 (WENO-C,
                                 default); WC_SCHEME_CL: the consistent limiter
                                 of Eq. 23-25 instead (WENO-CL, Sec. 3.4);
                                 the comparison schemes of Sec. 4.1.1,
                                 WC_SCHEME_W (Eq. 15 weights) and
                                 WC_SCHEME_JS (Jiang-Shu weights with js_eps):
                                 every primitive variable with its own
                                 weights, no coupling (Eq. 16), no limiters
                                 (Eq. 17-21; energy_limiter is ignored) and
                                 no bound restored after a stage; FP64
                                 only (WC_ERR_UNSUPPORTED otherwise) */
  int kmodel;                 /* K_p of Eq. 2-3: WC_KMODEL_ALLAIRE (K_p = 0,
                                 default) or WC_KMODEL_KAPILA (K_p = rho c^2 /
                                 (rho_p c_p^2) - 1 with Wood's mixture speed
                                 1/(rho c^2) = sum_p alpha_p/(rho_p c_p^2),
                                 which sum_p alpha_p K_p = 0 implies) */
  double js_eps;              /* epsilon of WC_SCHEME_JS (> 0; 0 = 1e-6, the
                                 value of Sec. 3.2) */
} wc_grid_desc;

typedef struct wc_grid wc_grid;

/* Calls that enqueue work on one grid must be ordered on one stream: the
 * grid's status word and window queue live in its workspace. */

/* Creates a grid handle from desc (copied).  Host only, no device work. */
wc_status wc_init_grid(const wc_grid_desc *desc, wc_grid **out);
void wc_destroy(wc_grid *g);

/* Number of variables 2N+d+1 and of interior cells. */
int wc_nvar(const wc_grid *g);
long wc_ncell(const wc_grid *g);

/* Device scratch that wc_rk_step needs: three state-sized FP64 buffers
 * (two Runge-Kutta stages and the direction accumulator) plus 256 bytes; for
 * WC_PREC_LEARNED one more buffer of 18 x ncell FP32 learned weights; for the
 * window schedule (seg = 0) of a 2-D or 3-D grid the primitive slots of a
 * stage's input, (NV + 1) x ncell FP64 words (Eq. 27 once a stage for every
 * cell, read by the stage's direction sweeps); and for the reduced
 * precisions (window schedule) the face buffer of the split sweep,
 * (2 NV + 1) x (n + 2) x ncell / n FP64 values for the direction with the
 * most (n = its cell count): the face pass of each direction stores the
 * limited face states and the cells' pressures there for its flux pass. */
size_t wc_workspace_bytes(const wc_grid *g);
/* The face buffer's part of wc_workspace_bytes (0 in FP64).  It is
 * optional: a workspace of at least wc_workspace_bytes(g) minus this runs
 * the single-pass sweep instead (same results, bit for bit). */
size_t wc_face_buffer_bytes(const wc_grid *g);
/* The primitive slots' part of wc_workspace_bytes (0 for the segment
 * schedule and for 1-D grids).  Optional too: a workspace of at least
 * wc_workspace_bytes(g) minus this and minus wc_face_buffer_bytes(g) runs
 * sweeps that convert their cells themselves (same results, bit for bit). */
size_t wc_prim_buffer_bytes(const wc_grid *g);

/* Binds the caller's device state array U_dev ([NV][ncell] FP64, advanced in
 * place by wc_rk_step) and a device workspace of wc_workspace_bytes(g) bytes
 * (256-byte aligned).  Smaller workspaces drop the optional parts: at least
 * wc_workspace_bytes(g) - wc_face_buffer_bytes(g) keeps the primitive slots
 * and runs the single-pass sweep; at least that minus
 * wc_prim_buffer_bytes(g) runs without either; less is WC_ERR_ARG. */
wc_status wc_set_state(wc_grid *g, double *U_dev, void *workspace_dev, size_t ws_bytes);

/* Validates a state against the admissible set of Eq. 8 (the paper's
 * definition of the states the scheme preserves): for every cell, masses
 * >= 0, fractions in [0, 1] with |sum_p alpha_p - 1| <= sum_tol, a positive
 * density, psi >= 0 (Eq. 9, the phasic minimum pressures of the grid), all
 * values finite.  U_dev: [NV][ncell] device state (e.g. before binding it
 * with wc_set_state); needs a bound workspace (two counters in its tail).
 * Synchronises stream.  Returns WC_ERR_INADMISSIBLE (message in
 * wc_last_error) when a cell is outside; *nbad and *first_bad (may be
 * null) receive the count and the first such cell (-1 when none). */
wc_status wc_check_state(wc_grid *g, const double *U_dev, double sum_tol, long *nbad,
                         long *first_bad, void *stream);

/* Copies a host state (pinned memory recommended) into / out of the bound
 * device state, asynchronously on stream. */
wc_status wc_upload_state(wc_grid *g, const double *U_host, void *stream);
wc_status wc_download_state(const wc_grid *g, double *U_host, void *stream);

/* psi_{V->U} and psi_{U->V} (mixture rules, Eq. 26, Eq. 27) on device arrays
 * of ncell cells laid out [NV][ncell]; ncell = wc_ncell(g). */
wc_status wc_prim_to_cons(const wc_grid *g, const double *V_dev, double *U_dev, void *stream);
wc_status wc_cons_to_prim(const wc_grid *g, const double *U_dev, double *V_dev, void *stream);

/* Mixture temperature of Eq. 29 into T_dev ([ncell]) for the state U_dev:
 * (rho E - |rho u|^2/(2 rho) - sum_p B_p^T alpha_p - sum_p D_p (alpha rho)_p) /
 * sum_p C_p^T (alpha rho)_p with B_p^T = Pinf_p (Eq. 26) and the caller's heat
 * capacities cT[N] (host array, > 0; Sec. 4.1.1 derives them from a
 * reference state: C_p^T = (A_p P0 + B_p - Pinf_p)/(rho_p T0)).  A diagnostic
 * of thermal equilibrium; asynchronous on stream. */
wc_status wc_temperature(const wc_grid *g, const double *U_dev, const double *cT, double *T_dev,
                         void *stream);

/* L = dU/dt of the hyperbolic step (Eq. 3) for the state U_dev (not the bound
 * state), summed over the directions; L_dev is overwritten. */
wc_status wc_rhs(wc_grid *g, const double *U_dev, double *L_dev, void *stream);

/* The limited face states of one direction's sweep of wc_rhs for the state
 * U_dev, as the grid's precision and scheme compute them: UL_dev[v][cell] =
 * U^L_{i+1/2} and UR_dev[v][cell] = U^R_{i-1/2} ([NV][ncell] FP64 each,
 * device), the conservative face states after Eq. 16-21 that the Riemann
 * solver receives (Eq. 8 is what they must satisfy).  A diagnostic of the
 * operator (the paper has no such call); the direction's rhs goes to the
 * workspace's accumulator.  Window schedule only (seg = 0, else
 * WC_ERR_UNSUPPORTED).  Asynchronous on stream. */
wc_status wc_faces(wc_grid *g, int dir, const double *U_dev, double *UL_dev, double *UR_dev,
                   void *stream);

/* L = dU/dt of the Phase-Field step (Eq. 5), + div F^PF, for the state U_dev
 * and the auxiliary fields Q_dev [N][ncell] of Eq. 4 (wc_qmap computes them).
 * Face gradients G are central differences of Q, zero on a face where both
 * cells have phi_p (1 - phi_p) <= 0 (Eq. 4 does not couple it), and, when
 * dt_limit > 0, limited to |G| <= dx / (12 d dt_limit) (the Phase-Field
 * step's sufficient condition for bounds at that time step); dt_limit = 0:
 * no limit.  The face states are the WENO-C reconstructions of U.  The
 * numerical flux (not printed in the paper, which cites it) is the
 * bound-preserving upwinding J_p = max(G,0) a_R (1-a_L) + min(G,0) a_L (1-a_R)
 * of phi_p (1 - phi_p) grad Q_p, masses alike with (alpha rho)_p in the
 * outgoing factor, corrected to sum_p J_p = 0 in proportion to the face
 * fractions; momentum and energy as in the last line of Eq. 1. */
wc_status wc_rhs_pf(wc_grid *g, const double *U_dev, const double *Q_dev, double dt_limit,
                    double *L_dev, void *stream);

/* ---- The Phase-Field mechanism of the time step (Sec. 2.2) ----
 * One time step is: the hyperbolic step (Eq. 3), then [div J_p]^ of Eq. 28
 * from the fractions phi_p = alpha_p of its result, the auxiliary fields Q_p
 * of Eq. 4, and the Phase-Field step (Eq. 5) with Q fixed.  Readings where
 * the paper is silent: eta = dx of the first axis; M = 0.5 eta max|u|;
 * second-order central Laplacian (mirrored cells at reflective/outflow
 * sides); midpoint-rule integrals; Eq. 28's singular N x N system solved with
 * B = 0 for absent phases and for the last present one.  Eq. 4 with the face
 * coefficient (c_a + c_b)/2, c = max(phi (1 - phi), 0); on each region that
 * coupled faces connect the part D_i s_k (D_i = sum_faces c_f/dx^2, s_k =
 * sum r / sum D) that no flux phi(1 - phi) grad Q can carry is removed, and
 * the rest is solved by conjugate gradients preconditioned with D; only the
 * face gradients of coupled faces are used (wc_rhs_pf). */

/* Device scratch of the mechanism: sixteen [N][ncell] FP64 fields, three
 * [N][ncell] int32 fields (region labels, the list of unknowns and its
 * inverse) and about 0.4 MB of reduction partials; grids up to 2^30 cells
 * (WC_ERR_UNSUPPORTED beyond). */
size_t wc_pf_workspace_bytes(const wc_grid *g);
/* Binds that scratch (256-byte aligned, at least wc_pf_workspace_bytes). */
wc_status wc_set_pf_workspace(wc_grid *g, void *ws_dev, size_t bytes);

/* [div J_p]^ of Eq. 28 for the fractions of U_dev into R_dev ([N][ncell];
 * may be null: kept in the scratch for wc_qmap).  eta <= 0: dx of the first
 * axis; M < 0: 0.5 eta max|u| (a reproducible device reduction), M >= 0: as
 * given.  Asynchronous on stream. */
wc_status wc_cac_rhs(wc_grid *g, const double *U_dev, double eta, double M, double *R_dev,
                     void *stream);

/* Q_dev ([N][ncell]) of Eq. 4 for the fractions of U_dev and the right-hand
 * sides R_dev (null: those of the last wc_cac_rhs).  warm != 0: Q_dev holds a
 * starting guess (e.g. the previous step's Q), else the iteration starts
 * from 0.  Conjugate gradients stop when every phase has sqrt(r.z / b.b/D)
 * <= tol (the D-weighted residual relative to the right-hand side b) or
 * after maxit iterations; *iters and *resid (may be null) report them.  The
 * region labelling, the region sums and the iterations run on the list of
 * cells that belong to a region (the interface bands) in one cooperative
 * launch of one block per SM (a second one when the band is too large for
 * registers), whose blocks meet at grid barriers with bounded waits
 * (WC_ERR_TIMEOUT if one gave up).  Synchronizes stream (the choice of the
 * second launch and the result read device flags).  The values of Q are fixed up to a constant per
 * region; the region sums use FP64 atomics, so Q varies at rounding level
 * between runs. */
wc_status wc_qmap(wc_grid *g, const double *U_dev, const double *R_dev, double *Q_dev,
                  double tol, int maxit, int warm, int *iters, double *resid, void *stream);

/* The Phase-Field step (Eq. 5) over dt on the bound state: SSP-RK3 with Q
 * fixed, face gradients limited to dx / (12 d dt). */
wc_status wc_pf_step(wc_grid *g, const double *Q_dev, double dt, void *stream);

/* nsteps full time steps on the bound state (wc_rk_step, wc_cac_rhs with the
 * default eta and M, wc_qmap with tol and maxit started from the previous
 * step's Q after the first step of a bound scratch, wc_pf_step with the same
 * time step: dt_fixed, or cfl over the hyperbolic step's rate).  Needs both
 * workspaces; synchronizes stream once per step (wc_qmap).  *dt_host (may be
 * null) receives the last time step. */
wc_status wc_step(wc_grid *g, double cfl, double dt_fixed, int nsteps, double tol, int maxit,
                  double *dt_host, void *stream);

/* Statistics of the last Q-map: CG iterations, labelling rounds, residual. */
wc_status wc_pf_stats(const wc_grid *g, int *cg_iters, int *label_rounds, double *resid);

/* The band of the last wc_qmap: unknowns[p] (p < N; may be null) the cells
 * of phase p that belong to a region (the unknowns of Eq. 4 the iteration
 * ran on), *per_thread (may be null) the unknowns a thread kept in
 * registers (1 or 2; 0: the iteration ran on the lists in memory). */
wc_status wc_pf_band(const wc_grid *g, int *unknowns, int *per_thread);
/* Device pointer to the Q of the last wc_step (inside the scratch), or null. */
const double *wc_pf_q(const wc_grid *g);

/* Time step from the bound state: dt = cfl / max_cells sum_d (|u_d| + c)/dx_d,
 * written to dt_dev (one double, device). */
wc_status wc_compute_dt(wc_grid *g, double cfl, double *dt_dev, void *stream);

/* nsteps steps of SSP-RK3 (Shu-Osher form) on the bound state, in place.
 * dt_fixed > 0 fixes the step; otherwise each step takes dt from cfl and
 * the state at its start (computed on the device, no host synchronisation).
 * When dt_host is not NULL the call synchronises the stream at the end and
 * writes the last step's dt there. */
wc_status wc_rk_step(wc_grid *g, double cfl, double dt_fixed, int nsteps, double *dt_host,
                     void *stream);

/* wc_rk_step from and to host memory: uploads U_in_host ([NV][ncell], the
 * layout of the bound state) into the bound state, runs nsteps >= 1 steps of
 * SSP-RK3 as wc_rk_step does (same results bit for bit), and downloads the
 * final state into U_out_host (may equal U_in_host: every upload completes
 * before the first download starts).  Asynchronous on stream; the host
 * buffers must stay valid until the stream has been synchronised.  With
 * page-locked buffers the copies overlap the sweeps: the first step's first
 * direction (x, which needs no time step) runs in 8 bands of rows, each
 * after its rows have arrived, and the last step's last sweep in 8 bands
 * of pencils (2-D: its last stage takes y first and x last, rows again; the
 * sum of the two directions' parts is the same), each copied back while the
 * next one runs (an internal stream and events; the caller's stream waits
 * for the last copy).  1-D
 * grids, the segment schedule and the learned precision copy, step and copy
 * back in sequence.  Errors: WC_ERR_ARG (null buffer, nsteps < 1, neither
 * cfl nor dt_fixed positive), WC_ERR_STATE (no state, workspace or
 * surrogate bound), WC_ERR_CUDA. */
wc_status wc_rk_step_host(wc_grid *g, const double *U_in_host, double *U_out_host, double cfl,
                          double dt_fixed, int nsteps, void *stream);

/* The limiter chain of WENO-C alone (Eq. 17-21) in direction dir on ncell
 * independent cells: Ubar [NV][ncell] conservative cell averages, VL / VR
 * [NV][ncell] raw reconstructed primitive values at x_{i+1/2} and x_{i-1/2};
 * outputs UL / UR [NV][ncell] limited conservative face states and, when
 * theta is not NULL, theta [3][ncell] = (min_p theta_p of Eq. 17, theta_i of
 * Eq. 20, theta^(psi) of Eq. 21).  All pointers are device pointers. */
wc_status wc_limit(const wc_grid *g, int dir, long ncell, const double *Ubar, const double *VL,
                   const double *VR, double *UL, double *UR, double *theta, void *stream);

/* wc_rk_step without a workspace and without any device allocation, for
 * callers that cannot allocate device memory (their device memory is owned
 * and budgeted by another component, or allocating is not allowed where they
 * run).  The paper has no counterpart: this is a deployment variant of
 * wc_rk_step.
 *
 * Steps the caller's device state U_dev ([NV][ncell] FP64, the grid's bound
 * state is not used) nsteps SSP-RK3 steps in place, with cfl / dt_fixed as in
 * wc_rk_step.  The stage buffers, the direction accumulator and the dt and
 * status words live in one scratch array compiled into the library (24 MiB
 * plus 256 bytes, held by every GPU that loads the library until the process
 * exits).  Grids whose three state-sized buffers do not fit (3 x NV x ncell
 * x 8 bytes, each rounded up to 256, at most 24 MiB; e.g. 2-D N = 2 up to
 * about 149,000 cells) are rejected with WC_ERR_ARG and a message in
 * wc_last_error before any work is enqueued; grids of precision
 * WC_PREC_LEARNED are rejected with WC_ERR_UNSUPPORTED.
 *
 * The first call on a device looks up the scratch's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Every call shares the one array and the array keeps the
 * last call's contents (the dt and status words are cleared by each call):
 * calls whose work overlaps on the GPU -- on different streams, or from
 * different host threads on one grid -- race and must be serialised by the
 * caller.  When status_host is not NULL the call synchronises the stream and
 * writes the device status bits of this call there (0 = no kernel-detected
 * problem; 1 = inadmissible state; 2 = non-finite value). */
wc_status wc_rk_step_noalloc(wc_grid *g, double *U_dev, double cfl, double dt_fixed, int nsteps,
                             int *status_host, void *stream);

/* ------------------------------------------------------------------------
 * Learned WENO-weight surrogate (no counterpart in the paper: a learned
 * stand-in for the weights of Eq. 15 in the coupled reconstruction, Eq. 16,
 * with the paper's limiter, Eq. 17-21, always applied afterwards).
 *
 * Network: 30 inputs (zero-padded to 32) -> 64 -> 64 -> 64 (ReLU) -> 9
 * outputs (padded to 16), a softmax over each phase's three outputs giving
 * the weights of the sub-stencils {i-2..i}, {i-1..i+1}, {i..i+2} (ordered
 * towards the face).  Inputs of one face side of one cell, per phase p < 3:
 * the five masses (alpha rho)_p of the stencil ordered towards the face,
 * minus the cell's own and divided by the largest absolute such difference
 * (0 for a flat stencil), then the five fractions alpha_p; phases beyond N
 * are zero.  Evaluated and trained on the tensor cores: BF16 weights,
 * activations and features, FP32 accumulation, biases and softmax.
 *
 * Parameter block (device, 16-byte aligned, wc_mlp_param_bytes() bytes):
 * BF16 W1[64][32], W2[64][64], W3[64][64], W4[16][64] (row = output unit),
 * then FP32 b1[64], b2[64], b3[64], b4[16].  FP32 arrays of wc_mlp_nparam()
 * entries (master copy, gradients, Adam moments) hold the same parameters in
 * the same order.  Padding (inputs 30-31, outputs 9-15) is kept zero.
 *
 * Feature rows (device, BF16 [rows][32], 16-byte aligned): row0 + 2 cell +
 * side, side 0 = face x_{i+1/2}, side 1 = x_{i-1/2} (mirrored stencil).
 * Targets (FP32 [rows][9]): the plain Eq. 15 weights of each phase's masses
 * on the oriented stencil (ideal weights 0.1/0.6/0.3 for phases beyond N). */
size_t wc_mlp_param_bytes(void);
int wc_mlp_nparam(void);
/* He-normal initial FP32 master parameters (host array of wc_mlp_nparam()
 * floats) from a seed; biases and padding zero. */
wc_status wc_mlp_init_master(float *master_host, unsigned long long seed);
/* Parameter block from FP32 masters (device to device, on stream). */
wc_status wc_mlp_pack(const float *master_dev, void *params_dev, void *stream);
/* Features (and targets when T_dev is not NULL) of both face sides of every
 * cell of the state U_dev in direction dir, written at rows row0 .. row0 + 2
 * ncell - 1.  Rows whose target weights differ from the ideal weights by
 * more than 1e-3 are counted in *count_dev (a device counter the caller
 * clears) and their row numbers appended to list_dev (when not NULL, up to
 * list_cap entries; the count may exceed list_cap). */
wc_status wc_mlp_features(const wc_grid *g, const double *U_dev, int dir, long row0, void *X_dev,
                          float *T_dev, long *list_dev, unsigned long long *count_dev,
                          long list_cap, void *stream);
/* Softmax weights Y_dev [nrows][9] (FP32) of feature rows X_dev.  Kernel
 * problems (a bounded tensor-core wait that ran out) set bit 4 of
 * *status_dev. */
wc_status wc_mlp_forward(const void *X_dev, long nrows, const void *params_dev, float *Y_dev,
                         unsigned *status_dev, void *stream);
/* Learned weights of direction dir for the state U_dev, features gathered
 * in the kernel: W_dev[(9 side + 3 p + s) ncell + cell] (FP32, 18 ncell). */
wc_status wc_mlp_infer(const wc_grid *g, const double *U_dev, int dir, const void *params_dev,
                       float *W_dev, unsigned *status_dev, void *stream);
/* Gradients of loss = (1/batch) sum_b sum_j (y_bj - T_bj)^2 over the batch
 * of rows idx_dev[0..batch) of X_dev / T_dev, ADDED to grads_dev (FP32,
 * wc_mlp_nparam() entries) and the loss added to *loss_dev. */
wc_status wc_mlp_gradients(const void *X_dev, const float *T_dev, const int *idx_dev, int batch,
                           const void *params_dev, float *grads_dev, float *loss_dev,
                           unsigned *status_dev, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with the
 * 1-based step number) on the FP32 masters; writes the parameter block and
 * clears the gradients. */
wc_status wc_mlp_adam(float *master_dev, void *params_dev, float *grads_dev, float *m_dev,
                      float *v_dev, float lr, int step, void *stream);
/* wc_mlp_gradients followed by wc_mlp_adam. */
wc_status wc_mlp_train_step(const void *X_dev, const float *T_dev, const int *idx_dev, int batch,
                            void *params_dev, float *master_dev, float *grads_dev, float *m_dev,
                            float *v_dev, float lr, int step, float *loss_dev,
                            unsigned *status_dev, void *stream);
/* Binds the surrogate used by a WC_PREC_LEARNED grid (params_dev stays the
 * caller's and must outlive its use).  For every interior cell, face side
 * and phase the learned weights replace the plain ones when both the mass
 * and the fraction reconstructed with them differ from their plain
 * reconstructions by at most tau x (max - min of the five stencil values);
 * otherwise, and for boundary cells, the plain weights stand (tau = 0 gives
 * the WC_PREC_MIXED result bit for bit).  counters_dev (optional, two device
 * uint64 the caller clears) accumulates the face sides decided and those
 * that fell back to the plain weights. */
wc_status wc_set_mlp(wc_grid *g, const void *params_dev, float tau,
                     unsigned long long *counters_dev);

/* ------------------------------------------------------------------------
 * Batched AMR-like patches.  npatch independent unit-cube patches, patch p
 * with edge[p] cells per axis (cell size 1/edge[p]), 3-D, all sharing one set
 * of materials.  Every face of every patch is an outflow boundary (zero-
 * gradient boundary cells, three deep -- the stencil reach of WENO5 plus the
 * neighbour face); the uniform-mesh operator is applied on each patch as on
 * one level of a block-structured mesh (Sec. 3.5).  The pooled state is
 * [NV][ncell_total] with patch p's cells at [offset(p), offset(p) + e^3)
 * in x-fastest order.  One persistent launch per RK stage processes all
 * patches; CTAs take whole patches, largest first. */
typedef struct {
  int nphase;
  double gamma[WC_MAX_PHASE];
  double pinf[WC_MAX_PHASE];
  double D[WC_MAX_PHASE];
  double pmin[WC_MAX_PHASE];
  int flux;            /* WC_FLUX_HLL or WC_FLUX_HLLC */
  int precision;       /* WC_PREC_FP64 or WC_PREC_MIXED */
  int energy_limiter;  /* 1: Eq. 21 applied */
  int npatch;
  int kmodel;          /* K_p of Eq. 2-3, as in wc_grid_desc: WC_KMODEL_ALLAIRE
                          (0, the default of a zero-filled descriptor) or
                          WC_KMODEL_KAPILA; anything else is WC_ERR_ARG */
} wc_patches_desc;

typedef struct wc_patches wc_patches;

/* Host only: copies desc and edges[npatch] (3..1024), builds offsets and the
 * largest-first order. */
wc_status wc_patches_init(const wc_patches_desc *desc, const int *edges, wc_patches **out);
void wc_patches_destroy(wc_patches *g);
long wc_patches_ncell(const wc_patches *g);
long wc_patches_offset(const wc_patches *g, int patch);
/* Four pooled state buffers (two stages, accumulator, autotune backup) plus
 * the patch table. */
size_t wc_patches_workspace_bytes(const wc_patches *g);
/* The part of wc_patches_workspace_bytes that holds the face buffer of the
 * window schedule's split sweep (mixed precision; 0 for FP64): room for the
 * face states of the largest group of equal patches, (2 NV + 1) e^2 (e + 2)
 * doubles a patch of edge e. */
size_t wc_patches_face_buffer_bytes(const wc_patches *g);
/* The part that holds the primitive slots of a stage's input for the window
 * schedule ((NV + 1) FP64 words a pooled cell; see wc_prim_buffer_bytes). */
size_t wc_patches_prim_buffer_bytes(const wc_patches *g);
/* Binds the pooled device state and workspace (256-byte aligned), uploads
 * the patch table on stream and synchronises it.  A workspace of at least
 * wc_patches_workspace_bytes - wc_patches_face_buffer_bytes is accepted:
 * without the face buffer the window schedule's mixed-precision sweep runs
 * in one pass, and with less than that minus wc_patches_prim_buffer_bytes
 * too the window sweeps convert their cells themselves (the same results,
 * bit for bit); below that, WC_ERR_ARG. */
wc_status wc_patches_set_state(wc_patches *g, double *U_dev, void *workspace_dev,
                               size_t ws_bytes, void *stream);
/* Schedule: threads per CTA (32/64/96/128), CTAs per SM (1..16), and the
 * kind: 1 one persistent launch per stage, CTAs taking whole patches from a
 * queue (largest first), each thread marching whole pencils; 0 the same with
 * a static round-robin; 2 window sweeps: per direction, one launch per
 * group of equal patches over all their pencils, one cell per lane in
 * windows of 32 (the grids' sweep, pencils mapped to patches through an
 * offset table; outflow cells at every pencil end), in mixed precision the
 * face and flux passes of the split sweep; block and CTAs per SM are then
 * those of the window sweep.  Anything else: WC_ERR_ARG. */
wc_status wc_patches_set_schedule(wc_patches *g, int block, int ctas_per_sm, int dynamic);
/* nsteps SSP-RK3 steps of every patch, one global dt (cfl, or dt_fixed > 0)
 * from all patches.  use_graph = 1 captures one step (rate reduction, queue
 * reset, the stage launches) into a CUDA graph on the first call and
 * replays it; stream must then be a created stream, not the legacy default. */
wc_status wc_patches_rk_step(wc_patches *g, double cfl, double dt_fixed, int nsteps,
                             int use_graph, void *stream);
/* psi_{V->U} (Eq. 26) on the pooled [NV][ncell_total] arrays. */
wc_status wc_patches_prim_to_cons(const wc_patches *g, const double *V_dev, double *U_dev,
                                  void *stream);
/* dU/dt of every patch for the pooled state U_dev into L_dev (Eq. 3). */
wc_status wc_patches_rhs(wc_patches *g, const double *U_dev, double *L_dev, void *stream);
wc_status wc_patches_sync_status(wc_patches *g, void *stream);
/* Times every candidate schedule (block 64/128 x CTAs per SM 2/3/4/6 x
 * dynamic/static persistent launches, and window sweeps of 128-thread
 * blocks at 2/3/4 per SM) over `steps` steps on a copy of the bound state
 * (the state is restored), applies and returns the fastest. */
wc_status wc_patches_autotune(wc_patches *g, double cfl, int steps, void *stream, int *block,
                              int *ctas_per_sm, int *dynamic, double *ms_per_step);
void wc_patches_last_error(const wc_patches *g, char *buf, size_t n);

/* Sweep timing (tracing): after wc_sweep_timing_begin(g, max_launches) the
 * library records a CUDA event pair on the launch stream around each of the
 * next max_launches direction-sweep launches of g and around the
 * primitive-slot passes of their stages (events are created here, no device
 * memory is allocated).  wc_sweep_timing_read synchronises on the last event
 * and returns the number of timed sweeps, the summed durations of the sweeps
 * and passes (so total / launches is a sweep with its share of its stage's
 * pass) and the largest sweep duration, in milliseconds, and stops the
 * timing. */
wc_status wc_sweep_timing_begin(wc_grid *g, int max_launches);
wc_status wc_sweep_timing_read(wc_grid *g, int *launches, double *total_ms, double *max_ms);

/* Synchronises the stream, reads and clears the device status word; returns
 * WC_OK or the first kernel-detected error. */
wc_status wc_sync_status(wc_grid *g, void *stream);

/* Copies the last error message into buf (NUL-terminated). */
void wc_last_error(const wc_grid *g, char *buf, size_t n);

/* Measured FP64 peak helper: runs a dependent-free DFMA loop of iters
 * iterations on blocks x threads threads and returns the flop count
 * (2 per DFMA) through *flops; time it with events on the stream. */
wc_status wc_fp64_peak_kernel(int blocks, int threads, int iters, double *sink_dev,
                              double *flops, void *stream);

/* The binary64 <-> binary32 conversions of the reduced-precision sweeps
 * (integer-pipe arithmetic on the IEEE 754 formats, the hardware conversion
 * for zeros, subnormals, infinities, NaNs and overflow): f_dev[i] = x_dev[i]
 * rounded to binary32 (nearest, ties to even) and back_dev[i] = f_dev[i]
 * widened to binary64, for i < n (device arrays of n elements).  The paper
 * has no counterpart; it lets a test hold them to the hardware conversions
 * bit for bit.  Asynchronous on stream. */
wc_status wc_convert_f32(const double *x_dev, float *f_dev, double *back_dev, long n,
                         void *stream);

/* The grid barrier of the Q-map's cooperative launch on its own: one block
 * of 256 threads per SM passes `rounds` barriers (words_dev: 4 device ints,
 * cleared by the call).  skip_block >= 0 makes that block leave before the
 * first barrier, so every other block's bounded wait runs out: the call then
 * returns WC_ERR_TIMEOUT (after a few seconds) and the context stays usable.
 * skip_block = -1: every block arrives, WC_OK.  The paper has no
 * counterpart; it lets a test exercise the barrier and its time-out.
 * Synchronizes stream. */
wc_status wc_grid_barrier_check(int *words_dev, int skip_block, int rounds, void *stream);

/* The neighbour barrier of the Q-map preconditioner's exchanges on its own:
 * one block of 256 threads per SM, blocks on a line, block b waiting in each
 * of `rounds` exchanges for the blocks within `span` (>= 1) of it (its
 * neighbours' epoch flags, acquire loads, bounded polls).  words_dev: at
 * least wc_neighbour_barrier_words() device ints (cleared by the call; 0 if
 * the device cannot be queried), nwords their number (WC_ERR_ARG if fewer).
 * skip_block >= 0 makes that block leave before the first exchange: its
 * neighbours' waits run out, every other block stops waiting on the error
 * word, and the call returns WC_ERR_TIMEOUT (after a few seconds) with the
 * context usable; skip_block = -1: WC_OK.  The paper has no counterpart; it
 * lets a test exercise the barrier and its time-out.  Synchronizes stream. */
size_t wc_neighbour_barrier_words(void);
wc_status wc_neighbour_barrier_check(int *words_dev, size_t nwords, int skip_block, int span,
                                     int rounds, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* WENOC_H */
