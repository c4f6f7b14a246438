/*
 * wenoc_oracle.c -- plain, slow, FP64 CPU oracle of the WENO-C finite-volume
 * operator of Huang, "Consistent and bound-preserving finite-volume WENO
 * scheme for compressible two-/N-phase flows with Phase-Field mechanism".
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header
 * or constant table with the CUDA path; it is the definition the CUDA path is
 * compared against.  Everything is FP64, evaluated literally, one cell and one
 * face at a time, in the order the paper states the steps (Eq. 15 -> Eq. 16 ->
 * Eq. 17/18 -> Eq. 19 -> Eq. 20 -> Eq. 21 -> flux -> Eq. 3 -> SSP-RK3).
 * Build with -ffp-contract=off so that no fused multiply-add changes the
 * rounding of the plain expressions below.
 *
 * Readings where the paper is silent or ambiguous (each one is listed in the
 * design notes of the repository):
 *  R1  WENO5 candidates, ideal weights and smoothness indicators are the
 *      uniform-mesh Jiang-Shu ones (Sec. 3.1 cites them; only the r = 1 case
 *      is printed, Eq. 11).  The right-face value f^R_{i-1/2} uses the mirrored
 *      stencil.
 *  R2  Eq. 15 with IS_k = 0 < IS_s: the ratio is infinite, so omega_s = 0.
 *  R3  Eq. 18: theta = 1 whenever min(f^C, f^L, f^R) >= f_min (this covers the
 *      printed 0/0 and x/0 cases); theta is clamped to [0, 1] (the paper states
 *      theta in [0, 1]) when the cell average itself is below f_min.
 *  R4  f_min = 0 for both the masses and the volume fractions (positivity).
 *  R5  psi of Eq. 9 with the Eq. 26 equation of state; the minimum pressures
 *      P_min are inputs.  theta^(psi) uses psi(U^C) with U^C from inverting
 *      Eq. 6 (N_quad = 4, w_1 = w_4 = 1/12, Sec. 4.2).
 *  R6  The Riemann solver receives, for each face state, the conservative
 *      vector U and the primitive vector V with U = psi_{V->U}(V).  When the
 *      energy limiter leaves the state unchanged (theta^(psi) = 1) V is the
 *      reconstructed primitive state; otherwise V is recovered from the
 *      limited U by Eq. 27.
 *  R7  HLL uses the Davis wave-speed estimates; HLLC is Toro's, with the
 *      masses and the volume fractions both scaled by (S_K-u_K)/(S_K-S*) in
 *      the star state (keeps mass/fraction consistency).  u-hat is the
 *      volume-fraction flux with alpha = 1 on both sides (Sec. 2.2.1).
 *  R8  Mixture sound speed of Eq. 2 for K_p = 0 (Allaire et al.), with the
 *      stiffened-gas phasic rho_p c_p^2 = gamma_p (P + Pinf_p).
 *  R9  Boundary cells: periodic copy; reflective mirror with the normal
 *      momentum negated; outflow zero-gradient copy.
 *  R10 Time step dt = CFL / max_cells sum_d (|u_d| + c) / dx_d, taken from U^n.
 *  R12 Phase-Field flux of Eq. 5 (its numerical form is not printed in the
 *      paper; parity unpinned beyond its invariants).  Given Q_p at cells,
 *      G_p = (Q_{p,R} - Q_{p,L})/dx at the face (0 on a face where both
 *      cells have phi_p (1 - phi_p) <= 0: Eq. 4 does not couple it, R17);
 *      with J_p = phi_p(1-phi_p)
 *      grad Q_p (implied by Eq. 4) discretised bound-preservingly as
 *      J_p = max(G_p,0) a_R (1 - a_L) + min(G_p,0) a_L (1 - a_R), the mass flux
 *      is the same with (alpha rho) in the outgoing factor, then
 *      sum_p J_p = 0 is enforced by removing sum_q J_q in proportion to the
 *      face fractions (a_L + a_R)/2 (masses with (alpha rho)_face); momentum
 *      and energy follow Eq. 1: sum_p F^{m_p} u_face and
 *      sum_p [F^{m_p} |u|^2/2 + F^{a_p} (A_p P + B_p) + D_p F^{m_p}], u_face and
 *      P_face the averages of the two face states.
 *  R11 Eq. 19 assumes S > 0.  When the positivity step has limited every
 *      fraction of a face to zero (S = 0) the cell keeps its averages on both
 *      faces (theta = 0, first order) for the masses and the fractions.
 *  R14 WENO-CL (Sec. 3.4, Eq. 23-25) replaces Eq. 19.  The gradients S of
 *      Eq. 24 enter Eq. 23 and Eq. 25 only through ratios and through
 *      theta S dx/2, so the common factor 2/dx is dropped: S_p = f_face -
 *      fbar.  p-hat is the first phase of largest |S^(alpha_p)|.  When every
 *      S^(alpha_p) of a face is zero the faces are left as they are; a
 *      ratio x/0 with x != 0 is +-infinity before the clamp to [0, 1].
 *      Eq. 20 and Eq. 21 follow as in WENO-C.
 *  R15 Kapila model (Sec. 2.1): K_p = rho c^2 / (rho_p c_p^2) - 1.  Put into
 *      Eq. 2 this is an identity for any rho c^2; the constraint
 *      sum_p alpha_p K_p = 0 stated with Eq. 2 fixes it: 1 / (rho c^2) =
 *      sum_p alpha_p / (rho_p c_p^2) (Wood), rho_p c_p^2 = gamma_p (P +
 *      Pinf_p).  The source factor alpha_p (1 + K_p) of Eq. 3 is evaluated
 *      at the cell average (as for K_p = 0); the wave speeds and the time
 *      step use this mixture sound speed.  In the sound speed a fraction
 *      below zero (an excursion of the scheme above its bound-preserving CFL
 *      number, or the rounding residue of R13) enters Wood's sum as zero: a
 *      phase cannot add negative compressibility, and at a low-pressure face
 *      state a gas fraction of -4e-4 beside water already turns the
 *      unclipped sum negative, leaving no real speed.  The source factors
 *      keep the sum over the fractions as they are: only then does sum_p
 *      alpha_p (1 + K_p) = 1 hold, which keeps the fraction sum at one.
 *  R13 Rounding residue below the bounds.  In exact arithmetic the faces
 *      scaled by Eq. 18 (f_min = 0), Eq. 20 and Eq. 21 have non-negative
 *      masses and fractions, and every Runge-Kutta stage (a convex
 *      combination of forward-Euler steps under the CFL condition, Sec. 4)
 *      keeps the cell masses non-negative and the fractions in [0, 1].  In
 *      floating point fbar + theta (f - fbar), meant to land on 0, can land
 *      an ulp below it; an absent phase's vanishing tail then becomes a
 *      negative average, and Eq. 18 on a negative average (theta = 0) taken
 *      into Eq. 20's minimum over phases drops the whole cell to first order.
 *      Such residues are set to the bound: scaled face masses and fractions
 *      below 0 become 0 when the cell average is non-negative, and stage
 *      results outside the bounds by at most 2^-48 of the magnitudes of the
 *      stage sum's terms become the bound.  A larger excursion is not
 *      rounding: at a time step above the sufficient CFL bound of Sec. 4.2
 *      (the paper's own tests run so) the scheme itself can leave the bounds
 *      slightly; that value stays, the next limiter (theta = 0 on a negative
 *      average) takes the cell to first order, and no clamp breaks the
 *      consistency of (alpha_p rho_p) and alpha_p or the pressure
 *      equilibrium (Sec. 4.1.1: WENO-C keeps both at round-off).
 *  R16 Comparison schemes (Sec. 3.2, Sec. 4.1.1: WENO-JS and WENO-W without
 *      Eq. 16-21).  Each primitive variable is reconstructed with its own
 *      weights and the faces go to the Riemann solver unlimited.  Without
 *      the limiters nothing keeps the stages inside the bounds, so values
 *      outside them are overshoots of the scheme, not rounding residue:
 *      R13's stage clamp is not applied (clamping alpha_1 at 1 while
 *      (alpha_1 rho_1) overshoots would itself break consistency).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Operation counting (OR_COUNT, a C++ build with oracle/op_count.hpp forced
 * in front): OR_CAT(c) attributes the arithmetic of the enclosing scope to
 * category c.  In the plain C build it expands to nothing. */
#ifdef OR_COUNT
extern "C" {
long long or_op_counts[OR_C_NCAT][OR_K_N];
void or_op_counts_reset(void) { memset(or_op_counts, 0, sizeof(or_op_counts)); }
void or_op_counts_read(long long *out) { memcpy(out, or_op_counts, sizeof(or_op_counts)); }
}
int or_op_cat = OR_C_OTHER;
#else
#define OR_CAT(c)
#endif
#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXP 8
#define OR_MAXV (2 * OR_MAXP + 4)

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_INADMISSIBLE = 3, OR_ERR_NAN = 4 };
enum { OR_BC_PERIODIC = 0, OR_BC_REFLECTIVE = 1, OR_BC_OUTFLOW = 2 };
enum { OR_FLUX_HLL = 0, OR_FLUX_HLLC = 1 };
enum { OR_WEIGHTS_W = 0, OR_WEIGHTS_JS = 1 };

typedef struct {
  int dim;              /* 1, 2 or 3 */
  int n[3];             /* interior cells per axis (1 for unused axes) */
  double dx[3];         /* uniform cell sizes */
  int N;                /* number of phases */
  double gamma[OR_MAXP], pinf[OR_MAXP], D[OR_MAXP], pmin[OR_MAXP];
  int flux;             /* OR_FLUX_HLL / OR_FLUX_HLLC */
  int weights;          /* OR_WEIGHTS_W (Eq. 15) or OR_WEIGHTS_JS (Eq. 12 form) */
  double js_eps;        /* epsilon of the JS comparator */
  int coupled;          /* 1: Eq. 16 coupling (WENO-C); 0: own weights per variable */
  int limiter;          /* 1: Eq. 17-20 applied; 0: skipped */
  int energy_limiter;   /* 1: Eq. 21 applied; 0: skipped */
  int bc[6];            /* lo/hi per axis: OR_BC_* */
  int consistent;       /* 0: Eq. 19 (WENO-C); 1: Eq. 23-25 (WENO-CL) */
  int kmodel;           /* K_p of Eq. 2-3: 0 Allaire (K_p = 0); 1 Kapila (R15) */
} or_grid;

/* ---- state layout ---------------------------------------------------------
 * U = [ (alpha rho)_1..N, (rho u)_1..d, rho E, alpha_1..N ]   (Eq. 1)
 * V = [ (alpha rho)_1..N,  u_1..d,       P,    alpha_1..N ]   (Sec. 2.2.2)
 */
static int nv(const or_grid *g) { return 2 * g->N + g->dim + 1; }
#define IMASS(p) (p)
#define IMOM(g, j) ((g)->N + (j))
#define IENE(g) ((g)->N + (g)->dim)
#define IALF(g, p) ((g)->N + (g)->dim + 1 + (p))

int or_nv(const or_grid *g) { return nv(g); }

/* Threads of the parallel sweeps (the CPU baselines time 1 and all). */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Eq. 26: A_p = 1/(gamma_p - 1), B_p = gamma_p Pinf_p / (gamma_p - 1). */
static double eos_A(const or_grid *g, int p) {
  OR_CAT(OR_C_CONST);
  return 1.0 / (g->gamma[p] - 1.0);
}
static double eos_B(const or_grid *g, int p) {
  OR_CAT(OR_C_CONST);
  return g->gamma[p] * g->pinf[p] / (g->gamma[p] - 1.0);
}

/* Mixture rules (Sec. 2.1) and the pressure of Eq. 27. */
static int cons_to_prim(const or_grid *g, const double *U, double *V) {
  OR_CAT(OR_C_PRIM);
  int N = g->N, d = g->dim;
  double rho = 0.0;
  for (int p = 0; p < N; p++) rho += U[IMASS(p)];
  if (!(rho > 0.0)) return OR_ERR_INADMISSIBLE;
  double mm = 0.0;
  for (int j = 0; j < d; j++) mm += U[IMOM(g, j)] * U[IMOM(g, j)];
  double sA = 0.0, sB = 0.0, sD = 0.0;
  for (int p = 0; p < N; p++) {
    sA += eos_A(g, p) * U[IALF(g, p)];
    sB += eos_B(g, p) * U[IALF(g, p)];
    sD += g->D[p] * U[IMASS(p)];
  }
  double P = (U[IENE(g)] - 0.5 * mm / rho - sB - sD) / sA;
  for (int p = 0; p < N; p++) {
    V[IMASS(p)] = U[IMASS(p)];
    V[IALF(g, p)] = U[IALF(g, p)];
  }
  for (int j = 0; j < d; j++) V[IMOM(g, j)] = U[IMOM(g, j)] / rho;
  V[IENE(g)] = P;
  return isfinite(P) ? OR_OK : OR_ERR_NAN;
}

/* psi_{V->U}: rho = sum (alpha rho)_p, rho u, and rho E from Eq. 26. */
static void prim_to_cons(const or_grid *g, const double *V, double *U) {
  OR_CAT(OR_C_V2U);
  int N = g->N, d = g->dim;
  double rho = 0.0;
  for (int p = 0; p < N; p++) rho += V[IMASS(p)];
  double uu = 0.0;
  for (int j = 0; j < d; j++) uu += V[IMOM(g, j)] * V[IMOM(g, j)];
  double P = V[IENE(g)];
  double e = 0.0;
  for (int p = 0; p < N; p++)
    e += V[IALF(g, p)] * (eos_A(g, p) * P + eos_B(g, p)) + g->D[p] * V[IMASS(p)];
  for (int p = 0; p < N; p++) {
    U[IMASS(p)] = V[IMASS(p)];
    U[IALF(g, p)] = V[IALF(g, p)];
  }
  for (int j = 0; j < d; j++) U[IMOM(g, j)] = rho * V[IMOM(g, j)];
  U[IENE(g)] = e + 0.5 * rho * uu;
}

/* Eq. 9 with Eq. 26: psi = rho E - |rho u|^2 / (2 rho)
 *                         - sum_p [ alpha_p (A_p Pmin_p + B_p) + D_p (alpha rho)_p ]. */
static double psi_energy(const or_grid *g, const double *U) {
  int N = g->N, d = g->dim;
  double rho = 0.0;
  for (int p = 0; p < N; p++) rho += U[IMASS(p)];
  double mm = 0.0;
  for (int j = 0; j < d; j++) mm += U[IMOM(g, j)] * U[IMOM(g, j)];
  double s = 0.0;
  for (int p = 0; p < N; p++)
    s += U[IALF(g, p)] * (eos_A(g, p) * g->pmin[p] + eos_B(g, p)) + g->D[p] * U[IMASS(p)];
  /* a face whose masses were all limited to zero carries rho u = 0: the
   * kinetic term tends to zero with rho */
  double ke = rho > 0.0 ? 0.5 * mm / rho : 0.0;
  return U[IENE(g)] - ke - s;
}

/* ---- WENO5 building blocks (R1) ------------------------------------------
 * f[0..4] = cell averages f_{i-2..i+2}; values at x_{i+1/2} of the three
 * quadratic candidates of sub-stencils s = {i-2..i}, {i-1..i+1}, {i..i+2},
 * and their smoothness indicators. */
void or_weno5_parts(const double *f, double *q, double *beta) {
  {
    OR_CAT(OR_C_CAND);
    q[0] = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;
    q[1] = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;
    q[2] = (2.0 * f[2] + 5.0 * f[3] - f[4]) / 6.0;
  }
  {
    OR_CAT(OR_C_BETA);
    double a, b;
    a = f[0] - 2.0 * f[1] + f[2];
    b = f[0] - 4.0 * f[1] + 3.0 * f[2];
    beta[0] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = f[1] - 2.0 * f[2] + f[3];
    b = f[1] - f[3];
    beta[1] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = f[2] - 2.0 * f[3] + f[4];
    b = 3.0 * f[2] - 4.0 * f[3] + f[4];
    beta[2] = 13.0 / 12.0 * a * a + 0.25 * b * b;
  }
}

static const double weno5_d[3] = {0.1, 0.6, 0.3};

/* Eq. 15: omega_s = d_s / (d_s + sum_{k != s} d_k (IS^(s,k))^2),
 * IS^(s,k) = 1 if IS_s = IS_k = 0, else IS_s / IS_k (R2 for IS_k = 0). */
void or_wenow_weights(const double *beta, double *w) {
  for (int s = 0; s < 3; s++) {
    double den = weno5_d[s];
    int infinite = 0;
    for (int k = 0; k < 3; k++) {
      if (k == s) continue;
      double r;
      if (beta[s] == 0.0 && beta[k] == 0.0) r = 1.0;
      else if (beta[k] == 0.0) { infinite = 1; r = 0.0; }
      else r = beta[s] / beta[k];
      den += weno5_d[k] * r * r;
    }
    w[s] = infinite ? 0.0 : weno5_d[s] / den;
  }
}

/* WENO-JS comparator (Eq. 12 in the fifth-order form): w_s ~ d_s/(IS_s+eps)^2. */
void or_wenojs_weights(const double *beta, double eps, double *w) {
  double a[3], s = 0.0;
  for (int k = 0; k < 3; k++) {
    a[k] = weno5_d[k] / ((beta[k] + eps) * (beta[k] + eps));
    s += a[k];
  }
  for (int k = 0; k < 3; k++) w[k] = a[k] / s;
}

static void weights(const or_grid *g, const double *beta, double *w) {
  OR_CAT(OR_C_WEIGHTS);
  if (g->weights == OR_WEIGHTS_JS) or_wenojs_weights(beta, g->js_eps, w);
  else or_wenow_weights(beta, w);
}

/* Eq. 10: f^L = sum_s omega_s f^(s). */
static double combine(const double *w, const double *q) {
  OR_CAT(OR_C_COMBINE);
  return w[0] * q[0] + w[1] * q[1] + w[2] * q[2];
}

/* Eq. 6 inverted for U^C with N_quad = 4 Gauss-Lobatto points, w_1 = 1/12. */
static double center_value(double fbar, double fL, double fR) {
  const double w1 = 1.0 / 12.0;
  return (fbar - w1 * fR - w1 * fL) / (1.0 - 2.0 * w1);
}

/* Eq. 18 with the explicit interior value f^C (R3). */
static double theta_lower(double fbar, double fC, double fL, double fR, double fmin) {
  double m = fC;
  if (fL < m) m = fL;
  if (fR < m) m = fR;
  if (m >= fmin) return 1.0;
  if (fbar <= fmin) return 0.0;
  double t = (fbar - fmin) / (fbar - m);
  return t < 1.0 ? t : 1.0;
}

/* R13 bookkeeping for the tests (no effect on any result): the face values
 * the face rule set to 0 (count, largest |x| / fbar) and a histogram of the
 * stage values found outside a bound, by floor(log2(excursion / sum of the
 * terms' magnitudes)) from -64 to +1, whether the stage rule clamped them
 * or not.  The stage rule's tolerance is a parameter only so that the tests
 * can run the method with another one. */
static double or_stage_tol = 0x1p-48;
static double r13_face_n, r13_face_max, r13_hist[66];

void or_r13_set_stage_tol(double tol) { or_stage_tol = tol; }
void or_r13_reset(void) {
  r13_face_n = r13_face_max = 0.0;
  for (int i = 0; i < 66; i++) r13_hist[i] = 0.0;
}
void or_r13_stats(double *out) {
  out[0] = r13_face_n;
  out[1] = r13_face_max;
  for (int i = 0; i < 66; i++) out[2 + i] = r13_hist[i];
}

/* R13: fbar + theta (f - fbar) below the bound 0 is rounding residue when
 * fbar >= 0 and becomes 0; with fbar < 0 (theta = 0, a stage that left the
 * bound) the value is fbar itself and stays. */
static double clamp0(double x, double fbar) {
  if (x < 0.0 && fbar >= 0.0) {
    double r = fbar > 0.0 ? -x / fbar : INFINITY;
#ifdef _OPENMP
#pragma omp critical(r13)
#endif
    {
      r13_face_n += 1.0;
      if (r > r13_face_max) r13_face_max = r;
    }
    return 0.0;
  }
  return x;
}

static double theta_pos(double fbar, double fL, double fR) {
  return theta_lower(fbar, center_value(fbar, fL, fR), fL, fR, 0.0);
}

/* The limiter chain of WENO-C for one cell and one direction.
 * Ubar: cell average (conservative).  VL, VR: reconstructed primitive values
 * at x_{i+1/2} (left state of that face) and x_{i-1/2} (right state), modified
 * in place by Eq. 17-20.  UL, UR: final conservative face states (Eq. 21).
 * VfL, VfR: primitive face states handed to the Riemann solver (R6).
 * th (optional, 3 values): min_p theta_p of Eq. 17, theta_i of Eq. 20,
 * theta^(psi) of Eq. 21. */
static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* Eq. 23-25 on one face (V holds the face's primitive values): with
 * S_p = alpha_p,face - alpha_p,bar (R14), p-hat = argmax |S_p|,
 * S-hat = S_phat - sum_p S_p, theta_phat = clamp(S-hat / S_phat) and
 * theta_p = clamp(S_phat / S-hat) otherwise; the phase's mass and fraction
 * both move to fbar + theta (f_face - fbar). */
static void consistent_limiter(const or_grid *g, const double *Ubar, double *V) {
  int N = g->N, ph = 0;
  double S[OR_MAXP], sum = 0.0, best = -1.0;
  for (int p = 0; p < N; p++) {
    S[p] = V[IALF(g, p)] - Ubar[IALF(g, p)];
    sum += S[p];
    if (fabs(S[p]) > best) {
      best = fabs(S[p]);
      ph = p;
    }
  }
  if (S[ph] == 0.0) return; /* every gradient is zero */
  double Shat = S[ph] - sum;
  for (int p = 0; p < N; p++) {
    double th;
    if (p == ph) th = clamp01(Shat / S[ph]);
    else if (Shat == 0.0) th = S[ph] > 0.0 ? 1.0 : 0.0; /* S_phat / 0 = +-inf */
    else th = clamp01(S[ph] / Shat);
    double mb = Ubar[IMASS(p)], ab = Ubar[IALF(g, p)];
    V[IMASS(p)] = clamp0(mb + th * (V[IMASS(p)] - mb), mb);
    V[IALF(g, p)] = clamp0(ab + th * (V[IALF(g, p)] - ab), ab);
  }
}

static int limit_chain(const or_grid *g, const double *Ubar, double *VL, double *VR,
                       double *UL, double *UR, double *VfL, double *VfR, double *th) {
  OR_CAT(OR_C_LIMIT);
  int N = g->N, nvar = nv(g);
  double th17 = 1.0, th20 = 1.0, thpsi = 1.0;
  if (g->limiter) {
    /* Eq. 17-18: positivity of (alpha rho)_p and alpha_p with a common theta_p. */
    for (int p = 0; p < N; p++) {
      double mb = Ubar[IMASS(p)], ab = Ubar[IALF(g, p)];
      double t1 = theta_pos(mb, VL[IMASS(p)], VR[IMASS(p)]);
      double t2 = theta_pos(ab, VL[IALF(g, p)], VR[IALF(g, p)]);
      double tp = t1 < t2 ? t1 : t2;
      if (tp < th17) th17 = tp;
      if (tp < 1.0) {
        VL[IMASS(p)] = clamp0(mb + tp * (VL[IMASS(p)] - mb), mb);
        VR[IMASS(p)] = clamp0(mb + tp * (VR[IMASS(p)] - mb), mb);
        VL[IALF(g, p)] = clamp0(ab + tp * (VL[IALF(g, p)] - ab), ab);
        VR[IALF(g, p)] = clamp0(ab + tp * (VR[IALF(g, p)] - ab), ab);
      }
    }
    if (g->consistent) {
      /* Eq. 23-25 (WENO-CL, R14) on each face instead of Eq. 19. */
      consistent_limiter(g, Ubar, VL);
      consistent_limiter(g, Ubar, VR);
    } else {
    /* Eq. 19: unity sum of the volume fractions on each face. */
    double SL = 0.0, SR = 0.0;
    for (int p = 0; p < N; p++) {
      SL += VL[IALF(g, p)];
      SR += VR[IALF(g, p)];
    }
    if (!(SL > 0.0) || !(SR > 0.0)) {
      /* R11: every fraction of a face was limited to zero, so Eq. 19 has no
       * sum to divide by; the cell falls back to its averages (theta = 0). */
      for (int p = 0; p < N; p++) {
        VL[IMASS(p)] = VR[IMASS(p)] = Ubar[IMASS(p)];
        VL[IALF(g, p)] = VR[IALF(g, p)] = Ubar[IALF(g, p)];
      }
      th17 = 0.0;
      SL = SR = 1.0;
    }
    for (int p = 0; p < N; p++) {
      VL[IMASS(p)] = VL[IMASS(p)] / SL;
      VL[IALF(g, p)] = VL[IALF(g, p)] / SL;
      VR[IMASS(p)] = VR[IMASS(p)] / SR;
      VR[IALF(g, p)] = VR[IALF(g, p)] / SR;
    }
    }
    /* Eq. 20: theta_i = min_p theta_p recomputed from the normalised faces. */
    for (int p = 0; p < N; p++) {
      double t1 = theta_pos(Ubar[IMASS(p)], VL[IMASS(p)], VR[IMASS(p)]);
      double t2 = theta_pos(Ubar[IALF(g, p)], VL[IALF(g, p)], VR[IALF(g, p)]);
      double tp = t1 < t2 ? t1 : t2;
      if (tp < th20) th20 = tp;
    }
    for (int p = 0; p < N; p++) {
      double mb = Ubar[IMASS(p)], ab = Ubar[IALF(g, p)];
      if (th20 < 1.0) {
        VL[IMASS(p)] = clamp0(mb + th20 * (VL[IMASS(p)] - mb), mb);
        VR[IMASS(p)] = clamp0(mb + th20 * (VR[IMASS(p)] - mb), mb);
        VL[IALF(g, p)] = clamp0(ab + th20 * (VL[IALF(g, p)] - ab), ab);
        VR[IALF(g, p)] = clamp0(ab + th20 * (VR[IALF(g, p)] - ab), ab);
      }
    }
  }
  /* V -> U at both faces. */
  prim_to_cons(g, VL, UL);
  prim_to_cons(g, VR, UR);
  if (g->energy_limiter) {
    /* Eq. 21 with psi evaluated at Ubar, U^L, U^R and U^C (R5). */
    double UC[OR_MAXV];
    for (int v = 0; v < nvar; v++) UC[v] = center_value(Ubar[v], UL[v], UR[v]);
    double pb = psi_energy(g, Ubar);
    double pL = psi_energy(g, UL), pR = psi_energy(g, UR), pC = psi_energy(g, UC);
    thpsi = theta_lower(pb, pC, pL, pR, 0.0);
    if (thpsi < 1.0) {
      for (int v = 0; v < nvar; v++) {
        UL[v] = Ubar[v] + thpsi * (UL[v] - Ubar[v]);
        UR[v] = Ubar[v] + thpsi * (UR[v] - Ubar[v]);
      }
      for (int p = 0; p < N; p++) {
        UL[IMASS(p)] = clamp0(UL[IMASS(p)], Ubar[IMASS(p)]);
        UR[IMASS(p)] = clamp0(UR[IMASS(p)], Ubar[IMASS(p)]);
        UL[IALF(g, p)] = clamp0(UL[IALF(g, p)], Ubar[IALF(g, p)]);
        UR[IALF(g, p)] = clamp0(UR[IALF(g, p)], Ubar[IALF(g, p)]);
      }
    }
  }
  if (thpsi < 1.0) {
    int e1 = cons_to_prim(g, UL, VfL), e2 = cons_to_prim(g, UR, VfR);
    if (e1) return e1;
    if (e2) return e2;
  } else {
    memcpy(VfL, VL, sizeof(double) * nvar);
    memcpy(VfR, VR, sizeof(double) * nvar);
  }
  if (th) {
    th[0] = th17;
    th[1] = th20;
    th[2] = thpsi;
  }
  return OR_OK;
}

/* Reconstruction of cell i in one direction: Ust = conservative averages of
 * cells i-2..i+2 (NV each).  Outputs the limited face states of the cell. */
static int recon_cell(const or_grid *g, const double *Ust, double *UL, double *UR,
                      double *VfL, double *VfR, double *th) {
  OR_CAT(OR_C_RECON);
  int N = g->N, d = g->dim, nvar = nv(g);
  double Vst[5][OR_MAXV];
  for (int k = 0; k < 5; k++) {
    int e = cons_to_prim(g, Ust + k * nvar, Vst[k]);
    if (e) return e;
  }
  double qL[OR_MAXV][3], bL[OR_MAXV][3], qR[OR_MAXV][3], bR[OR_MAXV][3];
  for (int v = 0; v < nvar; v++) {
    double f[5], fm[5];
    for (int k = 0; k < 5; k++) {
      f[k] = Vst[k][v];
      fm[k] = Vst[4 - k][v];
    }
    or_weno5_parts(f, qL[v], bL[v]);
    or_weno5_parts(fm, qR[v], bR[v]);
  }
  double VL[OR_MAXV], VR[OR_MAXV], w[3];
  for (int p = 0; p < N; p++) {
    /* Eq. 16: the weights of (alpha rho)_p reconstruct both (alpha rho)_p and alpha_p. */
    weights(g, bL[IMASS(p)], w);
    VL[IMASS(p)] = combine(w, qL[IMASS(p)]);
    if (!g->coupled) weights(g, bL[IALF(g, p)], w);
    VL[IALF(g, p)] = combine(w, qL[IALF(g, p)]);
    weights(g, bR[IMASS(p)], w);
    VR[IMASS(p)] = combine(w, qR[IMASS(p)]);
    if (!g->coupled) weights(g, bR[IALF(g, p)], w);
    VR[IALF(g, p)] = combine(w, qR[IALF(g, p)]);
  }
  /* u and P: each reconstructed with its own WENO-W weights (Sec. 3.3). */
  for (int v = N; v <= N + d; v++) {
    weights(g, bL[v], w);
    VL[v] = combine(w, qL[v]);
    weights(g, bR[v], w);
    VR[v] = combine(w, qR[v]);
  }
  return limit_chain(g, Ust + 2 * nvar, VL, VR, UL, UR, VfL, VfR, th);
}

/* rho c^2 of the mixture for the pressure P and fractions alpha: Eq. 2 with
 * K_p = 0 (R8), or Wood's formula for the Kapila model (R15), whose sum takes
 * a negative fraction as zero when clip is set (the sound speed). */
static double mixture_rhoc2(const or_grid *g, const double *alpha, double P, int clip) {
  int N = g->N;
  if (g->kmodel) {
    double s = 0.0;
    for (int p = 0; p < N; p++) {
      double a = clip && alpha[p] < 0.0 ? 0.0 : alpha[p];
      s += a / (g->gamma[p] * (P + g->pinf[p]));
    }
    return 1.0 / s;
  }
  double num = 0.0, den = 0.0;
  for (int p = 0; p < N; p++) {
    double Aa = eos_A(g, p) * alpha[p];
    num += Aa * (g->gamma[p] * (P + g->pinf[p]));
    den += Aa;
  }
  return num / den;
}

/* Mixture sound speed (R8, R15). */
static double sound_speed(const or_grid *g, const double *U, const double *V) {
  int N = g->N;
  double rho = 0.0, alpha[OR_MAXP];
  for (int p = 0; p < N; p++) {
    rho += U[IMASS(p)];
    alpha[p] = U[IALF(g, p)];
  }
  return sqrt(mixture_rhoc2(g, alpha, V[IENE(g)], 1) / rho);
}

/* Physical flux of Eq. 1 (hyperbolic part) in direction dir. */
static void phys_flux(const or_grid *g, int dir, const double *U, const double *V, double *F) {
  int N = g->N, d = g->dim;
  double un = V[IMOM(g, dir)], P = V[IENE(g)];
  for (int p = 0; p < N; p++) {
    F[IMASS(p)] = U[IMASS(p)] * un;
    F[IALF(g, p)] = U[IALF(g, p)] * un;
  }
  for (int j = 0; j < d; j++) F[IMOM(g, j)] = U[IMOM(g, j)] * un + (j == dir ? P : 0.0);
  F[IENE(g)] = un * (U[IENE(g)] + P);
}

/* HLL / HLLC numerical flux and the consistent face velocity u-hat (R7). */
int or_flux(const or_grid *g, int dir, const double *UL, const double *VL, const double *UR,
            const double *VR, double *F, double *uhat) {
  OR_CAT(OR_C_FLUX);
  int N = g->N, d = g->dim, nvar = nv(g);
  double uL = VL[IMOM(g, dir)], uR = VR[IMOM(g, dir)];
  double cL = sound_speed(g, UL, VL), cR = sound_speed(g, UR, VR);
  double sL = fmin(uL - cL, uR - cR);
  double sR = fmax(uL + cL, uR + cR);
  double FL[OR_MAXV], FR[OR_MAXV];
  phys_flux(g, dir, UL, VL, FL);
  phys_flux(g, dir, UR, VR, FR);
  if (sL >= 0.0) {
    memcpy(F, FL, sizeof(double) * nvar);
    *uhat = uL;
    return OR_OK;
  }
  if (sR <= 0.0) {
    memcpy(F, FR, sizeof(double) * nvar);
    *uhat = uR;
    return OR_OK;
  }
  if (g->flux == OR_FLUX_HLL) {
    for (int v = 0; v < nvar; v++)
      F[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) / (sR - sL);
    *uhat = (sR * uL * 1.0 - sL * uR * 1.0 + sL * sR * (1.0 - 1.0)) / (sR - sL);
    return OR_OK;
  }
  /* HLLC */
  double rL = 0.0, rR = 0.0;
  for (int p = 0; p < N; p++) {
    rL += UL[IMASS(p)];
    rR += UR[IMASS(p)];
  }
  double PL = VL[IENE(g)], PR = VR[IENE(g)];
  double sS = (PR - PL + rL * uL * (sL - uL) - rR * uR * (sR - uR)) /
              (rL * (sL - uL) - rR * (sR - uR));
  const double *UK, *VK, *FK;
  double sK, rK, uK;
  if (sS >= 0.0) { UK = UL; VK = VL; FK = FL; sK = sL; rK = rL; uK = uL; }
  else { UK = UR; VK = VR; FK = FR; sK = sR; rK = rR; uK = uR; }
  double chi = (sK - uK) / (sK - sS);
  double Us[OR_MAXV];
  for (int p = 0; p < N; p++) {
    Us[IMASS(p)] = UK[IMASS(p)] * chi;
    Us[IALF(g, p)] = UK[IALF(g, p)] * chi;
  }
  for (int j = 0; j < d; j++) Us[IMOM(g, j)] = rK * chi * (j == dir ? sS : VK[IMOM(g, j)]);
  Us[IENE(g)] = chi * (UK[IENE(g)] + (sS - uK) * (rK * sS + VK[IENE(g)] / (sK - uK)));
  for (int v = 0; v < nvar; v++) F[v] = FK[v] + sK * (Us[v] - UK[v]);
  *uhat = uK * 1.0 + sK * (1.0 * chi - 1.0);
  return OR_OK;
}

/* Boundary index map (R9).  Returns the interior index and sets *flip when the
 * normal momentum must be negated. */
static int bc_map(int j, int n, int bclo, int bchi, int *flip) {
  *flip = 0;
  if (j < 0) {
    if (bclo == OR_BC_PERIODIC) return ((j % n) + n) % n;
    if (bclo == OR_BC_REFLECTIVE) { *flip = 1; return -1 - j; }
    return 0;
  }
  if (j >= n) {
    if (bchi == OR_BC_PERIODIC) return j % n;
    if (bchi == OR_BC_REFLECTIVE) { *flip = 1; return 2 * n - 1 - j; }
    return n - 1;
  }
  return j;
}

static long ncells(const or_grid *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static void load_cell(const or_grid *g, const double *U, long cell, double *out) {
  long nc = ncells(g);
  for (int v = 0; v < nv(g); v++) out[v] = U[(long)v * nc + cell];
}

/* Limited face states of every cell of one pencil along dir (cells -1..n).
 * base = linear index of the pencil's cell 0, stride = index step along dir. */
static int pencil_faces(const or_grid *g, int dir, const double *U, long base, long stride,
                        double *FLs, double *FRs, double *VLs, double *VRs, double *TH) {
  int n = g->n[dir], nvar = nv(g);
  double Ust[5 * OR_MAXV];
  for (int i = -1; i <= n; i++) {
    for (int k = 0; k < 5; k++) {
      int flip;
      int jj = bc_map(i - 2 + k, n, g->bc[2 * dir], g->bc[2 * dir + 1], &flip);
      load_cell(g, U, base + jj * stride, Ust + k * nvar);
      if (flip) Ust[k * nvar + IMOM(g, dir)] = -Ust[k * nvar + IMOM(g, dir)];
    }
    int e = recon_cell(g, Ust, FLs + (i + 1) * nvar, FRs + (i + 1) * nvar,
                       VLs + (i + 1) * nvar, VRs + (i + 1) * nvar,
                       TH ? TH + 3 * (i + 1) : NULL);
    if (e) return e;
  }
  return OR_OK;
}

/* One direction's contribution to dU/dt (Eq. 3), added into Lout. */
static int rhs_dir(const or_grid *g, int dir, const double *U, double *Lout) {
  int nvar = nv(g), N = g->N, d = g->dim;
  int n = g->n[dir];
  long nc = ncells(g);
  long stride = dir == 0 ? 1 : (dir == 1 ? g->n[0] : (long)g->n[0] * g->n[1]);
  long npencil = nc / n;
  double dx = g->dx[dir];
  int err = OR_OK;
#pragma omp parallel
  {
    double *FLs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *FRs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *VLs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *VRs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *Fx = (double *)malloc(sizeof(double) * nvar * (n + 1));
    double *uh = (double *)malloc(sizeof(double) * (n + 1));
#pragma omp for schedule(dynamic, 4)
    for (long pc = 0; pc < npencil; pc++) {
      /* pencil pc -> linear index of its first cell */
      long base;
      if (dir == 0) base = pc * n;
      else if (dir == 1) base = (pc / g->n[0]) * ((long)g->n[0] * n) + pc % g->n[0];
      else base = pc;
      int e = pencil_faces(g, dir, U, base, stride, FLs, FRs, VLs, VRs, NULL);
      /* face m sits between cell m-1 (left state) and cell m (right state) */
      for (int m = 0; m <= n && !e; m++)
        e = or_flux(g, dir, FLs + m * nvar, VLs + m * nvar, FRs + (m + 1) * nvar,
                    VRs + (m + 1) * nvar, Fx + m * nvar, uh + m);
      if (e) {
#pragma omp critical
        err = e;
        continue;
      }
      for (int m = 0; m < n; m++) {
        OR_CAT(OR_C_UPDATE);
        long cell = base + m * stride;
        for (int v = 0; v < nvar; v++)
          Lout[v * nc + cell] += -(Fx[(m + 1) * nvar + v] - Fx[m * nvar + v]) / dx;
        /* H^HB(Ubar) div(u-hat): alpha_p (1 + K_p) at the cell average */
        double onepk[OR_MAXP];
        for (int p = 0; p < N; p++) onepk[p] = 1.0;
        if (g->kmodel) {
          double uc[OR_MAXV], vc[OR_MAXV], alpha[OR_MAXP];
          for (int v = 0; v < nvar; v++) uc[v] = U[(long)v * nc + cell];
          cons_to_prim(g, uc, vc);
          for (int p = 0; p < N; p++) alpha[p] = uc[IALF(g, p)];
          double rhoc2 = mixture_rhoc2(g, alpha, vc[IENE(g)], 0);
          for (int p = 0; p < N; p++)
            onepk[p] = rhoc2 / (g->gamma[p] * (vc[IENE(g)] + g->pinf[p]));
        }
        for (int p = 0; p < N; p++) {
          double ab = U[(long)IALF(g, p) * nc + cell];
          Lout[(long)IALF(g, p) * nc + cell] += ab * onepk[p] * (uh[m + 1] - uh[m]) / dx;
        }
      }
    }
    free(FLs); free(FRs); free(VLs); free(VRs); free(Fx); free(uh);
  }
  (void)d;
  return err;
}

/* R17: the coefficient phi (1 - phi) of Eq. 4 is taken as 0 for fractions
 * within one unit of rounding of 0 or 1 (phi < 2^-52 or 1 - phi < 2^-52):
 * such traces, left by the hyperbolic step far from any interface, are
 * below the resolution of the fraction sum.  A cell with an active fraction
 * couples its faces. */
#define OR_TRACE 0x1p-52
static int pf_active(double a) { return a >= OR_TRACE && 1.0 - a >= OR_TRACE; }

/* R12: Phase-Field flux at one face (Eq. 5), direction dir, from the face
 * states (UL, VL) of the left cell and (UR, VR) of the right cell and the face
 * gradients G[p] of Q_p.  F is the flux vector of Eq. 1 (last line). */
void or_pf_flux(const or_grid *g, int dir, const double *UL, const double *VL, const double *UR,
                const double *VR, const double *G, double *F) {
  int N = g->N, d = g->dim, nvar = nv(g);
  double J[OR_MAXP], M[OR_MAXP];
  double sumJ = 0.0, suma = 0.0;
  for (int p = 0; p < N; p++) {
    double aL = UL[IALF(g, p)], aR = UR[IALF(g, p)];
    double mL = UL[IMASS(p)], mR = UR[IMASS(p)];
    double gp = G[p] > 0.0 ? G[p] : 0.0, gm = G[p] < 0.0 ? G[p] : 0.0;
    J[p] = gp * aR * (1.0 - aL) + gm * aL * (1.0 - aR);
    M[p] = gp * mR * (1.0 - aL) + gm * mL * (1.0 - aR);
    sumJ += J[p];
    suma += 0.5 * (aL + aR);
  }
  for (int p = 0; p < N; p++) {
    double af = 0.5 * (UL[IALF(g, p)] + UR[IALF(g, p)]);
    double mf = 0.5 * (UL[IMASS(p)] + UR[IMASS(p)]);
    J[p] = J[p] - sumJ * af / suma;
    M[p] = M[p] - sumJ * mf / suma;
  }
  for (int v = 0; v < nvar; v++) F[v] = 0.0;
  double P = 0.5 * (VL[IENE(g)] + VR[IENE(g)]);
  double uu = 0.0;
  double u[3];
  for (int j = 0; j < d; j++) {
    u[j] = 0.5 * (VL[IMOM(g, j)] + VR[IMOM(g, j)]);
    uu += u[j] * u[j];
  }
  double msum = 0.0, e = 0.0;
  for (int p = 0; p < N; p++) {
    F[IMASS(p)] = M[p];
    F[IALF(g, p)] = J[p];
    msum += M[p];
    e += J[p] * (eos_A(g, p) * P + eos_B(g, p)) + g->D[p] * M[p];
  }
  for (int j = 0; j < d; j++) F[IMOM(g, j)] = msum * u[j];
  F[IENE(g)] = msum * 0.5 * uu + e;
  (void)dir;
}

/* dU/dt of the Phase-Field step (Eq. 5) for Q [N][cells]: +sum_d dF^PF/dx_d;
 * dt_limit > 0 limits the face gradients for that time step (R17). */
int or_pf_rhs(const or_grid *g, const double *U, const double *Q, double dt_limit, double *L);

static int check_grid(const or_grid *g) {
  if (g->dim < 1 || g->dim > 3 || g->N < 1 || g->N > OR_MAXP) return OR_ERR_ARG;
  for (int a = 0; a < 3; a++) {
    if (g->n[a] < 1) return OR_ERR_ARG;
    if (a < g->dim && g->n[a] < 3) return OR_ERR_ARG;
    if (a >= g->dim && g->n[a] != 1) return OR_ERR_ARG;
  }
  return OR_OK;
}

/* dU/dt of the hyperbolic step (Eq. 3), summed over the directions. */
int or_rhs(const or_grid *g, const double *U, double *L) {
  int e = check_grid(g);
  if (e) return e;
  long tot = ncells(g) * nv(g);
  for (long k = 0; k < tot; k++) L[k] = 0.0;
  for (int dir = 0; dir < g->dim; dir++) {
    e = rhs_dir(g, dir, U, L);
    if (e) return e;
  }
  for (long k = 0; k < tot; k++)
    if (!isfinite(L[k])) return OR_ERR_NAN;
  return OR_OK;
}

int or_pf_rhs(const or_grid *g, const double *U, const double *Q, double dt_limit, double *L) {
  int e = check_grid(g);
  if (e) return e;
  int nvar = nv(g), N = g->N;
  long nc = ncells(g);
  for (long k = 0; k < nc * nvar; k++) L[k] = 0.0;
  for (int dir = 0; dir < g->dim; dir++) {
    int n = g->n[dir];
    long stride = dir == 0 ? 1 : (dir == 1 ? g->n[0] : (long)g->n[0] * g->n[1]);
    long npencil = nc / n;
    double dx = g->dx[dir];
    double *FLs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *FRs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *VLs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *VRs = (double *)malloc(sizeof(double) * nvar * (n + 2));
    double *Fx = (double *)malloc(sizeof(double) * nvar * (n + 1));
    for (long pc = 0; pc < npencil && !e; pc++) {
      long base;
      if (dir == 0) base = pc * n;
      else if (dir == 1) base = (pc / g->n[0]) * ((long)g->n[0] * n) + pc % g->n[0];
      else base = pc;
      e = pencil_faces(g, dir, U, base, stride, FLs, FRs, VLs, VRs, NULL);
      for (int m = 0; m <= n && !e; m++) {
        /* face between cells m-1 and m; Q of the two cells (boundary mapped) */
        int f1, f2;
        int jl = bc_map(m - 1, n, g->bc[2 * dir], g->bc[2 * dir + 1], &f1);
        int jr = bc_map(m, n, g->bc[2 * dir], g->bc[2 * dir + 1], &f2);
        double G[OR_MAXP];
        for (int p = 0; p < N; p++) {
          /* R17: G = 0 on a face that Eq. 4 does not couple, c_f = 0 (both
           * cells with a zero coefficient) */
          double al = U[(long)IALF(g, p) * nc + base + jl * stride];
          double ar = U[(long)IALF(g, p) * nc + base + jr * stride];
          int coupled = pf_active(al) || pf_active(ar);
          G[p] = coupled ? (Q[(long)p * nc + base + jr * stride] -
                            Q[(long)p * nc + base + jl * stride]) / dx
                         : 0.0;
          /* R17: |G| <= dx / (12 d dt), the Phase-Field step's sufficient
           * condition for bounds with R12's flux */
          if (dt_limit > 0.0) {
            double gmax = dx / (12.0 * g->dim * dt_limit);
            if (G[p] > gmax) G[p] = gmax;
            if (G[p] < -gmax) G[p] = -gmax;
          }
        }
        or_pf_flux(g, dir, FLs + m * nvar, VLs + m * nvar, FRs + (m + 1) * nvar,
                   VRs + (m + 1) * nvar, G, Fx + m * nvar);
      }
      for (int m = 0; m < n && !e; m++) {
        long cell = base + m * stride;
        for (int v = 0; v < nvar; v++)
          L[v * nc + cell] += (Fx[(m + 1) * nvar + v] - Fx[m * nvar + v]) / dx;
      }
    }
    free(FLs); free(FRs); free(VLs); free(VRs); free(Fx);
  }
  return e;
}

/* Limited face states of every interior cell along dir (for the pins):
 * UL = U^L_{i+1/2}, UR = U^R_{i-1/2}, [NV][cells]; TH = [3][cells] or NULL. */
int or_faces(const or_grid *g, int dir, const double *U, double *ULo, double *URo, double *THo) {
  int e = check_grid(g);
  if (e) return e;
  int nvar = nv(g), n = g->n[dir];
  long nc = ncells(g);
  long stride = dir == 0 ? 1 : (dir == 1 ? g->n[0] : (long)g->n[0] * g->n[1]);
  long npencil = nc / n;
  double *FLs = (double *)malloc(sizeof(double) * nvar * (n + 2));
  double *FRs = (double *)malloc(sizeof(double) * nvar * (n + 2));
  double *VLs = (double *)malloc(sizeof(double) * nvar * (n + 2));
  double *VRs = (double *)malloc(sizeof(double) * nvar * (n + 2));
  double *TH = (double *)malloc(sizeof(double) * 3 * (n + 2));
  for (long pc = 0; pc < npencil && !e; pc++) {
    long base;
    if (dir == 0) base = pc * n;
    else if (dir == 1) base = (pc / g->n[0]) * ((long)g->n[0] * n) + pc % g->n[0];
    else base = pc;
    e = pencil_faces(g, dir, U, base, stride, FLs, FRs, VLs, VRs, TH);
    for (int m = 0; m < n && !e; m++) {
      long cell = base + m * stride;
      for (int v = 0; v < nvar; v++) {
        ULo[v * nc + cell] = FLs[(m + 1) * nvar + v];
        URo[v * nc + cell] = FRs[(m + 1) * nvar + v];
      }
      if (THo)
        for (int t = 0; t < 3; t++) THo[t * nc + cell] = TH[3 * (m + 1) + t];
    }
  }
  free(FLs); free(FRs); free(VLs); free(VRs); free(TH);
  return e;
}

/* Eq. 17-21 alone on given raw primitive faces of ncell independent cells.
 * Ubar [NV][ncell] conservative averages; VLraw, VRraw [NV][ncell] primitive
 * values at x_{i+1/2} and x_{i-1/2}; outputs ULo, URo [NV][ncell] and
 * THo [3][ncell] (may be NULL). */
int or_limit(const or_grid *g, long ncell, const double *Ubar, const double *VLraw,
             const double *VRraw, double *ULo, double *URo, double *THo) {
  int nvar = nv(g);
  for (long c = 0; c < ncell; c++) {
    double Ub[OR_MAXV], VL[OR_MAXV], VR[OR_MAXV], UL[OR_MAXV], UR[OR_MAXV];
    double VfL[OR_MAXV], VfR[OR_MAXV], th[3];
    for (int v = 0; v < nvar; v++) {
      Ub[v] = Ubar[v * ncell + c];
      VL[v] = VLraw[v * ncell + c];
      VR[v] = VRraw[v * ncell + c];
    }
    int e = limit_chain(g, Ub, VL, VR, UL, UR, VfL, VfR, th);
    if (e) return e;
    for (int v = 0; v < nvar; v++) {
      ULo[v * ncell + c] = UL[v];
      URo[v * ncell + c] = UR[v];
    }
    if (THo)
      for (int t = 0; t < 3; t++) THo[t * ncell + c] = th[t];
  }
  return OR_OK;
}

int or_cons_to_prim(const or_grid *g, long ncell, const double *U, double *V) {
  int nvar = nv(g);
  for (long c = 0; c < ncell; c++) {
    double u[OR_MAXV], w[OR_MAXV];
    for (int v = 0; v < nvar; v++) u[v] = U[v * ncell + c];
    int e = cons_to_prim(g, u, w);
    if (e) return e;
    for (int v = 0; v < nvar; v++) V[v * ncell + c] = w[v];
  }
  return OR_OK;
}

int or_prim_to_cons(const or_grid *g, long ncell, const double *V, double *U) {
  int nvar = nv(g);
  for (long c = 0; c < ncell; c++) {
    double u[OR_MAXV], w[OR_MAXV];
    for (int v = 0; v < nvar; v++) w[v] = V[v * ncell + c];
    prim_to_cons(g, w, u);
    for (int v = 0; v < nvar; v++) U[v * ncell + c] = u[v];
  }
  return OR_OK;
}

int or_psi(const or_grid *g, long ncell, const double *U, double *psi) {
  int nvar = nv(g);
  for (long c = 0; c < ncell; c++) {
    double u[OR_MAXV];
    for (int v = 0; v < nvar; v++) u[v] = U[v * ncell + c];
    psi[c] = psi_energy(g, u);
  }
  return OR_OK;
}

int or_sound_speed(const or_grid *g, long ncell, const double *U, double *c) {
  int nvar = nv(g);
  for (long k = 0; k < ncell; k++) {
    double u[OR_MAXV], w[OR_MAXV];
    for (int v = 0; v < nvar; v++) u[v] = U[v * ncell + k];
    int e = cons_to_prim(g, u, w);
    if (e) return e;
    c[k] = sound_speed(g, u, w);
  }
  return OR_OK;
}

/* R10: the largest sum_d (|u_d| + c)/dx_d over the cells. */
int or_max_rate(const or_grid *g, const double *U, double *rate) {
  int nvar = nv(g);
  long nc = ncells(g);
  double best = 0.0;
  for (long k = 0; k < nc; k++) {
    double u[OR_MAXV], w[OR_MAXV];
    for (int v = 0; v < nvar; v++) u[v] = U[v * nc + k];
    int e = cons_to_prim(g, u, w);
    if (e) return e;
    double c = sound_speed(g, u, w), r = 0.0;
    for (int j = 0; j < g->dim; j++) r += (fabs(w[IMOM(g, j)]) + c) / g->dx[j];
    if (r > best) best = r;
  }
  *rate = best;
  return OR_OK;
}

/* One Runge-Kutta stage, out = a U0 + b U1 + c dt L, element by element.
 * R13: a mass or fraction of the result outside its bound (0; 1 for a
 * fraction) by no more than the rounding of this sum, 2^-48 of the sum of
 * the terms' magnitudes, is set to the bound.  A larger excursion (a time
 * step above the sufficient CFL bound of Sec. 4.2) is the scheme's own and
 * stays; the limiter of the next stage treats it (Eq. 18: theta = 0 on a
 * negative average).  A mass and a fraction of one phase have terms in the
 * ratio rho_p, so they are kept or clamped together.  R16: no bound is
 * restored without Eq. 17-20. */
static void rk_stage(const or_grid *g, double a, const double *U0, double b, const double *U1,
                     double c, double dt, const double *L, double *out) {
  OR_CAT(OR_C_RK);
  long n = ncells(g), tot = n * nv(g);
  for (long k = 0; k < tot; k++) {
    double t0 = a * U0[k], t1 = b * U1[k], t2 = c * dt * L[k];
    double x = t0 + t1 + t2;
    int v = (int)(k / n);
    int bounded = g->limiter && (v < g->N || v >= IALF(g, 0));
    if (bounded) {
      double mag = fabs(t0) + fabs(t1) + fabs(t2);
      double exc = x < 0.0 ? -x : (v >= IALF(g, 0) && x > 1.0 ? x - 1.0 : 0.0);
      if (exc > 0.0) {
        int bin = mag > 0.0 ? (int)floor(log2(exc / mag)) : 1;
        bin = bin < -64 ? -64 : (bin > 1 ? 1 : bin);
        r13_hist[bin + 64] += 1.0;
      }
      double tol = or_stage_tol * mag;
      if (x < 0.0 && -x <= tol) x = 0.0;
      if (v >= IALF(g, 0) && x > 1.0 && x - 1.0 <= tol) x = 1.0;
    }
    out[k] = x;
  }
}

/* One stage alone, for the tests of R13's stage rule. */
void or_rk_stage(const or_grid *g, double a, const double *U0, double b, const double *U1,
                 double c, double dt, const double *L, double *out) {
  rk_stage(g, a, U0, b, U1, c, dt, L, out);
}

/* One third-order SSP (TVD) Runge-Kutta step of Shu & Osher, in place.
 * dt_fixed > 0 gives the time step; otherwise dt = cfl / max rate (R10). */
int or_rk3_step(const or_grid *g, double *U, double cfl, double dt_fixed, double *dt_used) {
  int e = check_grid(g);
  if (e) return e;
  long tot = ncells(g) * nv(g);
  double dt = dt_fixed;
  if (!(dt > 0.0)) {
    double rate;
    e = or_max_rate(g, U, &rate);
    if (e) return e;
    dt = cfl / rate;
  }
  double *U0 = (double *)malloc(sizeof(double) * tot), *U1 = (double *)malloc(sizeof(double) * tot);
  double *L = (double *)malloc(sizeof(double) * tot);
  memcpy(U0, U, sizeof(double) * tot);
  e = or_rhs(g, U0, L);
  if (!e) {
    rk_stage(g, 1.0, U0, 0.0, U0, 1.0, dt, L, U1);
    e = or_rhs(g, U1, L);
  }
  if (!e) {
    rk_stage(g, 0.75, U0, 0.25, U1, 0.25, dt, L, U1);
    e = or_rhs(g, U1, L);
  }
  if (!e) rk_stage(g, 1.0 / 3.0, U0, 2.0 / 3.0, U1, 2.0 / 3.0, dt, L, U);
  free(U0); free(U1); free(L);
  if (dt_used) *dt_used = dt;
  return e;
}

#ifdef __cplusplus
}
#endif
