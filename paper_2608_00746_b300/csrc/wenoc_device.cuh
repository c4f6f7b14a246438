// wenoc_device.cuh -- device building blocks of the WENO-C operator for
// sm_103a: equation of state (Eq. 26-27), WENO5 smoothness indicators and
// candidates, the relative-smoothness weights (Eq. 15), the coupled
// reconstruction (Eq. 16), the limiter chain (Eq. 17-21) and the HLL/HLLC
// fluxes with the consistent face velocity.
//
// Precision is a template choice: T is the type of the reconstruction
// (smoothness indicators, weights, candidates) and TF the type of the flux
// components.  The limiter factors, the unity-sum normalisation, the
// primitive-to-conservative map, the pressure recovery and every
// accumulation are FP64 in all modes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace wc {

constexpr int MAXP = 8;

// Status bits set by kernels (read by wc_sync_status).
enum : unsigned { ST_INADMISSIBLE = 1u, ST_NAN = 2u };

struct Mat {
  int N;
  int hasD;                 // any D_p != 0
  double A[MAXP];           // 1/(gamma-1)
  double B[MAXP];           // gamma Pinf/(gamma-1)
  double D[MAXP];
  double pinf[MAXP];
  double Ag[MAXP];          // A gamma (mixture sound speed, Eq. 2, K = 0)
  double Cmin[MAXP];        // A Pmin + B: alpha_p rho_p e_p(Pmin_p, rho_p) per alpha_p
  double Apmin[MAXP];       // A Pmin
  int cl;                   // 1: WENO-CL (Eq. 23-25 instead of Eq. 19)
  int kapila;               // K_p of Eq. 2-3: 0 Allaire (K_p = 0), 1 Kapila (Wood speed)
  double gam[MAXP];         // gamma_p
  int cmp;                  // CMP_NONE, or a comparison scheme without Eq. 16-21
  double js_eps;            // epsilon of the WENO-JS comparison
  double psi_floor;         // a pressure from which on psi at a face is >= 0 (psi_face_floor)
};

// The lowest pressure t from which on every phase's factor of psi at a face
// (Eq. 9 with Eq. 26: alpha_p A_p (P - Pmin_p), formed as fma(A_p, P, -A_p
// Pmin_p)) is >= 0: the largest Pmin_p, raised by ulps until each of those
// fused multiply-adds is >= 0 at t (then also at every P >= t, A_p > 0).  A
// face with fractions >= 0 and P >= t has psi >= 0, whatever the rounding
// of its sum of non-negative terms.
inline double psi_face_floor(const Mat& m) {
  double t = -HUGE_VAL;
  for (int p = 0; p < m.N; p++) {
    double tp = m.Apmin[p] / m.A[p];
    for (int k = 0; k < 64; k++) {
      const double r = std::fma(m.A[p], tp, -m.Apmin[p]);
      if (r >= 0.0 && !std::signbit(r)) break;
      tp = std::nextafter(tp, HUGE_VAL);
    }
    if (!(std::fma(m.A[p], tp, -m.Apmin[p]) >= 0.0)) return HUGE_VAL;  // never taken
    if (tp > t) t = tp;
  }
  return t;
}

// Comparison schemes (Sec. 3.2, Sec. 4.1.1): every primitive variable with
// its own weights, no coupling (Eq. 16) and no limiters (Eq. 17-21); run by
// the sweep variant V = 2.
enum : int { CMP_NONE = 0, CMP_W = 1, CMP_JS = 2 };

template <int N, int D>
struct Idx {
  static constexpr int NV = 2 * N + D + 1;
  static constexpr int E = N + D;
  __host__ __device__ static constexpr int M(int p) { return p; }
  __host__ __device__ static constexpr int U(int j) { return N + j; }
  __host__ __device__ static constexpr int A(int p) { return N + D + 1 + p; }
};

// ------------------------------------------------------------------ arithmetic helpers
// Reciprocal by the Newton-Raphson iteration r <- r + r (1 - x r) (quadratic
// convergence; see Muller et al., Handbook of Floating-Point Arithmetic,
// division by Newton-Raphson iteration), started from the hardware
// approximation rcp.approx.ftz.f64; two steps reach full double precision.
// For normal, finite x only (callers check the range).
#ifndef WC_RCP_APPROX_F64
#define WC_RCP_APPROX_F64(r, x) asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x))
#define WC_RSQRT_APPROX_F64(r, x) asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x))
#endif
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  WC_RCP_APPROX_F64(r, x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float rcp_nr(float x) { return 1.0f / x; }

// 1/sqrt(x) by the Newton-Raphson iteration y <- y + y (1/2 - x y^2 / 2)
// (same reference), started from rsqrt.approx.ftz.f64.  Normal positive x.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  WC_RSQRT_APPROX_F64(y, x);
  const double h = 0.5 * x;
  double e = fma(-h * y, y, 0.5);
  y = fma(y, e, y);
  e = fma(-h * y, y, 0.5);
  return fma(y, e, y);
}
__device__ __forceinline__ float rsqrt_nr(float x) { return rsqrtf(x); }

// Bit-level tests on non-negative or signed values (integer pipe, not FP64).
__device__ __forceinline__ bool has_sign(double x) { return __double2hiint(x) < 0; }
__device__ __forceinline__ bool has_sign(float x) { return __float_as_int(x) < 0; }
__device__ __forceinline__ bool is_pos_zero(double x) { return __double_as_longlong(x) == 0; }
__device__ __forceinline__ bool is_pos_zero(float x) { return __float_as_int(x) == 0; }
// max of non-negative values: their bit patterns order like the values
__device__ __forceinline__ double max_nonneg(double a, double b) {
  long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ __forceinline__ float max_nonneg(float a, float b) {
  int ia = __float_as_int(a), ib = __float_as_int(b);
  return __int_as_float(ia > ib ? ia : ib);
}
// Comparisons decided on the bit patterns (integer pipe; the FP64 pipe is
// the sweep's bottleneck).  For doubles that are >= +0 (not NaN) the bit
// patterns order like the values; any double is <= 0 iff its pattern, read
// as a signed integer, is <= 0 (+0, -0 and the negatives).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool le0(double x) { return dbits(x) <= 0; }
__device__ __forceinline__ bool le0(float x) { return x <= 0.0f; }
__device__ __forceinline__ bool ge0(double x) {
  const long long b = dbits(x);
  return b >= 0 || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool ge0(float x) { return x >= 0.0f; }
// a < b and min(a, b) for a, b >= +0
__device__ __forceinline__ bool lt_nonneg(double a, double b) { return dbits(a) < dbits(b); }
__device__ __forceinline__ bool lt_nonneg(float a, float b) { return a < b; }
__device__ __forceinline__ double min_nonneg(double a, double b) {
  return __longlong_as_double(dbits(a) < dbits(b) ? dbits(a) : dbits(b));
}
// lo < x < hi for x of any sign, 0 < lo < hi (a NaN fails)
__device__ __forceinline__ bool in_range(double x, double lo, double hi) {
  const long long b = dbits(x);
  return b > dbits(lo) && b < dbits(hi);
}
__device__ __forceinline__ bool in_range(float x, float lo, float hi) { return x > lo && x < hi; }
// min / max of two non-NaN doubles of any sign on the integer pipe: the key
// b ^ ((b >> 63) & 0x7FF..F) orders like the values (-0 below +0)
__device__ __forceinline__ long long dkey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
// x >= t for a non-NaN t; false for a NaN x (integer pipe)
__device__ __forceinline__ bool ge_floor(double x, double t) {
  const long long k = dkey(x);
  return k >= dkey(t) && k <= 0x7FF0000000000000LL;
}
// x is +0, positive or +inf (not NaN, no sign bit; integer pipe)
__device__ __forceinline__ bool nonneg_num(double x) {
  return (unsigned long long)dbits(x) <= 0x7FF0000000000000ULL;
}
__device__ __forceinline__ double dmin(double a, double b) { return dkey(b) < dkey(a) ? b : a; }
__device__ __forceinline__ double dmax(double a, double b) { return dkey(b) > dkey(a) ? b : a; }
__device__ __forceinline__ float dmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float dmax(float a, float b) { return fmaxf(a, b); }
// x < 0, x >= 0 and x > 1 with the IEEE results for every double (-0 is not
// below zero; a NaN compares false), decided on the bit pattern
__device__ __forceinline__ bool lt0_ieee(double x) {
  const long long b = dbits(x);
  const unsigned long long mag = (unsigned long long)(b & 0x7FFFFFFFFFFFFFFFLL);
  return b < 0 && mag - 1ull < 0x7FF0000000000000ull;  // nonzero, not NaN
}
__device__ __forceinline__ bool ge0_ieee(double x) {
  const long long b = dbits(x);
  return (b >= 0 && b <= 0x7FF0000000000000LL) || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool gt1_ieee(double x) {
  const long long b = dbits(x);
  return b > 0x3FF0000000000000LL && b <= 0x7FF0000000000000LL;
}
// infinite or NaN
__device__ __forceinline__ bool not_finite(double x) {
  return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}

// ------------------------------------------------------------------ conversions
// Between binary64 and binary32 on the integer pipe (hardware conversions
// run on the FP64 pipe, the sweep's bottleneck), from the IEEE 754 formats:
// sign, 11-bit exponent biased by 1023 and 52-bit fraction against sign,
// 8-bit exponent biased by 127 and 23-bit fraction.  Values whose binary32
// image is normal, and zeros (frequent: a uniform region has zero velocity
// components and flat stencils), are converted here; subnormal results,
// infinities, NaNs and overflowing values take the hardware conversion.
//
// binary64 -> binary32, round to nearest, ties to even: keep the top 23
// fraction bits, add one when the 29 dropped bits are above half, or exactly
// half with the kept bits odd (a carry into the exponent is the correct
// result, up to infinity above the largest binary32).
// The hardware conversions for the rare values the integer paths leave to
// them, out of line: inlined, the compiler may issue them, predicated off,
// on every conversion, and each issue holds the FP64 pipe.
static __device__ __noinline__ float f64_to_f32_hw(double x) { return (float)x; }
static __device__ __noinline__ double f32_to_f64_hw(float x) { return (double)x; }

__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {  // binary32 exponent e - 896 in 1..254
    unsigned r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ? 1u : 0u;
    return __uint_as_float(r | (hi & 0x80000000u));
  }
  if (e < 873u) return __uint_as_float(hi & 0x80000000u);  // |x| < 2^-150: a signed zero
  return f64_to_f32_hw(x);
}
// binary32 -> binary64 (exact): exponent rebased by 1023 - 127 = 896, the 23
// fraction bits on top of the 52.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned b = __float_as_uint(x), em = b & 0x7fffffffu;
  if (em - 0x00800000u < 0x7f000000u)  // normal
    return __hiloint2double((int)((b & 0x80000000u) | ((em >> 3) + (896u << 20))),
                            (int)(em << 29));
  if (em == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);  // a signed zero
  return f32_to_f64_hw(x);
}
// T(x) and double(x) of the precision templates through the helpers above
template <typename T> __device__ __forceinline__ T cvt(double x);
template <> __device__ __forceinline__ double cvt<double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt<float>(double x) { return f64_to_f32(x); }
__device__ __forceinline__ double wide(double x) { return x; }
__device__ __forceinline__ double wide(float x) { return f32_to_f64(x); }

// 2^-e(m) with e(m) the binary exponent of m > 0 (m * scale in [1, 2)), or 0
// when m is outside [2^-1000, 2^1000] (caller takes a slower exact path).
__device__ __forceinline__ double exp_scale(double m) {
  int e = (__double2hiint(m) >> 20) & 0x7ff;
  if (e < 23 || e > 2023) return 0.0;
  return __hiloint2double((2046 - e) << 20, 0);
}
__device__ __forceinline__ float exp_scale(float m) {
  int e = (__float_as_int(m) >> 23) & 0xff;
  if (e < 1 || e > 253) return 0.0f;
  return __int_as_float((254 - e) << 23);
}
// b * sc for b >= 0 and sc a power of two from exp_scale: for a normal b
// whose product stays normal, the exponent field is shifted on the integer
// pipe (exact); otherwise the multiplication does it.
__device__ __forceinline__ double mul_pow2(double b, double sc) {
  const long long bb = dbits(b);
  const long long r = bb + (dbits(sc) - 0x3FF0000000000000LL);
  if (bb == 0) return 0.0;
  return ((bb >> 52) >= 1 && (r >> 52) >= 1) ? __longlong_as_double(r) : b * sc;
}
__device__ __forceinline__ float mul_pow2(float b, float sc) { return b * sc; }

// ------------------------------------------------------------------ EOS
// Mixture rules and Eq. 27.  V gets u and P; masses and fractions are copies.
template <int N, int D>
__device__ __forceinline__ void cons_to_prim(const Mat& m, const double* U, double* V) {
  using I = Idx<N, D>;
  double rho = U[0];
#pragma unroll
  for (int p = 1; p < N; p++) rho += U[p];
  double mm = 0.0;
#pragma unroll
  for (int j = 0; j < D; j++) mm = fma(U[I::U(j)], U[I::U(j)], mm);
  double sA = 0.0, sB = 0.0, sD = 0.0;
#pragma unroll
  for (int p = 0; p < N; p++) {
    sA = fma(m.A[p], U[I::A(p)], sA);
    sB = fma(m.B[p], U[I::A(p)], sB);
    if (m.hasD) sD = fma(m.D[p], U[p], sD);
  }
  // one reciprocal for 1/rho and 1/sum A alpha
  double inv, inv_sA;
  double prod = rho * sA;
  if (in_range(prod, 1e-280, 1e280)) {
    double r = rcp_nr(prod);
    inv = sA * r;
    inv_sA = rho * r;
  } else {
    inv = 1.0 / rho;
    inv_sA = 1.0 / sA;
  }
#pragma unroll
  for (int p = 0; p < N; p++) {
    V[p] = U[p];
    V[I::A(p)] = U[I::A(p)];
  }
#pragma unroll
  for (int j = 0; j < D; j++) V[I::U(j)] = U[I::U(j)] * inv;
  V[I::E] = (U[I::E] - 0.5 * mm * inv - sB - sD) * inv_sA;
}

// psi_{V->U} for one face: rho, rho u, rho E (Eq. 26).  Masses/fractions copied.
template <int N, int D>
__device__ __forceinline__ void prim_to_cons(const Mat& m, const double* V, double* U) {
  using I = Idx<N, D>;
  double rho = V[0];
#pragma unroll
  for (int p = 1; p < N; p++) rho += V[p];
  double uu = 0.0;
#pragma unroll
  for (int j = 0; j < D; j++) uu = fma(V[I::U(j)], V[I::U(j)], uu);
  double P = V[I::E];
  double e = 0.0;
#pragma unroll
  for (int p = 0; p < N; p++) {
    e = fma(V[I::A(p)], fma(m.A[p], P, m.B[p]), e);
    if (m.hasD) e = fma(m.D[p], V[p], e);
  }
#pragma unroll
  for (int p = 0; p < N; p++) {
    U[p] = V[p];
    U[I::A(p)] = V[I::A(p)];
  }
#pragma unroll
  for (int j = 0; j < D; j++) U[I::U(j)] = rho * V[I::U(j)];
  U[I::E] = fma(0.5 * rho, uu, e);
}

// psi of Eq. 9 for a state given by its primitive values: with rho E from
// Eq. 26 the kinetic and D terms cancel and psi = sum_p alpha_p A_p (P - Pmin_p).
template <int N, int D>
__device__ __forceinline__ double psi_prim(const Mat& m, const double* alpha, double P) {
  double s = 0.0;
#pragma unroll
  for (int p = 0; p < N; p++) s = fma(alpha[p], fma(m.A[p], P, -m.Apmin[p]), s);
  return s;
}

// psi of Eq. 9 from a conservative vector (used for the interior value U^C).
template <int N, int D>
__device__ __forceinline__ double psi_cons(const Mat& m, const double* U) {
  using I = Idx<N, D>;
  double rho = U[0];
#pragma unroll
  for (int p = 1; p < N; p++) rho += U[p];
  double mm = 0.0;
#pragma unroll
  for (int j = 0; j < D; j++) mm = fma(U[I::U(j)], U[I::U(j)], mm);
  double s = 0.0;
#pragma unroll
  for (int p = 0; p < N; p++) {
    s = fma(U[I::A(p)], m.Cmin[p], s);
    if (m.hasD) s = fma(m.D[p], U[p], s);
  }
  double ke = 0.0;
  if (in_range(rho, 1e-280, 1.7e308)) ke = 0.5 * mm * rcp_nr(rho);
  else if (rho > 0.0) ke = 0.5 * mm / rho;
  return U[I::E] - ke - s;
}

// ------------------------------------------------------------------ WENO5
// The stencil f_{i-2..i+2} enters as differences from the centre value,
// da = f_{i-2} - f_i, db = f_{i-1} - f_i, dd = f_{i+1} - f_i, de = f_{i+2} - f_i,
// so a constant stencil reconstructs to f_i exactly in any precision.
template <typename T>
struct Stencil {
  T c, da, db, dd, de;
};
template <typename T>
__device__ __forceinline__ Stencil<T> stencil(T a, T b, T c, T d, T e) {
  return Stencil<T>{c, a - c, b - c, d - c, e - c};
}

// Smoothness indicators of the three sub-stencils (Jiang-Shu), scaled by
// 12/13 (t1^2 + (3/13) t2^2); Eq. 15 uses only their ratios.  The mirrored
// stencil of the right face has the same three values in reverse order.
template <typename T>
__device__ __forceinline__ void smoothness(const Stencil<T>& s, T& b0, T& b1, T& b2) {
  const T c = T(3) / T(13);
  T t1 = fma(T(-2), s.db, s.da), t2 = fma(T(-4), s.db, s.da);
  b0 = fma(t1, t1, (c * t2) * t2);
  t1 = s.db + s.dd;
  t2 = s.db - s.dd;
  b1 = fma(t1, t1, (c * t2) * t2);
  t1 = fma(T(-2), s.dd, s.de);
  t2 = fma(T(-4), s.dd, s.de);
  b2 = fma(t1, t1, (c * t2) * t2);
}

template <typename T> __device__ __forceinline__ T tiny_norm();
template <> __device__ __forceinline__ double tiny_norm<double>() { return 1e-140; }
template <> __device__ __forceinline__ float tiny_norm<float>() { return 1e-17f; }

// Weights of both faces of a cell in unnormalised form: omega^L_s =
// aL[s] invL, omega^R_s = aR[s] invR (invL, invR also carry the 1/6 of the
// candidates).
template <typename T>
struct W6 {
  T aL0, aL1, aL2, aR0, aR1, aR2, invL, invR;
};

// Eq. 15 for both faces from the shared indicators (b0, b1, b2) of the
// sub-stencils {i-2..i}, {i-1..i+1}, {i..i+2}; ideal weights (0.1, 0.6, 0.3)
// left to right for the left face and mirrored for the right face.
//  * all indicators positive: Eq. 15 divided through by IS_s^2 is
//    omega_s = (d_s prod_{k!=s} IS_k^2) / sum_t (d_t prod_{k!=t} IS_k^2).  The
//    indicators are scaled by a power of two (exact) so their maximum is in
//    [1, 2); the products IS_j^2 IS_k^2 are shared by both faces, and one
//    reciprocal of sumL sumR serves both normalisations.  A single zero
//    indicator is covered too (its stencil gets all the weight);
//  * two or three zero indicators: the zero stencils share the weight in
//    proportion to d (every other ratio is infinite, omega = 0);
//  * products beyond the range of T: the ratio form of Eq. 15 itself.
template <typename T>
__device__ __forceinline__ W6<T> weights_of(const Stencil<T>& st) {
  T b0, b1, b2;
  smoothness(st, b0, b1, b2);
  const T d0 = T(0.1), d1 = T(0.6), d2 = T(0.3);
  const T sixth = T(1) / T(6);
  W6<T> w;
  T mx = max_nonneg(b0, max_nonneg(b1, b2));
  T sc = exp_scale(mx);
  if (!is_pos_zero(sc)) {
    T x0 = mul_pow2(b0, sc), x1 = mul_pow2(b1, sc), x2 = mul_pow2(b2, sc);
    T s0 = x0 * x0, s1 = x1 * x1, s2 = x2 * x2;
    T p12 = s1 * s2, p02 = s0 * s2, p01 = s0 * s1;
    w.aL0 = d0 * p12;
    w.aL1 = d1 * p02;
    w.aL2 = d2 * p01;
    w.aR0 = d0 * p01;
    w.aR1 = d1 * p02;
    w.aR2 = d2 * p12;
    T sumL = w.aL0 + w.aL1 + w.aL2;
    T sumR = w.aR0 + w.aR1 + w.aR2;
    if (!lt_nonneg(sumL, tiny_norm<T>()) && !lt_nonneg(sumR, tiny_norm<T>())) {
      T r = rcp_nr(sumL * sumR) * sixth;
      w.invL = sumR * r;
      w.invR = sumL * r;
      return w;
    }
  }
  const bool z0 = is_pos_zero(b0), z1 = is_pos_zero(b1), z2 = is_pos_zero(b2);
  if (int(z0) + int(z1) + int(z2) >= 2 || is_pos_zero(mx)) {
    // Eq. 15 zero cases; ideal weights of the zero stencils, renormalised
    w.aL0 = z0 ? d0 : T(0);
    w.aL1 = z1 ? d1 : T(0);
    w.aL2 = z2 ? d2 : T(0);
    w.aR0 = z2 ? d0 : T(0);
    w.aR1 = z1 ? d1 : T(0);
    w.aR2 = z0 ? d2 : T(0);
    w.invL = sixth / (w.aL0 + w.aL1 + w.aL2);
    w.invR = sixth / (w.aR0 + w.aR1 + w.aR2);
    return w;
  }
  // Eq. 15 in ratio form (extreme ratios, single zeros far out of range)
  auto ratio_w = [](T bA, T bB, T bC, T dA, T dB, T dC) {
    T den = dA;
    bool inf = false;
    if (is_pos_zero(bA) && is_pos_zero(bB)) den += dB;
    else if (is_pos_zero(bB)) inf = true;
    else { T r = bA / bB; den += dB * r * r; }
    if (is_pos_zero(bA) && is_pos_zero(bC)) den += dC;
    else if (is_pos_zero(bC)) inf = true;
    else { T r = bA / bC; den += dC * r * r; }
    return inf ? T(0) : dA / den;
  };
  w.aL0 = ratio_w(b0, b1, b2, d0, d1, d2);
  w.aL1 = ratio_w(b1, b0, b2, d1, d0, d2);
  w.aL2 = ratio_w(b2, b0, b1, d2, d0, d1);
  w.aR0 = ratio_w(b2, b1, b0, d0, d1, d2);
  w.aR1 = ratio_w(b1, b2, b0, d1, d0, d2);
  w.aR2 = ratio_w(b0, b2, b1, d2, d0, d1);
  w.invL = sixth;
  w.invR = sixth;
  return w;
}

// Comparison weights (Sec. 3.2, the fifth-order form of Eq. 12): omega_s
// proportional to d_s / (IS_s + eps)^2 with the Jiang-Shu indicators IS_s =
// (13/12) b_s.  Each term is taken relative to the smallest IS_k + eps, so it
// lies in (0, d_s] whatever the scale of f (the normalised weights are the
// same).
template <typename T>
__device__ __forceinline__ W6<T> weights_js(const Stencil<T>& st, T eps) {
  T b0, b1, b2;
  smoothness(st, b0, b1, b2);
  const T k = T(13) / T(12);
  const T e0 = fma(k, b0, eps), e1 = fma(k, b1, eps), e2 = fma(k, b2, eps);
  const T mn = fmin(e0, fmin(e1, e2));
  const T r0 = mn / e0, r1 = mn / e1, r2 = mn / e2;
  const T q0 = r0 * r0, q1 = r1 * r1, q2 = r2 * r2;
  const T sixth = T(1) / T(6);
  W6<T> w;
  w.aL0 = T(0.1) * q0;
  w.aL1 = T(0.6) * q1;
  w.aL2 = T(0.3) * q2;
  w.aR0 = T(0.1) * q2;
  w.aR1 = T(0.6) * q1;
  w.aR2 = T(0.3) * q0;
  w.invL = sixth / (w.aL0 + w.aL1 + w.aL2);
  w.invR = sixth / (w.aR0 + w.aR1 + w.aR2);
  return w;
}

// The weights of a sweep variant: Eq. 15, or for the comparison variant
// (V = 2) the configured comparison scheme's.
template <int V, typename T>
__device__ __forceinline__ W6<T> sweep_weights(const Mat& m, const Stencil<T>& st) {
  if constexpr (V == 2) {
    if (m.cmp == CMP_JS) return weights_js<T>(st, T(m.js_eps));
  }
  return weights_of<T>(st);
}

// Eq. 10 at x_{i+1/2} (fL) and x_{i-1/2} (fR): the candidates' values minus
// f_i, times 6, are 2da-7db, 2dd-db, 5dd-de (left face) and the mirror images.
// The operations are written as explicit fused multiply-adds, so every
// inlined copy rounds identically whatever the compiler shares between them.
template <typename T>
__device__ __forceinline__ void reconstruct(const W6<T>& w, const Stencil<T>& s, T& fL, T& fR) {
  const T qL0 = fma(T(2), s.da, T(-7) * s.db), qL1 = fma(T(2), s.dd, -s.db),
          qL2 = fma(T(5), s.dd, -s.de);
  const T qR0 = fma(T(2), s.de, T(-7) * s.dd), qR1 = fma(T(2), s.db, -s.dd),
          qR2 = fma(T(5), s.db, -s.da);
  fL = fma(fma(w.aL2, qL2, fma(w.aL1, qL1, w.aL0 * qL0)), w.invL, s.c);
  fR = fma(fma(w.aR2, qR2, fma(w.aR1, qR1, w.aR0 * qR0)), w.invR, s.c);
}

// Mass and fraction faces of the reduced-precision path: the weighted
// candidate offsets (Eq. 10 minus the cell value) in T, added to the cell
// value in FP64, so a flat stencil reconstructs to the FP64 cell value
// exactly (a constant fraction stays constant) and the FP32 rounding is
// relative to the stencil's variation, not to the values.  (Velocity and
// pressure keep the value form: FP64 noise of a uniform field below the FP32
// resolution then gives exactly uniform faces, which equilibrium needs.)
template <typename T>
__device__ __forceinline__ void offsets(const W6<T>& w, const Stencil<T>& s, T& oL, T& oR) {
  const T qL0 = fma(T(2), s.da, T(-7) * s.db), qL1 = fma(T(2), s.dd, -s.db),
          qL2 = fma(T(5), s.dd, -s.de);
  const T qR0 = fma(T(2), s.de, T(-7) * s.dd), qR1 = fma(T(2), s.db, -s.dd),
          qR2 = fma(T(5), s.db, -s.da);
  oL = fma(w.aL2, qL2, fma(w.aL1, qL1, w.aL0 * qL0)) * w.invL;
  oR = fma(w.aR2, qR2, fma(w.aR1, qR1, w.aR0 * qR0)) * w.invR;
}
template <typename T>
__device__ __forceinline__ void reconstruct_offset(const W6<T>& w, const Stencil<T>& s,
                                                   double cd, double& fL, double& fR) {
  T oL, oR;
  offsets(w, s, oL, oR);
  fL = cd + wide(oL);
  fR = cd + wide(oR);
}

// ------------------------------------------------------------------ limiters
// Eq. 18 (f_min = 0) with f^C from Eq. 6 inverted (N_quad = 4, w = 1/12):
// theta = 1 when min(f^C, f^L, f^R) >= 0, else fbar / (fbar - min), clamped
// to [0, 1].
__device__ __forceinline__ double theta_pos(double fb, double fL, double fR) {
  double fC = (fb - (fL + fR) * (1.0 / 12.0)) * 1.2;
  // common case decided on the sign bits (a -0.0 takes the exact path below,
  // which returns 1 as well)
  if (!(has_sign(fC) | has_sign(fL) | has_sign(fR))) return 1.0;
  const double m = dmin(fC, dmin(fL, fR));
  if (ge0(m)) return 1.0;
  if (le0(fb)) return 0.0;
  const double den = fb - m;
  const double t = in_range(den, 1e-300, 1e300) ? fb * rcp_nr(den) : fb / den;
  return min_nonneg(t, 1.0);
}

__device__ __forceinline__ double theta_lower(double fb, double fC, double fL, double fR) {
  if (!(has_sign(fC) | has_sign(fL) | has_sign(fR))) return 1.0;
  double m = fmin(fC, fmin(fL, fR));
  if (m >= 0.0) return 1.0;
  if (fb <= 0.0) return 0.0;
  return fmin(fb / (fb - m), 1.0);
}

// A face state handed to the Riemann solver: conservative U and the primitive
// velocity and pressure of the same state.
template <int N, int D>
struct Face {
  double U[Idx<N, D>::NV];
  double u[D];
  double P;
};

// The limiter chain for one cell: Ub cell average (FP64, conservative), Pb
// its pressure; mL/aL (mR/aR) reconstructed masses and fractions at
// x_{i+1/2} (x_{i-1/2}); uL, PL (uR, PR) reconstructed velocity and pressure.
// Produces the two limited face states.  th (optional) receives
// (min_p theta_p of Eq. 17, theta_i of Eq. 20, theta^(psi) of Eq. 21).
// Rounding residue below a bound: with fbar >= 0 the limited face values
// fbar + theta (f - fbar) of Eq. 18, Eq. 20, Eq. 21 and Eq. 25 are
// non-negative in exact arithmetic, but a value that should land on zero can
// land an ulp below it; it becomes 0.  With fbar < 0 (a stage that left the
// bound, theta = 0) the value is fbar itself and stays.  A NaN stays a NaN.
__device__ __forceinline__ double nonneg(double x, double fb) {
  return lt0_ieee(x) && ge0_ieee(fb) ? 0.0 : x;
}

// The same rule at the end of a Runge-Kutta stage x = t0 + t1 + t2: a mass
// or fraction outside its bound (0; 1 for a fraction) by at most 2^-48 of
// |t0| + |t1| + |t2| is rounding of the stage sum and becomes the bound; a
// larger excursion (a time step above the sufficient CFL bound) stays for
// the next limiter.  A phase's mass and fraction have terms in the ratio
// rho_p, so they are kept or clamped together.
constexpr double STAGE_TOL = 0x1p-48;
__device__ __forceinline__ double stage_bound(double x, double t0, double t1, double t2,
                                              bool frac) {
  const bool lo = lt0_ieee(x), hi = frac && gt1_ieee(x);
  if (lo || hi) {
    const double tol = STAGE_TOL * (fabs(t0) + fabs(t1) + fabs(t2));
    if (lo && -x <= tol) return 0.0;
    if (hi && x - 1.0 <= tol) return 1.0;
  }
  return x;
}

// One Runge-Kutta stage value x = r0 u0 + r1 u1 + r2dt L (r2dt = r2 dt) as two
// fused multiply-adds: three FP64 operations where the terms rounded one by
// one take five, with a rounding error of at most three units of 2^-53 of
// |r0 u0| + |r1 u1| + |r2dt L|, far inside the stage rule's 2^-48.  For a
// bounded variable (mass or fraction) the terms of that rule are formed only
// when x has left its bound.
__device__ __forceinline__ double rk_combine(double r0, double u0, double r1, double u1,
                                             double r2dt, double L, bool bounded, bool frac) {
  double x = fma(r2dt, L, fma(r1, u1, r0 * u0));
  if (bounded && (lt0_ieee(x) || (frac && gt1_ieee(x))))
    x = stage_bound(x, r0 * u0, r1 * u1, r2dt * L, frac);
  return x;
}

// Eq. 23-25 (WENO-CL) on one face: S_p = alpha_p,face - alpha_p,bar (the
// factor 2/dx of Eq. 24 cancels), p-hat the first phase of largest |S_p|,
// S-hat = S_phat - sum_p S_p, theta_phat = clamp(S-hat / S_phat),
// theta_p = clamp(S_phat / S-hat) for the others (x/0 = +-infinity before
// the clamp), masses and fractions moved to fbar + theta (f - fbar).
// Returns whether a face value moved.
template <int N, int D>
__device__ __forceinline__ bool consistent_face(const double* Ub, double* mf, double* af) {
  using I = Idx<N, D>;
  double S[N], sum = 0.0, Sph = 0.0;
  long long best = -1;
#pragma unroll
  for (int p = 0; p < N; p++) {
    S[p] = af[p] - Ub[I::A(p)];
    sum += S[p];
    const long long b = dbits(S[p]) & 0x7FFFFFFFFFFFFFFFLL;
    if (b > best) {
      best = b;
      Sph = S[p];
    }
  }
  if (best == 0) return false;  // every gradient is zero
  const double Shat = Sph - sum;
  const double a1 = fabs(Sph), a2 = fabs(Shat);
  const double th_ph = in_range(a1, 1e-300, 1e300) ? Shat * rcp_nr(Sph) : Shat / Sph;
  double th_o;
  if (dbits(a2) == 0) th_o = has_sign(Sph) ? 0.0 : 1.0;
  else th_o = in_range(a2, 1e-300, 1e300) ? Sph * rcp_nr(Shat) : Sph / Shat;
  const double tph = th_ph < 0.0 ? 0.0 : (th_ph > 1.0 ? 1.0 : th_ph);
  const double to = th_o < 0.0 ? 0.0 : (th_o > 1.0 ? 1.0 : th_o);
  bool moved = false, seen = false;
#pragma unroll
  for (int p = 0; p < N; p++) {
    // p-hat is the first phase whose |S| is the largest
    const bool is_ph = !seen && (dbits(S[p]) & 0x7FFFFFFFFFFFFFFFLL) == best;
    seen = seen || is_ph;
    const double th = is_ph ? tph : to;
    if (lt_nonneg(th, 1.0)) {
      const double mb = Ub[p], ab = Ub[I::A(p)];
      mf[p] = nonneg(fma(th, mf[p] - mb, mb), mb);
      af[p] = nonneg(fma(th, af[p] - ab, ab), ab);
      moved = true;
    }
  }
  return moved;
}

template <int N, int D, bool LIMIT = true>
__device__ __forceinline__ void limit_chain(const Mat& m, const double* Ub, double Pb,
                                            double* mL, double* aL, double* mR, double* aR,
                                            const double* uL, double PL, const double* uR,
                                            double PR, int energy_limiter, Face<N, D>& FL,
                                            Face<N, D>& FR, double* th) {
  using I = Idx<N, D>;
  double th17 = 1.0, thi = 1.0;
  // (LIMIT = false, the comparison schemes: raw faces to the Riemann solver)
  if constexpr (LIMIT) {
  // Eq. 17-18: common theta_p for (alpha rho)_p and alpha_p
#pragma unroll
  for (int p = 0; p < N; p++) {
    double mb = Ub[p], ab = Ub[I::A(p)];
    double tp = min_nonneg(theta_pos(mb, mL[p], mR[p]), theta_pos(ab, aL[p], aR[p]));
    if (lt_nonneg(tp, 1.0)) {
      mL[p] = nonneg(fma(tp, mL[p] - mb, mb), mb);
      mR[p] = nonneg(fma(tp, mR[p] - mb, mb), mb);
      aL[p] = nonneg(fma(tp, aL[p] - ab, ab), ab);
      aR[p] = nonneg(fma(tp, aR[p] - ab, ab), ab);
      th17 = min_nonneg(th17, tp);
    }
  }
  bool cl_moved = false;
  double SL = 1.0, SR = 1.0;
  if (m.cl) {
    // Eq. 23-25 (WENO-CL) instead of Eq. 19
    cl_moved = consistent_face<N, D>(Ub, mL, aL);
    cl_moved = consistent_face<N, D>(Ub, mR, aR) || cl_moved;
  } else {
  // Eq. 19: unity sum on each face
  SL = aL[0];
  SR = aR[0];
#pragma unroll
  for (int p = 1; p < N; p++) {
    SL += aL[p];
    SR += aR[p];
  }
  // (the face fractions are >= 0 here: raw faces with theta = 1, or clamped)
  if (dbits(SL) <= 0 || dbits(SR) <= 0) {
    // every fraction of a face limited to zero: first order for the cell
#pragma unroll
    for (int p = 0; p < N; p++) {
      mL[p] = mR[p] = Ub[p];
      aL[p] = aR[p] = Ub[I::A(p)];
    }
    th17 = 0.0;
  } else {
    if (dbits(SL) != dbits(1.0)) {
      double r = in_range(SL, 1e-300, 1e300) ? rcp_nr(SL) : 1.0 / SL;
#pragma unroll
      for (int p = 0; p < N; p++) {
        mL[p] *= r;
        aL[p] *= r;
      }
    }
    if (dbits(SR) != dbits(1.0)) {
      double r = in_range(SR, 1e-300, 1e300) ? rcp_nr(SR) : 1.0 / SR;
#pragma unroll
      for (int p = 0; p < N; p++) {
        mR[p] *= r;
        aR[p] *= r;
      }
    }
  }
  }
  // Eq. 20: theta_i = min_p theta_p recomputed on the normalised faces (when
  // Eq. 17 and Eq. 19 left every face value unchanged, the recomputed thetas
  // are those of Eq. 17, all one)
  if (lt_nonneg(th17, 1.0) || cl_moved || dbits(SL) != dbits(1.0) ||
      dbits(SR) != dbits(1.0)) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      double tp =
          min_nonneg(theta_pos(Ub[p], mL[p], mR[p]), theta_pos(Ub[I::A(p)], aL[p], aR[p]));
      thi = min_nonneg(thi, tp);
    }
  }
  if (lt_nonneg(thi, 1.0)) {
#pragma unroll
    for (int p = 0; p < N; p++) {
      double mb = Ub[p], ab = Ub[I::A(p)];
      mL[p] = nonneg(fma(thi, mL[p] - mb, mb), mb);
      mR[p] = nonneg(fma(thi, mR[p] - mb, mb), mb);
      aL[p] = nonneg(fma(thi, aL[p] - ab, ab), ab);
      aR[p] = nonneg(fma(thi, aR[p] - ab, ab), ab);
    }
  }
  }
  // V -> U at both faces
  double VL[I::NV], VR[I::NV];
#pragma unroll
  for (int p = 0; p < N; p++) {
    VL[p] = mL[p];
    VR[p] = mR[p];
    VL[I::A(p)] = aL[p];
    VR[I::A(p)] = aR[p];
  }
#pragma unroll
  for (int j = 0; j < D; j++) {
    VL[I::U(j)] = uL[j];
    VR[I::U(j)] = uR[j];
  }
  VL[I::E] = PL;
  VR[I::E] = PR;
  prim_to_cons<N, D>(m, VL, FL.U);
  prim_to_cons<N, D>(m, VR, FR.U);
#pragma unroll
  for (int j = 0; j < D; j++) {
    FL.u[j] = uL[j];
    FR.u[j] = uR[j];
  }
  FL.P = PL;
  FR.P = PR;
  double thpsi = 1.0;
  if (energy_limiter) {
    // Eq. 21: theta^(psi) from psi at the average, both faces and U^C
    double UC[I::NV];
#pragma unroll
    for (int v = 0; v < I::NV; v++) UC[v] = (Ub[v] - (FL.U[v] + FR.U[v]) * (1.0 / 12.0)) * 1.2;
    const double pC = psi_cons<N, D>(m, UC);
    // psi at both faces is >= 0 without evaluating it when their fractions
    // are >= 0 and their pressures at least m.psi_floor: then psi(U^C) alone
    // decides theta_lower's common case, and psi at the average is not needed
    bool faces_ok = ge_floor(PL, m.psi_floor) && ge_floor(PR, m.psi_floor);
#pragma unroll
    for (int p = 0; p < N; p++) faces_ok = faces_ok && nonneg_num(aL[p]) && nonneg_num(aR[p]);
    if (faces_ok && !has_sign(pC)) {
      thpsi = 1.0;
    } else {
      const double pb = psi_prim<N, D>(m, Ub + I::A(0), Pb);
      const double pL = psi_prim<N, D>(m, aL, PL);
      const double pR = psi_prim<N, D>(m, aR, PR);
      thpsi = theta_lower(pb, pC, pL, pR);
    }
    if (lt_nonneg(thpsi, 1.0)) {
#pragma unroll
      for (int v = 0; v < I::NV; v++) {
        FL.U[v] = fma(thpsi, FL.U[v] - Ub[v], Ub[v]);
        FR.U[v] = fma(thpsi, FR.U[v] - Ub[v], Ub[v]);
        if (v < N || v >= I::A(0)) {
          FL.U[v] = nonneg(FL.U[v], Ub[v]);
          FR.U[v] = nonneg(FR.U[v], Ub[v]);
        }
      }
      double W[I::NV];
      cons_to_prim<N, D>(m, FL.U, W);
#pragma unroll
      for (int j = 0; j < D; j++) FL.u[j] = W[I::U(j)];
      FL.P = W[I::E];
      cons_to_prim<N, D>(m, FR.U, W);
#pragma unroll
      for (int j = 0; j < D; j++) FR.u[j] = W[I::U(j)];
      FR.P = W[I::E];
    }
  }
  if (th) {
    th[0] = th17;
    th[1] = thi;
    th[2] = thpsi;
  }
}

// 1 / (rho_p c_p^2) = 1 / (gamma_p (P + Pinf_p)) of the stiffened gas
template <typename TF>
__device__ __forceinline__ TF inv_rhoc2_phase(const Mat& m, int p, TF P) {
  const TF x = cvt<TF>(m.gam[p]) * (P + cvt<TF>(m.pinf[p]));
  if constexpr (sizeof(TF) == 8) {
    return in_range(x, 1e-300, 1e300) ? rcp_nr(x) : 1.0 / x;
  } else {
    return TF(1) / x;
  }
}

// Source factors alpha_p (1 + K_p) of Eq. 3 at a cell average (alpha from the
// conservative state U, pressure P): alpha_p for K_p = 0; for the Kapila
// model alpha_p rho c^2 / (rho_p c_p^2) with Wood's rho c^2 over the fractions
// as they are (unlike the sound speed, no clip: sum_p alpha_p (1 + K_p) = 1
// keeps the fraction sum at one).
template <int N, int D>
__device__ __forceinline__ void source_factors(const Mat& m, const double* U, double P,
                                               double* f) {
  using I = Idx<N, D>;
  if (!m.kapila) {
#pragma unroll
    for (int p = 0; p < N; p++) f[p] = U[I::A(p)];
    return;
  }
  double r[N], sw = 0.0;
#pragma unroll
  for (int p = 0; p < N; p++) {
    r[p] = inv_rhoc2_phase<double>(m, p, P);
    sw = fma(U[I::A(p)], r[p], sw);
  }
  const double rhoc2 = in_range(sw, 1e-300, 1e300) ? rcp_nr(sw) : 1.0 / sw;
#pragma unroll
  for (int p = 0; p < N; p++) f[p] = U[I::A(p)] * (r[p] * rhoc2);
}

// ------------------------------------------------------------------ fluxes
// Mixture sound speed of Eq. 2 with K_p = 0: rho c^2 = sum A g alpha (P+Pinf)
// / sum A alpha.
template <int N, int D, typename TF>
__device__ __forceinline__ TF sound_speed(const Mat& m, const double* U, TF rho, TF P) {
  using I = Idx<N, D>;
  if (m.kapila) {
    // Kapila model: K_p = rho c^2 / (rho_p c_p^2) - 1 with sum alpha_p K_p = 0
    // gives Wood's 1 / (rho c^2) = sum_p alpha_p / (rho_p c_p^2).  A fraction
    // below zero enters as zero: at a low-pressure face a gas fraction of
    // -4e-4 beside water turns the unclipped sum negative (no real speed)
    TF sw = TF(0);
#pragma unroll
    for (int p = 0; p < N; p++)
      sw = sw + dmax(cvt<TF>(U[I::A(p)]), TF(0)) * inv_rhoc2_phase<TF>(m, p, P);
    const TF xw = rho * sw;
    if (in_range(xw, TF(1e-30), TF(1e30))) return rsqrt_nr(xw);
    return TF(1) / sqrt(xw);
  }
  TF num = TF(0), den = TF(0);
#pragma unroll
  for (int p = 0; p < N; p++) {
    TF a = cvt<TF>(U[I::A(p)]);
    num = num + cvt<TF>(m.Ag[p]) * a * (P + cvt<TF>(m.pinf[p]));
    den = den + cvt<TF>(m.A[p]) * a;
  }
  // c = sqrt(num / (den rho)) = num / sqrt(num den rho)
  TF x = num * den * rho;
  if (in_range(x, TF(1e-30), TF(1e30))) return num * rsqrt_nr(x);
  return sqrt(num / (den * rho));
}

// HLL in FP64 from the physical fluxes of Eq. 1 at the two face states:
// F = F_L + k ((F_L - F_R) + s_R (U_R - U_L)), k = s_L/(s_R - s_L), for every
// component, and u_hat with alpha = 1 on both sides.  In FP64 the physical
// fluxes keep u and P uniform across an isolated interface to the round-off
// of rho E, as the remainder form below does in reduced precision, with
// about 45 fewer FP64 operations a face.
template <int N, int D>
__device__ __forceinline__ void hll_fp64(const Mat& m, int dir, const Face<N, D>& L,
                                         const Face<N, D>& R, double* F, double& uhat) {
  using I = Idx<N, D>;
  double rL = L.U[0], rR = R.U[0];
#pragma unroll
  for (int p = 1; p < N; p++) {
    rL += L.U[p];
    rR += R.U[p];
  }
  double uL = L.u[0], uR = R.u[0];
#pragma unroll
  for (int j = 1; j < D; j++)
    if (j == dir) {
      uL = L.u[j];
      uR = R.u[j];
    }
  const double cL = sound_speed<N, D, double>(m, L.U, rL, L.P);
  const double cR = sound_speed<N, D, double>(m, R.U, rR, R.P);
  const double sL = dmin(uL - cL, uR - cR);
  const double sR = dmax(uL + cL, uR + cR);
  double k;
  if (ge0(sL)) k = 0.0;
  else if (le0(sR)) k = -1.0;  // F_R, with s_R taken as 0
  else k = sL * rcp_nr(sR - sL);
  const double sRu = le0(sR) ? 0.0 : sR;
  // F_L + k ((F_L - F_R) + s_R (U_R - U_L)) for a component whose physical
  // flux is u x is a x_L + b x_R with a = u_L + k (u_L - s_R) and b =
  // k (s_R - u_R) (a + b = u_hat, the flux of alpha = 1); the pressure
  // terms add (1 + k) P_L - k P_R to the normal momentum and (1 + k) u_L P_L
  // - k u_R P_R to the energy
  const double a = fma(k, uL - sRu, uL), b = k * (sRu - uR);
  uhat = a + b;
#pragma unroll
  for (int p = 0; p < N; p++) {
    F[I::A(p)] = fma(a, L.U[I::A(p)], b * R.U[I::A(p)]);
    F[p] = fma(a, L.U[p], b * R.U[p]);
  }
  const double kp = 1.0 + k;
  const double pw = fma(kp, L.P, -k * R.P);
#pragma unroll
  for (int j = 0; j < D; j++) {
    const double f = fma(a, L.U[I::U(j)], b * R.U[I::U(j)]);
    F[I::U(j)] = j == dir ? f + pw : f;
  }
  F[I::E] = fma(a, L.U[I::E], fma(b, R.U[I::E], fma(kp * uL, L.P, -k * (uR * R.P))));
}

// HLL or HLLC flux across the face between the left state L (from cell i) and
// the right state R (from cell i+1), direction dir, and u_hat, the flux of a
// volume fraction equal to one on both sides (Sec. 2.2.1).  HLL in FP64 is
// hll_fp64; the rest is written as follows.
//
// Both solvers are linear in (U, F) component by component for given wave
// speeds.  The flux is assembled from that linearity so that it keeps
// equilibrium and consistency in any precision TF:
//  * fraction and mass fluxes and u_hat are FP64 (their sums over the phases
//    match u_hat and the density flux to FP64 rounding);
//  * with ub = (u_L + u_R)/2 and Pb = (P_L + P_R)/2, rho u_j = ub_j rho +
//    rho (u_j - ub_j) and E_r = rho E - sum B alpha - sum D (alpha rho)
//    = Pb sum A alpha + |ub|^2 rho / 2 + Et, so
//      F^{rho u_j} = ub_j F^rho + F[rho (u_j - ub_j)] + delta_jn F[P],
//      F^{rho E}   = sum_p (B_p + Pb A_p) F^{alpha_p} + sum_p D_p F^{(alpha rho)_p}
//                    + |ub|^2 F^rho / 2 + Pb u_hat + F[Et],
//    where F[Et] is the flux of Et with the work term u (P - Pb) (the work
//    u Pb has no state part, so its flux is Pb u_hat in both solvers);
//    the bracketed remainders vanish exactly for uniform u and P, so an
//    isolated interface keeps u and P uniform whatever TF is, and pressure
//    differences far below the TF resolution of P are still damped;
//  * wave speeds, the HLLC contact speed and the remainders are in TF.
// HLL is written as F_L + k ((F_L - F_R) + s_R (U_R - U_L)), k = s_L/(s_R - s_L),
// which returns F_L exactly for equal states.
template <int N, int D, typename TF>
__device__ __forceinline__ void riemann(const Mat& m, int dir, int hllc, const Face<N, D>& L,
                                        const Face<N, D>& R, double* F, double& uhat) {
  using I = Idx<N, D>;
  if constexpr (sizeof(TF) == 8) {
    if (!hllc) {
      hll_fp64<N, D>(m, dir, L, R, F, uhat);
      return;
    }
  }
  double rLd = L.U[0], rRd = R.U[0];
#pragma unroll
  for (int p = 1; p < N; p++) {
    rLd += L.U[p];
    rRd += R.U[p];
  }
  double uLd = L.u[0], uRd = R.u[0];
#pragma unroll
  for (int j = 1; j < D; j++)
    if (j == dir) {
      uLd = L.u[j];
      uRd = R.u[j];
    }
  double ub[D];
#pragma unroll
  for (int j = 0; j < D; j++) ub[j] = 0.5 * (L.u[j] + R.u[j]);
  const double dPd = L.P - R.P;  // exact when P_L, P_R are close
  const TF rL = cvt<TF>(rLd), rR = cvt<TF>(rRd), uL = cvt<TF>(uLd), uR = cvt<TF>(uRd);
  const TF PL = cvt<TF>(L.P), PR = cvt<TF>(R.P);
  const TF cL = sound_speed<N, D, TF>(m, L.U, rL, PL);
  const TF cR = sound_speed<N, D, TF>(m, R.U, rR, PR);
  const TF sL = dmin(uL - cL, uR - cR);
  const TF sR = dmax(uL + cL, uR + cR);
  // remainder energy Et_K = sum A alpha_K (P_K - Pb) + rho_K (|u_K|^2 - |ub|^2)/2
  TF AaL = TF(0), AaR = TF(0);
#pragma unroll
  for (int p = 0; p < N; p++) {
    AaL += cvt<TF>(m.A[p]) * cvt<TF>(L.U[I::A(p)]);
    AaR += cvt<TF>(m.A[p]) * cvt<TF>(R.U[I::A(p)]);
  }
  TF wL[D], wR[D];
  TF kinL = TF(0), kinR = TF(0);
#pragma unroll
  for (int j = 0; j < D; j++) {
    wL[j] = cvt<TF>(L.u[j] - ub[j]);
    wR[j] = cvt<TF>(R.u[j] - ub[j]);
    kinL += wL[j] * cvt<TF>(L.u[j] + ub[j]);
    kinR += wR[j] * cvt<TF>(R.u[j] + ub[j]);
  }
  const TF halfdP = cvt<TF>(0.5 * dPd);
  const TF EtL = halfdP * AaL + TF(0.5) * rL * kinL;
  const TF EtR = -halfdP * AaR + TF(0.5) * rR * kinR;

  double Frho = 0.0;
  if (!hllc) {
    // ---------------- HLL
    double kd, sRd;
    TF k;
    if (ge0(sL)) {
      k = TF(0);
    } else if (le0(sR)) {
      k = TF(-1);  // F_L + (-1)((F_L - F_R) + s_R (U_R - U_L)) with s_R = 0
    } else {
      k = sL * rcp_nr(sR - sL);
    }
    const TF sRu = le0(sR) ? TF(0) : sR;
    kd = wide(k);
    sRd = wide(sRu);
    // masses and fractions as a x_L + b x_R (see hll_fp64); a + b = u_hat
    const double ad = fma(kd, uLd - sRd, uLd), bd = kd * (sRd - uRd);
    uhat = ad + bd;
#pragma unroll
    for (int p = 0; p < N; p++) {
      F[I::A(p)] = fma(ad, L.U[I::A(p)], bd * R.U[I::A(p)]);
      const double fm = fma(ad, L.U[p], bd * R.U[p]);
      F[p] = fm;
      Frho += fm;
    }
    // momentum remainders and pressure part
#pragma unroll
    for (int j = 0; j < D; j++) {
      TF qL = rL * wL[j], qR = rR * wR[j];
      TF fl = qL * uL, fr = qR * uR;
      TF fw = fl + k * ((fl - fr) + sRu * (qR - qL));
      double f = ub[j] * Frho + wide(fw);
      if (j == dir) f += L.P + kd * dPd;
      F[I::U(j)] = f;
    }
    // energy remainder, with the pressure work of Pb taken out: the flux
    // of u Pb (no state part) is Pb u_hat, added in FP64 below, so the
    // remainder carries P - Pb = +-dP/2 and keeps the dissipation of
    // pressure differences far below the TF resolution of P itself
    TF gl = uL * (EtL + halfdP), gr = uR * (EtR - halfdP);
    TF g = gl + k * ((gl - gr) + sRu * (EtR - EtL));
    double fe = wide(g);
    double ub2 = 0.0;
#pragma unroll
    for (int j = 0; j < D; j++) ub2 = fma(ub[j], ub[j], ub2);
    const double Pb = L.P - 0.5 * dPd;
    fe = fma(Pb, uhat, fe);
#pragma unroll
    for (int p = 0; p < N; p++) {
      fe = fma(fma(m.A[p], Pb, m.B[p]), F[I::A(p)], fe);
      if (m.hasD) fe = fma(m.D[p], F[p], fe);
    }
    F[I::E] = fma(0.5 * ub2, Frho, fe);
    return;
  }
  // ---------------- HLLC
  double ubn = ub[0];
#pragma unroll
  for (int j = 1; j < D; j++)
    if (j == dir) ubn = ub[j];
  bool left;
  TF sK, chi, chim1, sS;
  // u_K - S*, formed from the differences to ub_n (in TF, u_K and S* round
  // to the same value when they differ by less than the TF resolution of
  // u, and the star pressure P_K + rho_K (s_K - u_K)(S* - u_K) would lose
  // its correction)
  TF uKmS = TF(0);
  double sSd;  // contact speed in FP64 (ub_n + correction) for the momentum flux
  if (ge0(sL) || le0(sR)) {
    left = ge0(sL);
    sK = TF(0);
    chi = TF(1);
    chim1 = TF(0);
    sS = left ? uL : uR;
    sSd = left ? uLd : uRd;
  } else {
    // contact speed relative to ub_n (exact for uniform u and P)
    TF num = cvt<TF>(-dPd) + rL * cvt<TF>(uLd - ubn) * (sL - uL) - rR * cvt<TF>(uRd - ubn) * (sR - uR);
    TF den = rL * (sL - uL) - rR * (sR - uR);
    TF rel = num / den;
    sS = cvt<TF>(ubn) + rel;
    sSd = ubn + wide(rel);
    left = sS >= TF(0);
    sK = left ? sL : sR;
    TF uK = left ? uL : uR;
    // u_K - S* = (u_K - ub_n) - rel
    uKmS = cvt<TF>((left ? uLd : uRd) - ubn) - rel;
    // chi - 1 = (S* - u_K)/(s_K - S*) directly: chi itself rounds to 1 in
    // TF when S* - u_K is below the TF resolution, and u_hat = u_K +
    // s_K (chi - 1) would lose the contact's response to pressure jumps
    const TF dK = sK - uK + uKmS;
    chim1 = -uKmS / dK;
    chi = (sK - uK) / dK;
  }
  const TF uK = left ? uL : uR, rK = left ? rL : rR;
  const TF EtK = left ? EtL : EtR;
  const double uKd = left ? uLd : uRd;
  // u_hat = u_K + s_K (chi - 1)
  uhat = uKd + wide(sK * chim1);
#pragma unroll
  for (int p = 0; p < N; p++) {
    double aK = left ? L.U[I::A(p)] : R.U[I::A(p)];
    double mK = left ? L.U[p] : R.U[p];
    F[I::A(p)] = aK * uhat;
    F[p] = mK * uhat;
    Frho += F[p];
  }
#pragma unroll
  for (int j = 0; j < D; j++) {
    if (j == dir) {
      // S* F^rho + P_K + rho_K (u_K - s_K)(u_K - S*)
      double f = sSd * Frho + (left ? L.P : R.P);
      f += wide(rK * (uK - sK) * uKmS);
      F[I::U(j)] = f;
    } else {
      F[I::U(j)] = (left ? L.u[j] : R.u[j]) * Frho;
    }
  }
  // remainder energy with the HLLC star state.  The pressure work of the
  // star flux is u_K P_K + s_K chi (S* - u_K) P_K / (s_K - u_K) = P_K u_hat;
  // its part Pb u_hat is added in FP64 below and the remainder carries
  // P_K - Pb = +-dP/2, far below the TF resolution of P itself
  const TF pK = left ? halfdP : -halfdP;
  TF Es = chi * (EtK - uKmS * (rK * sS + pK / (sK - uK)));
  if (sK == TF(0)) Es = EtK;
  TF g = uK * (EtK + pK) + sK * (Es - EtK);
  double fe = wide(g);
  double ub2 = 0.0;
#pragma unroll
  for (int j = 0; j < D; j++) ub2 = fma(ub[j], ub[j], ub2);
  const double Pb = L.P - 0.5 * dPd;
  fe = fma(Pb, uhat, fe);
#pragma unroll
  for (int p = 0; p < N; p++) {
    fe = fma(fma(m.A[p], Pb, m.B[p]), F[I::A(p)], fe);
    if (m.hasD) fe = fma(m.D[p], F[p], fe);
  }
  F[I::E] = fma(0.5 * ub2, Frho, fe);
}

// ------------------------------------------------------------------ Phase-Field flux
// Numerical Phase-Field flux of Eq. 5 at the face between L (from cell i) and
// R (from cell i+1), given the face gradients G[p] = (Q_{p,i+1} - Q_{p,i})/dx
// of the auxiliary variables of Eq. 4.  J_p = phi_p (1 - phi_p) grad Q_p is
// upwinded so that it takes phase p only from the side that has it and gives
// it only to the side with room for it:
//   J_p = max(G_p,0) a_R (1 - a_L) + min(G_p,0) a_L (1 - a_R),
// the mass flux has (alpha rho)_p in the outgoing factor (consistent with
// the fractions), and sum_p J_p = 0 is restored by removing sum_q J_q in
// proportion to the face fractions (masses in proportion to the face
// masses), which leaves an absent phase untouched.  Momentum and energy
// follow the last line of Eq. 1 with the mean face velocity and pressure.
// The face gradient of Q_p handed to the Phase-Field flux (Eq. 4-5, reading
// R17): zero on a face Eq. 4 does not couple (both cells with a zero
// coefficient), else (q_r - q_l)/dx limited to |G| <= gmax (gmax > 0, the
// Phase-Field step's sufficient condition for bounds).
// A fraction couples its cell's faces in Eq. 4 when its coefficient
// phi (1 - phi) is nonzero; fractions within one unit of rounding of 0 or 1
// (phi < 2^-52 or 1 - phi < 2^-52, traces the hyperbolic step leaves far
// from any interface) count as 0 (reading R17).
constexpr double PF_TRACE = 0x1p-52;
__device__ __forceinline__ bool pf_active(double a) { return a >= PF_TRACE && 1.0 - a >= PF_TRACE; }

__device__ __forceinline__ double pf_gradient(double ql, double qr, double al, double ar,
                                              double inv_dx, double gmax) {
  const bool coupled = pf_active(al) || pf_active(ar);
  double G = coupled ? (qr - ql) * inv_dx : 0.0;
  if (gmax > 0.0) G = G > gmax ? gmax : (G < -gmax ? -gmax : G);
  return G;
}

template <int N, int D>
__device__ __forceinline__ void pf_flux(const Mat& m, const Face<N, D>& L, const Face<N, D>& R,
                                        const double* G, double* F) {
  using I = Idx<N, D>;
  double J[N], M[N];
  double sumJ = 0.0, suma = 0.0;
#pragma unroll
  for (int p = 0; p < N; p++) {
    const double aL = L.U[I::A(p)], aR = R.U[I::A(p)];
    const double gp = fmax(G[p], 0.0), gm = fmin(G[p], 0.0);
    J[p] = gp * aR * (1.0 - aL) + gm * aL * (1.0 - aR);
    M[p] = gp * R.U[p] * (1.0 - aL) + gm * L.U[p] * (1.0 - aR);
    sumJ += J[p];
    suma += 0.5 * (aL + aR);
  }
  const double r = sumJ / suma;
  double msum = 0.0, e = 0.0;
  const double P = 0.5 * (L.P + R.P);
#pragma unroll
  for (int p = 0; p < N; p++) {
    J[p] -= r * (0.5 * (L.U[I::A(p)] + R.U[I::A(p)]));
    M[p] -= r * (0.5 * (L.U[p] + R.U[p]));
    F[p] = M[p];
    F[I::A(p)] = J[p];
    msum += M[p];
    e = fma(J[p], fma(m.A[p], P, m.B[p]), e);
    if (m.hasD) e = fma(m.D[p], M[p], e);
  }
  double uu = 0.0;
#pragma unroll
  for (int j = 0; j < D; j++) {
    const double u = 0.5 * (L.u[j] + R.u[j]);
    F[I::U(j)] = msum * u;
    uu = fma(u, u, uu);
  }
  F[I::E] = fma(msum, 0.5 * uu, e);
}

}  // namespace wc

