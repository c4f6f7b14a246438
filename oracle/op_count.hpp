// op_count.hpp -- the oracle's operation counter (TEST INFRASTRUCTURE).
//
// Compiling wenoc_oracle.c as C++ with -DOR_COUNT and this header forced in
// front (-include) turns every `double` of the oracle into or_cd, a double
// that counts its arithmetic: add/subtract, multiply, divide, square root
// and comparisons, each attributed to the category of the innermost
// OR_CAT(...) scope the operation runs in.  The arithmetic itself is
// unchanged (each operation is the double operation), so the counting build
// computes the same results as the oracle.  Only tests/ and the op-count
// script under oracle/ load it.
#pragma once
#include <cmath>
#include <cstdlib>
#include <cstring>

enum {
  OR_C_OTHER = 0, OR_C_PRIM, OR_C_BETA, OR_C_CAND, OR_C_WEIGHTS, OR_C_COMBINE, OR_C_LIMIT,
  OR_C_V2U, OR_C_FLUX, OR_C_UPDATE, OR_C_RK, OR_C_CONST, OR_C_RECON, OR_C_NCAT
};
enum { OR_K_ADD = 0, OR_K_MUL, OR_K_DIV, OR_K_SQRT, OR_K_CMP, OR_K_CALLS, OR_K_N };

extern "C" {
extern long long or_op_counts[OR_C_NCAT][OR_K_N];
}
extern int or_op_cat;

struct or_cat_scope {
  int prev;
  explicit or_cat_scope(int c) : prev(or_op_cat) {
    or_op_cat = c;
    or_op_counts[c][OR_K_CALLS] += 1;
  }
  ~or_cat_scope() { or_op_cat = prev; }
};
#define OR_CAT(c) or_cat_scope or_cat_scope_guard_(c)

inline void or_tick(int k) { or_op_counts[or_op_cat][k] += 1; }

struct or_cd {
  double v;
  or_cd() = default;
  or_cd(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  or_cd& operator+=(or_cd o) { or_tick(OR_K_ADD); v += o.v; return *this; }
  or_cd& operator-=(or_cd o) { or_tick(OR_K_ADD); v -= o.v; return *this; }
  or_cd& operator*=(or_cd o) { or_tick(OR_K_MUL); v *= o.v; return *this; }
  or_cd& operator/=(or_cd o) { or_tick(OR_K_DIV); v /= o.v; return *this; }
  or_cd operator-() const { return or_cd(-v); }
  or_cd operator+() const { return *this; }
};
static_assert(sizeof(or_cd) == sizeof(double), "or_cd must lay out as a double");

inline or_cd operator+(or_cd a, or_cd b) { or_tick(OR_K_ADD); return or_cd(a.v + b.v); }
inline or_cd operator-(or_cd a, or_cd b) { or_tick(OR_K_ADD); return or_cd(a.v - b.v); }
inline or_cd operator*(or_cd a, or_cd b) { or_tick(OR_K_MUL); return or_cd(a.v * b.v); }
inline or_cd operator/(or_cd a, or_cd b) { or_tick(OR_K_DIV); return or_cd(a.v / b.v); }
inline bool operator<(or_cd a, or_cd b) { or_tick(OR_K_CMP); return a.v < b.v; }
inline bool operator>(or_cd a, or_cd b) { or_tick(OR_K_CMP); return a.v > b.v; }
inline bool operator<=(or_cd a, or_cd b) { or_tick(OR_K_CMP); return a.v <= b.v; }
inline bool operator>=(or_cd a, or_cd b) { or_tick(OR_K_CMP); return a.v >= b.v; }
inline bool operator==(or_cd a, or_cd b) { or_tick(OR_K_CMP); return a.v == b.v; }
inline bool operator!=(or_cd a, or_cd b) { or_tick(OR_K_CMP); return a.v != b.v; }
inline bool operator!(or_cd a) { return !a.v; }

inline or_cd sqrt(or_cd a) { or_tick(OR_K_SQRT); return or_cd(std::sqrt(a.v)); }
inline or_cd fabs(or_cd a) { return or_cd(std::fabs(a.v)); }
inline or_cd fmin(or_cd a, or_cd b) { or_tick(OR_K_CMP); return or_cd(std::fmin(a.v, b.v)); }
inline or_cd fmax(or_cd a, or_cd b) { or_tick(OR_K_CMP); return or_cd(std::fmax(a.v, b.v)); }
inline or_cd floor(or_cd a) { return or_cd(std::floor(a.v)); }
inline or_cd log2(or_cd a) { return or_cd(std::log2(a.v)); }
inline bool isfinite(or_cd a) { return std::isfinite(a.v); }
using std::isfinite;

#define double or_cd
