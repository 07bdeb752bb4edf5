/*
 * Counting build of the oracle (TEST INFRASTRUCTURE; see d2q37_oracle.c).
 *
 * The oracle's C source is compiled here as C++ with its `double` replaced by
 * a type that counts every floating-point addition, subtraction,
 * multiplication and division it performs (comparisons, conversions and
 * copies are not counted).  The arithmetic itself is unchanged.
 * orc_count_collide_form returns the operations of one site collision
 * (moments, shifted fields, equilibrium, relaxation), in the oracle's form
 * (the equilibrium as the full Hermite tensor contractions) or in the
 * hand-contracted scalar form of collide_contracted.c, the plain
 * per-population FP64 work of the method.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

namespace flopcount {

// every operation, and the non-trivial ones: a product or quotient with an
// operand of exactly 0 or +-1 (the Kronecker factors of the tensor form) and a
// sum with an operand of exactly 0 are left out of the second count
static uint64_t g_ops = 0, g_nontrivial = 0;

inline bool unitish(double x) { return x == 0.0 || x == 1.0 || x == -1.0; }
inline void count_add(double a, double b) { ++g_ops; if (a != 0.0 && b != 0.0) ++g_nontrivial; }
inline void count_mul(double a, double b) { ++g_ops; if (!unitish(a) && !unitish(b)) ++g_nontrivial; }
inline void count_div(double a, double b) { ++g_ops; if (a != 0.0 && b != 1.0 && b != -1.0) ++g_nontrivial; }

struct cd {
  double v;
  cd() : v(0.0) {}
  cd(double x) : v(x) {}
  operator double() const { return v; }
  cd& operator+=(cd o) { count_add(v, o.v); v += o.v; return *this; }
  cd& operator-=(cd o) { count_add(v, o.v); v -= o.v; return *this; }
  cd& operator*=(cd o) { count_mul(v, o.v); v *= o.v; return *this; }
  cd& operator/=(cd o) { count_div(v, o.v); v /= o.v; return *this; }
};
inline cd operator+(cd a, cd b) { count_add(a.v, b.v); return cd(a.v + b.v); }
inline cd operator-(cd a, cd b) { count_add(a.v, b.v); return cd(a.v - b.v); }
inline cd operator*(cd a, cd b) { count_mul(a.v, b.v); return cd(a.v * b.v); }
inline cd operator/(cd a, cd b) { count_div(a.v, b.v); return cd(a.v / b.v); }
inline cd operator-(cd a) { return cd(-a.v); }
inline cd operator+(cd a, double b) { return a + cd(b); }
inline cd operator+(double a, cd b) { return cd(a) + b; }
inline cd operator-(cd a, double b) { return a - cd(b); }
inline cd operator-(double a, cd b) { return cd(a) - b; }
inline cd operator*(cd a, double b) { return a * cd(b); }
inline cd operator*(double a, cd b) { return cd(a) * b; }
inline cd operator/(cd a, double b) { return a / cd(b); }
inline cd operator/(double a, cd b) { return cd(a) / b; }
inline cd operator*(cd a, int b) { return a * cd((double)b); }
inline cd operator*(int a, cd b) { return cd((double)a) * b; }
inline cd operator/(cd a, int b) { return a / cd((double)b); }

}  // namespace flopcount

using flopcount::cd;
#define double cd
#include "d2q37_oracle.c"
#include "collide_contracted.c"
#undef double

extern "C" {

/* FP64 operations of one site collision of the oracle (orc_count_setup
 * first): all of them, or (nontrivial != 0) those without a trivial operand.
 * form 0: the oracle's collision (equilibrium as the full tensor
 * contractions); form 1: the same collision with the hand-contracted scalar
 * equilibrium of collide_contracted.c. */
long long orc_count_collide_form(int form, int nontrivial) {
  cd fc[Q], oc[Q];
  for (int l = 0; l < Q; ++l) fc[l] = cd(w_[l].v * (1.0 + 0.01 * (l % 5)));
  flopcount::g_ops = flopcount::g_nontrivial = 0;
  if (form == 0)
    orc_collide_site(fc, cd(0.8), cd(0.0), cd(-1e-4), oc);
  else
    orc_collide_site_contracted(fc, cd(0.8), cd(0.0), cd(-1e-4), oc);
  return (long long)(nontrivial ? flopcount::g_nontrivial : flopcount::g_ops);
}

long long orc_count_collide_site(int nontrivial) { return orc_count_collide_form(0, nontrivial); }

/* The relaxed populations of either form for populations f (plain doubles
 * in and out), so that tests can check that the counted forms agree. */
void orc_collide_form_values(int form, const double* f, double tau, double gx, double gy,
                             double* out) {
  cd fc[Q], oc[Q];
  for (int l = 0; l < Q; ++l) fc[l] = cd(f[l]);
  if (form == 0)
    orc_collide_site(fc, cd(tau), cd(gx), cd(gy), oc);
  else
    orc_collide_site_contracted(fc, cd(tau), cd(gx), cd(gy), oc);
  for (int l = 0; l < Q; ++l) out[l] = oc[l].v;
}

}

extern "C" int orc_count_setup(double s, const double* w_shell) {
  cd w[NSHELL];
  for (int k = 0; k < NSHELL; ++k) w[k] = cd(w_shell[k]);
  return orc_setup(cd(s), w);
}
