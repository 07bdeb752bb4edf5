// Quadrature of the D2Q37 lattice, solved on the host in double-double
// arithmetic when the library is first used.
//
// The paper uses a 37-velocity lattice with hops of up to 3 sites (Sec.
// "Lattice Boltzmann methods", Fig. streamscheme) but does not print the
// velocities or weights.  This library reads the set as every integer c with
// |c|^2 <= 10 (8 shells) and xi_l = s c_l, and fixes s and one weight per
// shell by the 9 Gaussian moment conditions
//     sum_l w_l xi_x^i xi_y^j = E[X^i] E[Y^j],
//     (i,j) in {(0,0),(2,0),(4,0),(2,2),(6,0),(4,2),(8,0),(6,2),(4,4)},
// which make the rule exact to degree 9 (enough for the 4th-order Hermite
// equilibrium of Eq. MASTERSHIFT3).
//
// Method: for a given s the conditions are linear in the weights; the eight
// conditions other than (8,0) are solved for w(s) and the remaining residual
// r(s) = sum_l w_l(s) xi_x^8 - 105 is driven to zero by bisection.  All of it
// runs in double-double (about 106 significant bits; Dekker's two-product via
// fma and Knuth's two-sum, as in Hida, Li & Bailey's QD library), so the
// rounded FP64 results carry no error from the solve.
#include <cmath>
#include <cstdlib>

#include "d2q37_lattice.cuh"

namespace d2q37 {
namespace {

struct dd {
  double hi, lo;
};

dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}

dd make(double a) { return {a, 0.0}; }

dd add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

dd neg(dd x) { return {-x.hi, -x.lo}; }
dd sub(dd x, dd y) { return add(x, neg(y)); }

dd mul(dd x, dd y) {
  double p = x.hi * y.hi;
  double e = std::fma(x.hi, y.hi, -p);
  e += x.hi * y.lo + x.lo * y.hi;
  return quick_two_sum(p, e);
}

dd div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = sub(x, mul(make(q1), y));
  double q2 = r.hi / y.hi;
  r = sub(r, mul(make(q2), y));
  double q3 = r.hi / y.hi;
  dd q = quick_two_sum(q1, q2);
  return add(q, make(q3));
}

dd ipow(dd x, int n) {
  dd r = make(1.0);
  for (int i = 0; i < n; ++i) r = mul(r, x);
  return r;
}

double dabs(dd x) { return std::fabs(x.hi); }

const int kOrders[9][2] = {{0, 0}, {2, 0}, {4, 0}, {2, 2}, {6, 0}, {4, 2}, {8, 0}, {6, 2}, {4, 4}};

// E[Z^k] of a standard normal.
double normal_moment(int k) {
  if (k % 2) return 0.0;
  double m = 1.0;
  for (int i = k - 1; i > 0; i -= 2) m *= i;
  return m;
}

// Integer shell sums B[e][k] = sum_{l in shell k} cx^i cy^j (exact in FP64).
void shell_sums(double B[9][kShells]) {
  for (int e = 0; e < 9; ++e)
    for (int k = 0; k < kShells; ++k) B[e][k] = 0.0;
  for (int l = 0; l < kQ; ++l) {
    for (int e = 0; e < 9; ++e) {
      double v = 1.0;
      for (int a = 0; a < kOrders[e][0]; ++a) v *= kCx[l];
      for (int a = 0; a < kOrders[e][1]; ++a) v *= kCy[l];
      B[e][kShellOf[l]] += v;
    }
  }
}

// Weights at scale s from the eight conditions other than (8,0); returns the
// residual of the (8,0) condition, or a NaN if the system is singular.
dd weights_at(dd s, const double B[9][kShells], dd w[kShells]) {
  dd A[8][kShells + 1];
  int row = 0;
  for (int e = 0; e < 9; ++e) {
    if (kOrders[e][0] == 8) continue;
    dd sn = ipow(s, kOrders[e][0] + kOrders[e][1]);
    for (int k = 0; k < kShells; ++k) A[row][k] = mul(sn, make(B[e][k]));
    A[row][kShells] = make(normal_moment(kOrders[e][0]) * normal_moment(kOrders[e][1]));
    ++row;
  }
  for (int c = 0; c < kShells; ++c) {
    int p = c;
    for (int r = c + 1; r < kShells; ++r)
      if (dabs(A[r][c]) > dabs(A[p][c])) p = r;
    if (dabs(A[p][c]) == 0.0) return make(NAN);
    for (int k = 0; k <= kShells; ++k) {
      dd t = A[c][k];
      A[c][k] = A[p][k];
      A[p][k] = t;
    }
    for (int r = c + 1; r < kShells; ++r) {
      dd f = div(A[r][c], A[c][c]);
      for (int k = c; k <= kShells; ++k) A[r][k] = sub(A[r][k], mul(f, A[c][k]));
    }
  }
  for (int r = kShells - 1; r >= 0; --r) {
    dd acc = A[r][kShells];
    for (int k = r + 1; k < kShells; ++k) acc = sub(acc, mul(A[r][k], w[k]));
    w[r] = div(acc, A[r][r]);
  }
  dd s8 = ipow(s, 8);
  dd acc = make(0.0);
  for (int k = 0; k < kShells; ++k) acc = add(acc, mul(w[k], make(B[6][k])));
  return sub(mul(s8, acc), make(normal_moment(8)));
}

}  // namespace

bool solve_quadrature(double* s_out, double w_shell_out[kShells]) {
  double B[9][kShells];
  shell_sums(B);
  dd w[kShells];
  // bracket a sign change of the residual by scanning s in [0.3, 2.5]
  dd lo = make(0.3), hi;
  dd r_lo = weights_at(lo, B, w);
  bool found = false;
  for (int i = 1; i <= 220; ++i) {
    hi = make(0.3 + 0.01 * i);
    dd r_hi = weights_at(hi, B, w);
    if (std::isfinite(r_lo.hi) && std::isfinite(r_hi.hi) && (r_lo.hi < 0) != (r_hi.hi < 0)) {
      found = true;
      break;
    }
    lo = hi;
    r_lo = r_hi;
  }
  if (!found) return false;
  for (int it = 0; it < 200; ++it) {
    dd mid = mul(add(lo, hi), make(0.5));
    dd r_mid = weights_at(mid, B, w);
    if ((r_mid.hi < 0) == (r_lo.hi < 0)) {
      lo = mid;
      r_lo = r_mid;
    } else {
      hi = mid;
    }
    if (dabs(sub(hi, lo)) < 1e-31) break;
  }
  dd s = mul(add(lo, hi), make(0.5));
  weights_at(s, B, w);
  *s_out = s.hi + s.lo;
  for (int k = 0; k < kShells; ++k) {
    if (!(w[k].hi > 0.0)) return false;
    w_shell_out[k] = w[k].hi + w[k].lo;
  }
  return true;
}

}  // namespace d2q37
