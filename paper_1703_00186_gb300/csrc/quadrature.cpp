// D2Q37 quadrature and wall ratios, derived on the host in double-double
// arithmetic and rounded once to float64.
//
// The paper uses the D2Q37 model (Sect. 2) without listing it.  The velocity
// set is the 37 integer vectors xi with |xi_x|, |xi_y| <= 3 and |xi|^2 in
// {0,1,2,4,5,8,9,10}; c_l = r xi_l.  The eight shell weights and r make every
// even moment of order <= 8 equal to that of a unit Gaussian:
//   sum_l w_l (r xi_lx)^a (r xi_ly)^b = (a-1)!! (b-1)!!,
// nine independent conditions under the square symmetry.  They are solved
// here by Newton's method on the nine unknowns (w_0..w_7, y = 1/r^2) with
// double-double arithmetic (error-free transforms of Dekker and Knuth), so
// that every constant handed to the kernels is the float64 nearest to its
// exact value.  The wall ratios of the bc are formed the same way.
//
// Compiled with -ffp-contract=off: the error-free transforms rely on
// separately rounded products and sums.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>

#include "lbm_internal.h"

namespace lbm {
namespace {

struct dd {
  double hi, lo;
};

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
inline dd fast_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
inline dd D(double a) { return {a, 0.0}; }
inline dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return {-a.hi, -a.lo}; }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = a - b * D(q1);
  double q2 = r.hi / b.hi;
  r = r - b * D(q2);
  double q3 = r.hi / b.hi;
  return fast_two_sum(q1, q2) + D(q3);
}
inline dd dd_sqrt(dd a) {
  double x = std::sqrt(a.hi);
  dd xx = D(x);
  // two Newton steps x <- x + (a - x^2) / (2x)
  for (int i = 0; i < 2; ++i) xx = xx + (a - xx * xx) / (D(2.0) * xx);
  return xx;
}
inline double dabs(dd a) { return std::fabs(a.hi); }

constexpr int kShell[NSHELL] = {0, 1, 2, 4, 5, 8, 9, 10};
// Isotropy monomials xi_x^a xi_y^b, a >= b, both even, a + b <= 8.
constexpr int kMonA[9] = {0, 2, 4, 2, 6, 4, 8, 6, 4};
constexpr int kMonB[9] = {0, 0, 0, 2, 0, 2, 0, 2, 4};

double ipow(int v, int e) {
  double out = 1.0;
  for (int i = 0; i < e; ++i) out *= v;
  return out;
}
double double_factorial(int n) {  // (n)!!, with (-1)!! = 1
  double out = 1.0;
  for (int k = n; k > 1; k -= 2) out *= k;
  return out;
}

// Solve the 9x9 system A x = b in double-double (Gaussian elimination with
// partial pivoting).  Returns false if singular.
bool solve9(dd A[9][9], dd b[9], dd x[9]) {
  const int n = 9;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (dabs(A[r][c]) > dabs(A[p][c])) p = r;
    if (A[p][c].hi == 0.0) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c][k], A[p][k]);
      std::swap(b[c], b[p]);
    }
    for (int r = c + 1; r < n; ++r) {
      dd f = A[r][c] / A[c][c];
      for (int k = c; k < n; ++k) A[r][k] = A[r][k] - f * A[c][k];
      b[r] = b[r] - f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    dd s = b[r];
    for (int k = r + 1; k < n; ++k) s = s - A[r][k] * x[k];
    x[r] = s / A[r][r];
  }
  return true;
}

// phi(s) = f^eq(1, 0, T) / w for a population of shell |xi|^2 = s:
// 1 + theta (c2 - 2) / 2 + theta^2 (c2^2 - 8 c2 + 8) / 8, c2 = s / y.
dd phi_over_w(dd y, int s, dd theta) {
  dd c2 = D((double)s) / y;
  dd t1 = theta * (c2 - D(2.0)) / D(2.0);
  dd t2 = theta * theta * (c2 * c2 - D(8.0) * c2 + D(8.0)) / D(8.0);
  return D(1.0) + t1 + t2;
}

}  // namespace

int solve_quadrature(Quadrature* out, char* err, size_t errlen) {
  // Moment matrix: M[i][j] = sum over shell j of xi_x^a_i xi_y^b_i (integers).
  double M[9][NSHELL];
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < NSHELL; ++j) {
      double acc = 0.0;
      for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
          if (a * a + b * b == kShell[j]) acc += ipow(a, kMonA[i]) * ipow(b, kMonB[i]);
      M[i][j] = acc;
    }
  double G[9];
  int K[9];
  for (int i = 0; i < 9; ++i) {
    G[i] = double_factorial(kMonA[i] - 1) * double_factorial(kMonB[i] - 1);
    K[i] = (kMonA[i] + kMonB[i]) / 2;
  }
  // Newton on F_i(w, y) = sum_j M_ij w_j - G_i y^K_i.
  dd w[NSHELL] = {D(0.23), D(0.1), D(0.05), D(0.015), D(0.005), D(0.001), D(0.0003), D(0.0003)};
  dd y = D(0.7);
  double last = 1.0;
  for (int it = 0; it < 60; ++it) {
    dd A[9][9], F[9], dx[9];
    for (int i = 0; i < 9; ++i) {
      dd yk = D(1.0);
      for (int k = 0; k < K[i]; ++k) yk = yk * y;
      dd f = -(D(G[i]) * yk);
      for (int j = 0; j < NSHELL; ++j) {
        f = f + D(M[i][j]) * w[j];
        A[i][j] = D(M[i][j]);
      }
      dd ykm1 = D(1.0);
      for (int k = 0; k + 1 < K[i]; ++k) ykm1 = ykm1 * y;
      A[i][8] = K[i] ? -(D(G[i] * K[i]) * ykm1) : D(0.0);
      F[i] = -f;
    }
    if (!solve9(A, F, dx)) {
      std::snprintf(err, errlen, "quadrature Newton step singular");
      return -1;
    }
    double step = 0.0;
    for (int j = 0; j < NSHELL; ++j) {
      w[j] = w[j] + dx[j];
      step = std::fmax(step, std::fabs(dx[j].hi));
    }
    y = y + dx[8];
    step = std::fmax(step, std::fabs(dx[8].hi));
    if (step < 1e-31 || (step >= last && step < 1e-28)) break;
    last = step;
  }
  // Verify all nine conditions at double-double accuracy.
  for (int i = 0; i < 9; ++i) {
    dd yk = D(1.0);
    for (int k = 0; k < K[i]; ++k) yk = yk * y;
    dd f = -(D(G[i]) * yk);
    for (int j = 0; j < NSHELL; ++j) f = f + D(M[i][j]) * w[j];
    if (std::fabs(f.hi) > 1e-28 * std::fmax(1.0, G[i])) {
      std::snprintf(err, errlen, "quadrature residual %g in condition %d", f.hi, i);
      return -1;
    }
  }
  for (int j = 0; j < NSHELL; ++j)
    if (!(w[j].hi > 0.0)) {
      std::snprintf(err, errlen, "non-positive quadrature weight");
      return -1;
    }
  dd r = D(1.0) / dd_sqrt(y);
  out->r = r.hi;
  out->y = y.hi;
  for (int j = 0; j < NSHELL; ++j) {
    out->w_shell[j] = w[j].hi;
    out->c2_shell[j] = (D((double)kShell[j]) / y).hi;
  }
  for (int l = 0; l < NPOP; ++l) out->w[l] = w[shell_index(sq(l))].hi;
  for (int j = 0; j < NSHELL; ++j) out->w_shell_lo[j] = w[j].lo;
  out->y_lo = y.lo;
  return 0;
}

void wall_ratios(const Quadrature& q, double t_wall, int wall, double out[NPOP]) {
  dd theta = two_sum(t_wall, -1.0);
  dd y = {q.y, q.y_lo};
  dd phi[NPOP];
  for (int l = 0; l < NPOP; ++l) {
    int j = shell_index(sq(l));
    phi[l] = dd{q.w_shell[j], q.w_shell_lo[j]} * phi_over_w(y, sq(l), theta);
  }
  // Unknown slots: rows d = 0, 1, 2 from the wall; population l is unknown in
  // row d if its velocity component towards the lattice exceeds d.
  dd tot = D(0.0);
  for (int d = 0; d < 3; ++d)
    for (int l = 0; l < NPOP; ++l) {
      int toward = wall == 0 ? vy(l) : -vy(l);
      if (toward > d) tot = tot + phi[l];
    }
  for (int l = 0; l < NPOP; ++l) {
    int toward = wall == 0 ? vy(l) : -vy(l);
    out[l] = toward > 0 ? (phi[l] / tot).hi : 0.0;
  }
}

// Inverse Gram blocks of the w-weighted monomials xi_x^c xi_y^d (c + d <= 4)
// over the 37 velocities, split by the parity of (c, d):
//   EE [1, x^2, y^2, x^4, x^2 y^2, y^4], OE [x, x^3, x y^2],
//   EO [y, y^3, x^2 y], OO [x y, x^3 y, x y^3],
// inverted in double-double and rounded once.  Output order: EE (36), OE (9),
// EO (9), OO (9), each row-major.
namespace {
bool invert_dd(int n, dd (*A)[6], dd (*X)[6]) {
  dd M[6][12];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? A[i][j] : D(j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (dabs(M[r][c]) > dabs(M[p][c])) p = r;
    if (M[p][c].hi == 0.0) return false;
    if (p != c)
      for (int k = 0; k < 2 * n; ++k) std::swap(M[c][k], M[p][k]);
    const dd inv = D(1.0) / M[c][c];
    for (int k = 0; k < 2 * n; ++k) M[c][k] = M[c][k] * inv;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const dd f = M[r][c];
        for (int k = 0; k < 2 * n; ++k) M[r][k] = M[r][k] - f * M[c][k];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) X[i][j] = M[i][n + j];
  return true;
}
}  // namespace

int regularization_gram_inverse(const Quadrature& q, double out[63]) {
  static const int blocks[4][6][2] = {
      {{0, 0}, {2, 0}, {0, 2}, {4, 0}, {2, 2}, {0, 4}},
      {{1, 0}, {3, 0}, {1, 2}, {0, 0}, {0, 0}, {0, 0}},
      {{0, 1}, {0, 3}, {2, 1}, {0, 0}, {0, 0}, {0, 0}},
      {{1, 1}, {3, 1}, {1, 3}, {0, 0}, {0, 0}, {0, 0}}};
  static const int sizes[4] = {6, 3, 3, 3};
  int o = 0;
  for (int b = 0; b < 4; ++b) {
    const int n = sizes[b];
    dd G[6][6], X[6][6];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        dd acc = D(0.0);
        for (int l = 0; l < NPOP; ++l) {
          const double m = ipow(vx(l), blocks[b][i][0] + blocks[b][j][0]) * ipow(vy(l), blocks[b][i][1] + blocks[b][j][1]);
          const int s = shell_index(sq(l));
          acc = acc + dd{q.w_shell[s], q.w_shell_lo[s]} * D(m);
        }
        G[i][j] = acc;
      }
    if (!invert_dd(n, G, X)) return -1;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) out[o++] = X[i][j].hi;
  }
  return 0;
}

}  // namespace lbm
