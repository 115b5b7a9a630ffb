// Host-side set-up of libltsoct: the refinement predicate's thresholds (the octree
// and its neighbour tables are built on the device, octree.cu), the operators' weights
// and the time-integration tables (eq. rk_schemes; eqs. rk_crrection, fc_1, fc_2).
//
// Compiled with -ffp-contract=off: the refinement predicate's thresholds come
// from double arithmetic that must give the same integers on every machine.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ltsoct_internal.h"
#include "refine.h"

namespace ltsoct {

namespace {
thread_local std::string g_last_error;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Refinement predicate thresholds in lattice units (the octree itself is built on the
// device, octree.cu): integer geometric predicates in place of the wavelet criterion of
// Sec. 3.2.2, the circle's radius and band, and the wavelet criterion's field.
// ---------------------------------------------------------------------------
Predicate make_predicate(const lts_refine_spec& s) {
  Predicate p;
  p.kind = s.kind;
  p.l_min = s.l_min;
  p.l_max = s.l_max;
  p.n = s.kind == 0 || s.kind == 3 ? s.n_centers : 1;
  const double scale = static_cast<double>(int64_t(1) << kDepth);
  const double ext = s.hi - s.lo;
  for (int i = 0; i < p.n; ++i)
    for (int d = 0; d < 3; ++d) {
      p.c[i][d] = std::llround((s.centers[i][d] - s.lo) / ext * scale);
      p.centers[i][d] = s.centers[i][d];
    }
  p.ring_r = s.radius / ext * scale;
  p.ring_b = s.band / ext * scale;
  const double outer = s.kind == 1 ? s.radius + s.band : s.radius;
  const double ro = outer / ext * scale;
  p.r2_out = static_cast<int64_t>(std::floor(ro * ro));
  if (s.kind == 1) {
    const double inner = s.radius - s.band;
    if (inner > 0) {
      const double ri = inner / ext * scale;
      p.r2_in = static_cast<int64_t>(std::ceil(ri * ri));
    }
  }
  p.lo = s.lo;
  p.hi = s.hi;
  p.radius = s.radius;
  p.band = s.band;
  p.eps = s.eps;
  return p;
}

// ---------------------------------------------------------------------------
// Operators
// ---------------------------------------------------------------------------

// 1-D degree-6 Lagrange basis on nodes 0..6 at positions r/2, r = 0..12 (rows of
// even r are exact unit vectors).
void lagrange_7_to_13(double W[13][7]) {
  for (int r = 0; r < 13; ++r) {
    const double x = 0.5 * r;
    for (int m = 0; m < 7; ++m) {
      if (r % 2 == 0) {
        W[r][m] = (2 * m == r) ? 1.0 : 0.0;
        continue;
      }
      double num = 1.0, den = 1.0;
      for (int q = 0; q < 7; ++q) {
        if (q == m) continue;
        num *= x - q;
        den *= double(m - q);
      }
      W[r][m] = num / den;
    }
  }
}

// cubic extrapolation to -m (m = 1..3) from the values at 0, 1, 2, 3
void cubic_extrapolation(double E[4][4]) {
  std::memset(E, 0, sizeof(double) * 16);
  for (int m = 1; m <= 3; ++m)
    for (int q = 0; q < 4; ++q) {
      double num = 1.0, den = 1.0;
      for (int s = 0; s < 4; ++s) {
        if (s == q) continue;
        num *= double(-m - s);
        den *= double(q - s);
      }
      E[m][q] = num / den;
    }
}

// ---------------------------------------------------------------------------
// RK tableaus and the stage corrections
// ---------------------------------------------------------------------------
namespace {

// Gauss-Jordan inverse of a small dense matrix
bool invert(int n, const double A[4][4], double out[4][4]) {
  double M[4][8] = {};
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) M[i][j] = A[i][j];
    M[i][n + i] = 1.0;
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return false;
    for (int j = 0; j < 2 * n; ++j) std::swap(M[c][j], M[piv][j]);
    const double inv = 1.0 / M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == c || M[r][c] == 0.0) continue;
      const double f = M[r][c];
      for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i][j] = M[i][n + j];
  return true;
}

double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }

}  // namespace

bool make_tables(int rk, Tables* t) {
  std::memset(t, 0, sizeof(*t));
  if (rk == 4) {
    t->p = 4;
    t->a[1][0] = 0.5;
    t->a[2][1] = 0.5;
    t->a[3][2] = 1.0;
    t->w[0] = 1.0 / 6.0;
    t->w[1] = 1.0 / 3.0;
    t->w[2] = 1.0 / 3.0;
    t->w[3] = 1.0 / 6.0;
  } else if (rk == 3) {
    t->p = 3;
    t->a[1][0] = 1.0;
    t->a[2][0] = 0.25;
    t->a[2][1] = 0.25;
    t->w[0] = 1.0 / 6.0;
    t->w[1] = 1.0 / 6.0;
    t->w[2] = 2.0 / 3.0;
  } else {
    return false;
  }
  const int p = t->p;
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) t->c[i] += t->a[i][j];
  // eq. rk_crrection for a linear autonomous right-hand side: stage i is
  // sum_m C[i][m] dt^m d^(m+1)u/dt^(m+1) with C[.][0] = 1 and C[.][m] = A C[.][m-1]
  double C[4][4] = {};
  for (int i = 0; i < p; ++i) C[i][0] = 1.0;
  for (int m = 1; m < p; ++m)
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) C[i][m] += t->a[i][j] * C[j][m - 1];
  double Ci[4][4];
  if (!invert(p, C, Ci)) return false;
  // gamma = A C
  for (int s = 0; s < p; ++s)
    for (int m = 0; m < p; ++m)
      for (int j = 0; j < p; ++j) t->gamma[s][m] += t->a[s][j] * C[j][m];
  // eqs. fc_1 / fc_2 in units dt_source = 1: a requester step starting theta later
  // with dt = rho rebuilds the source's derivatives (C^-1), shifts them by theta
  // (Taylor matrix B_theta) and forms its own stage inputs with P_rho and A.
  const double rel[4][2] = {{0.0, 1.0}, {0.0, 2.0}, {0.0, 0.5}, {0.5, 0.5}};
  for (int r = 0; r < 4; ++r) {
    const double th = rel[r][0], rho = rel[r][1];
    for (int s = 0; s < p; ++s) {
      double row[4] = {};
      for (int m = 0; m < p; ++m) row[m] = std::pow(th, m + 1) / fact(m + 1);
      for (int q = 0; q < p; ++q) {
        double aC = 0.0;
        for (int j = 0; j < p; ++j) aC += t->a[s][j] * C[j][q];
        const double coef = rho * aC * std::pow(rho, q);
        for (int m = q; m < p; ++m) row[m] += coef * std::pow(th, m - q) / fact(m - q);
      }
      for (int j = 0; j < p; ++j) {
        double v = 0.0;
        for (int m = 0; m < p; ++m) v += row[m] * Ci[m][j];
        t->omega[r][s][j] = v;
      }
    }
  }
  // the same-level relation is the tableau itself; store it exactly
  for (int s = 0; s < p; ++s)
    for (int j = 0; j < p; ++j) t->omega[0][s][j] = t->a[s][j];
  return true;
}

}  // namespace ltsoct
