// Host-side set-up of libltsoct: octree construction and 2:1 balance (Sec. 3.2.2,
// 3.2.3), neighbour tables (o2o, Sec. 3.2.4) and the time-integration tables
// (eq. rk_schemes; eqs. rk_crrection, fc_1, fc_2).
//
// Compiled with -ffp-contract=off: the refinement predicate's thresholds come
// from double arithmetic that must give the same integers on every machine.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <unordered_set>

#include "ltsoct_internal.h"

namespace ltsoct {

namespace {
thread_local std::string g_last_error;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Morton keys (SFC order, Sec. 3.2.4): x in bit 0, y in bit 1, z in bit 2 of
// each 3-bit group.  Magic-number spreading of 20-bit coordinates.
// ---------------------------------------------------------------------------
static uint64_t spread_bits(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

uint64_t morton_key(uint32_t x, uint32_t y, uint32_t z) {
  return spread_bits(x) | (spread_bits(y) << 1) | (spread_bits(z) << 2);
}

// ---------------------------------------------------------------------------
// Refinement predicate in lattice units (integer geometric predicate in place
// of the wavelet criterion of Sec. 3.2.2).
// ---------------------------------------------------------------------------
namespace {

struct Predicate {
  int kind = 0;
  int n = 0;
  int64_t c[8][3];
  int64_t r2_out = 0;  // squared outer radius (floor)
  int64_t r2_in = 0;   // squared inner radius (ceil), shell only
  double ring_r = 0, ring_b = 0;  // circle: radius and band in lattice units
  lts_refine_spec spec;           // wavelet criterion: the field and tolerance
};

Predicate make_predicate(const lts_refine_spec& s) {
  Predicate p;
  p.kind = s.kind;
  p.spec = s;
  p.n = s.kind == 0 || s.kind == 3 ? s.n_centers : 1;
  const double scale = static_cast<double>(int64_t(1) << kDepth);
  const double ext = s.hi - s.lo;
  for (int i = 0; i < p.n; ++i)
    for (int d = 0; d < 3; ++d) p.c[i][d] = std::llround((s.centers[i][d] - s.lo) / ext * scale);
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
  return p;
}

// squared distances from a point to the nearest and farthest points of a closed box
inline void box_distances(const int64_t lo[3], int64_t edge, const int64_t c[3], int64_t* dmin2, int64_t* dmax2) {
  int64_t a = 0, b = 0;
  for (int d = 0; d < 3; ++d) {
    const int64_t hi = lo[d] + edge;
    const int64_t below = c[d] < lo[d] ? lo[d] - c[d] : 0;
    const int64_t above = c[d] > hi ? c[d] - hi : 0;
    const int64_t near = below + above;
    a += near * near;
    const int64_t f = std::max(std::llabs(c[d] - lo[d]), std::llabs(hi - c[d]));
    b += f * f;
  }
  *dmin2 = a;
  *dmax2 = b;
}

// circle of radius R in the plane z = c_z around the axis through c: the box's
// distance to it is sqrt(drho^2 + dz^2), drho the gap between R and the box's
// range [rho_min, rho_max] of distances from the axis, dz its gap to the plane.
// Evaluated in IEEE doubles (exact integer inputs, correctly rounded sqrt, no
// contraction), so the decision is the same on every host.
bool ring_holds(const Predicate& p, const int64_t lo[3], int64_t edge) {
  int64_t near2 = 0, far2 = 0;
  for (int d = 0; d < 2; ++d) {
    const int64_t hi = lo[d] + edge, c = p.c[0][d];
    const int64_t gap = c < lo[d] ? lo[d] - c : (c > hi ? c - hi : 0);
    near2 += gap * gap;
    const int64_t f = std::max(std::llabs(c - lo[d]), std::llabs(hi - c));
    far2 += f * f;
  }
  const int64_t cz = p.c[0][2];
  const int64_t dz = cz < lo[2] ? lo[2] - cz : (cz > lo[2] + edge ? cz - lo[2] - edge : 0);
  const double rho_min = std::sqrt(static_cast<double>(near2));
  const double rho_max = std::sqrt(static_cast<double>(far2));
  const double drho = std::max(0.0, std::max(rho_min - p.ring_r, p.ring_r - rho_max));
  const double z = static_cast<double>(dz);
  return drho * drho + z * z <= p.ring_b * p.ring_b;
}

// Wavelet criterion (Sec. 3.2.2): the largest failure, over the half-node points of the
// box that are not its nodes, of the degree-6 Lagrange interpolant from the box's 7^3
// nodes to reproduce the field sum_c exp(-(|x - c| - radius)^2 / band).  Weights are the
// exact rationals prod_{m != j} (k - 2m) / prod_{m != j} (2j - 2m), each rounded once;
// sums run in a fixed order without contraction, so every host decides alike.
double wavelet_coefficient(const lts_refine_spec& s, const int64_t anchor[3], int64_t edge) {
  double w[13][7];
  for (int k = 0; k < 13; ++k)
    for (int j = 0; j < 7; ++j) {
      int64_t num = 1, den = 1;
      for (int m = 0; m < 7; ++m)
        if (m != j) {
          num *= int64_t(k - 2 * m);
          den *= int64_t(2 * j - 2 * m);
        }
      w[k][j] = double(num) / double(den);
    }
  std::vector<double> F(13 * 13 * 13);
  const double lattice6 = 6.0 * double(int64_t(1) << kDepth);
  for (int kz = 0; kz < 13; ++kz)
    for (int ky = 0; ky < 13; ++ky)
      for (int kx = 0; kx < 13; ++kx) {
        const int64_t kk[3] = {kx, ky, kz};
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = s.lo + (s.hi - s.lo) * (double(6 * anchor[d] + kk[d] * (edge / 2)) / lattice6);
        double f = 0.0;
        for (int c = 0; c < s.n_centers; ++c) {
          double d2 = 0.0;
          for (int d = 0; d < 3; ++d) {
            const double t = x[d] - s.centers[c][d];
            d2 += t * t;
          }
          const double r = std::sqrt(d2) - s.radius;
          f += std::exp(-(r * r) / s.band);
        }
        F[kx + 13 * ky + 169 * kz] = f;
      }
  double worst = 0.0;
  for (int kz = 0; kz < 13; ++kz)
    for (int ky = 0; ky < 13; ++ky)
      for (int kx = 0; kx < 13; ++kx) {
        if (!((kx | ky | kz) & 1)) continue;
        double vz = 0.0;
        for (int c = 0; c < 7; ++c) {
          double vy = 0.0;
          for (int b = 0; b < 7; ++b) {
            double vx = 0.0;
            for (int a = 0; a < 7; ++a) vx = vx + w[kx][a] * F[2 * a + 26 * b + 338 * c];
            vy = vy + w[ky][b] * vx;
          }
          vz = vz + w[kz][c] * vy;
        }
        const double gap = std::fabs(F[kx + 13 * ky + 169 * kz] - vz);
        if (gap > worst) worst = gap;
      }
  return worst;
}

bool predicate_holds(const Predicate& p, const Oct& o) {
  const int64_t lo[3] = {o.x, o.y, o.z};
  const int64_t edge = int64_t(1) << (kDepth - o.l);
  if (p.kind == 2) return ring_holds(p, lo, edge);
  if (p.kind == 3) return wavelet_coefficient(p.spec, lo, edge) > p.spec.eps;
  for (int i = 0; i < p.n; ++i) {
    int64_t dmin2, dmax2;
    box_distances(lo, edge, p.c[i], &dmin2, &dmax2);
    if (p.kind == 0) {
      if (dmin2 <= p.r2_out) return true;
    } else if (dmin2 <= p.r2_out && dmax2 >= p.r2_in) {
      return true;
    }
  }
  return false;
}

inline uint64_t pack_anchor(int32_t x, int32_t y, int32_t z) { return morton_key(x, y, z); }

inline Oct child_of(const Oct& o, int c) {
  const int32_t h = int32_t(1) << (kDepth - o.l - 1);
  return Oct{o.x + (c & 1) * h, o.y + ((c >> 1) & 1) * h, o.z + ((c >> 2) & 1) * h, o.l + 1};
}

}  // namespace

// Sec. 3.2.2 + 3.2.3.  Refinement breadth-first by level, then the 2:1 balance
// as the closure of the node set under (i) parents, (ii) siblings and (iii) the
// parent of every same-size neighbour box of a node, applied finest level first
// so one sweep suffices; its leaves are the coarsest 26-neighbour balanced
// refinement of the refined tree.
bool build_octree(const lts_refine_spec& spec, std::vector<Oct>* leaves, std::string* err) {
  if (!(spec.hi > spec.lo) || spec.l_min < 0 || spec.l_max < spec.l_min || spec.l_max > kMaxLevel ||
      spec.kind < 0 || spec.kind > 3 ||
      ((spec.kind == 0 || spec.kind == 3) && (spec.n_centers < 1 || spec.n_centers > 8)) ||
      (spec.kind == 3 && !(spec.band > 0.0 && spec.eps > 0.0))) {
    *err = "octree_build: invalid refinement spec (need lo < hi, 0 <= l_min <= l_max <= 18, kind 0..3, 1..8 centers; "
           "kind 3: band > 0, eps > 0)";
    return false;
  }
  const Predicate pred = make_predicate(spec);
  // refinement, level by level
  std::vector<Oct> cur{Oct{0, 0, 0, 0}}, next, refined;
  while (!cur.empty()) {
    next.clear();
    for (const Oct& o : cur) {
      const bool split = o.l < spec.l_min || (o.l < spec.l_max && predicate_holds(pred, o));
      if (split)
        for (int c = 0; c < 8; ++c) next.push_back(child_of(o, c));
      else
        refined.push_back(o);
    }
    std::swap(cur, next);
  }
  // balance by closure, per level sets of anchors
  const int top = spec.l_max;
  std::vector<std::unordered_set<uint64_t>> S(top + 2);
  for (const Oct& o : refined) S[o.l].insert(pack_anchor(o.x, o.y, o.z));
  auto unpack = [](uint64_t k, int l) {
    uint32_t c[3] = {0, 0, 0};
    for (int b = 0; b < 21; ++b)
      for (int d = 0; d < 3; ++d) c[d] |= static_cast<uint32_t>((k >> (3 * b + d)) & 1u) << b;
    return Oct{int32_t(c[0]), int32_t(c[1]), int32_t(c[2]), l};
  };
  const int64_t root = int64_t(1) << kDepth;
  for (int l = top; l >= 1; --l) {
    // (ii) siblings: every node's parent gets all 8 children
    std::vector<uint64_t> nodes(S[l].begin(), S[l].end());
    const int32_t pe = int32_t(1) << (kDepth - l + 1);
    for (uint64_t k : nodes) {
      Oct o = unpack(k, l);
      Oct par{o.x / pe * pe, o.y / pe * pe, o.z / pe * pe, l - 1};
      for (int c = 0; c < 8; ++c) {
        Oct ch = child_of(par, c);
        S[l].insert(pack_anchor(ch.x, ch.y, ch.z));
      }
    }
    // (i) parents and (iii) parents of neighbour boxes
    const int32_t e = int32_t(1) << (kDepth - l);
    for (uint64_t k : S[l]) {
      Oct o = unpack(k, l);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int64_t nx = int64_t(o.x) + dx * e, ny = int64_t(o.y) + dy * e, nz = int64_t(o.z) + dz * e;
            if (nx < 0 || ny < 0 || nz < 0 || nx >= root || ny >= root || nz >= root) continue;
            S[l - 1].insert(pack_anchor(int32_t(nx / pe * pe), int32_t(ny / pe * pe), int32_t(nz / pe * pe)));
          }
    }
  }
  // leaves: nodes without children
  leaves->clear();
  for (int l = 0; l <= top; ++l)
    for (uint64_t k : S[l]) {
      Oct o = unpack(k, l);
      if (l + 1 <= top && S[l + 1].count(pack_anchor(o.x, o.y, o.z))) continue;
      leaves->push_back(o);
    }
  std::sort(leaves->begin(), leaves->end(), [](const Oct& a, const Oct& b) {
    if (a.l != b.l) return a.l < b.l;
    return morton_key(a.x, a.y, a.z) < morton_key(b.x, b.y, b.z);
  });
  return true;
}

// o2o (Sec. 3.2.4) through per-level hash maps of the leaves.
lts_status build_neighbours(const std::vector<Oct>& octs, Neighbours* out, std::string* err) {
  const int64_t n = static_cast<int64_t>(octs.size());
  int lmax = 0;
  for (const Oct& o : octs) lmax = std::max(lmax, int(o.l));
  std::vector<std::unordered_map<uint64_t, int32_t>> at(lmax + 2);
  for (int64_t i = 0; i < n; ++i) at[octs[i].l][morton_key(octs[i].x, octs[i].y, octs[i].z)] = int32_t(i);
  out->nbr.assign(n * 27, -1);
  out->fine.clear();
  const int64_t root = int64_t(1) << kDepth;
  for (int64_t b = 0; b < n; ++b) {
    const Oct& o = octs[b];
    const int32_t e = int32_t(1) << (kDepth - o.l);
    for (int d = 0; d < 27; ++d) {
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const int64_t nx = int64_t(o.x) + dx * e, ny = int64_t(o.y) + dy * e, nz = int64_t(o.z) + dz * e;
      int32_t& slot = out->nbr[b * 27 + d];
      if (nx < 0 || ny < 0 || nz < 0 || nx >= root || ny >= root || nz >= root) {
        slot = -1;
        continue;
      }
      auto it = at[o.l].find(morton_key(uint32_t(nx), uint32_t(ny), uint32_t(nz)));
      if (it != at[o.l].end()) {
        slot = it->second;
        continue;
      }
      if (o.l >= 1) {
        const int64_t pe = int64_t(2) * e;
        auto ip = at[o.l - 1].find(morton_key(uint32_t(nx / pe * pe), uint32_t(ny / pe * pe), uint32_t(nz / pe * pe)));
        if (ip != at[o.l - 1].end()) {
          slot = ip->second;
          continue;
        }
        // a leaf two or more levels coarser covers the box: unbalanced
        for (int l = o.l - 2; l >= 0; --l) {
          const int64_t ae = int64_t(1) << (kDepth - l);
          if (at[l].count(morton_key(uint32_t(nx / ae * ae), uint32_t(ny / ae * ae), uint32_t(nz / ae * ae)))) {
            *err = "lts_plan_create: octree is not 2:1 balanced across faces, edges and corners";
            return LTS_EUNBALANCED;
          }
        }
      }
      // the box is split: its children (those touching b must be leaves)
      const int32_t f = int32_t(out->fine.size() / 8);
      const int32_t h = e / 2;
      for (int c = 0; c < 8; ++c) {
        const int64_t cx = nx + (c & 1) * h, cy = ny + ((c >> 1) & 1) * h, cz = nz + ((c >> 2) & 1) * h;
        auto ic = o.l + 1 <= lmax ? at[o.l + 1].find(morton_key(uint32_t(cx), uint32_t(cy), uint32_t(cz)))
                                  : at[o.l].end();
        const bool leaf = o.l + 1 <= lmax && ic != at[o.l + 1].end();
        out->fine.push_back(leaf ? ic->second : -1);
        const bool touches = (dx == 0 || (dx < 0) == ((c & 1) == 1)) && (dy == 0 || (dy < 0) == (((c >> 1) & 1) == 1)) &&
                             (dz == 0 || (dz < 0) == (((c >> 2) & 1) == 1));
        if (touches && !leaf) {
          *err = "lts_plan_create: octree is not 2:1 balanced (a finer neighbour is two levels finer)";
          return LTS_EUNBALANCED;
        }
      }
      slot = -(2 + f);
    }
  }
  return LTS_OK;
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
