// Refinement predicates of the octree construction (Sec. 3.2.2), evaluated on the
// device by the octree build; shared by its host set-up (thresholds) and its kernels.
//
// Integer geometric predicates in lattice units (kinds 0, 1), the box-to-circle distance
// in IEEE doubles from exact integer extents (kind 2), and the wavelet criterion (kind 3).
// Floating-point expressions use explicitly rounded operations on the device (no
// contraction), matching the host's -ffp-contract=off arithmetic step for step.
#pragma once

#include <cmath>
#include <cstdint>

#include "ltsoct_internal.h"

#ifdef __CUDACC__
#define LTS_HD __host__ __device__
#else
#define LTS_HD
#endif

namespace ltsoct {

// Morton key (SFC order, Sec. 3.2.4): x in bit 0, y in bit 1, z in bit 2 of each
// 3-bit group, 20-bit coordinates
LTS_HD inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

LTS_HD inline uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x | x >> 2) & 0x10c30c30c30c30c3ull;
  x = (x | x >> 4) & 0x100f00f00f00f00full;
  x = (x | x >> 8) & 0x1f0000ff0000ffull;
  x = (x | x >> 16) & 0x1f00000000ffffull;
  x = (x | x >> 32) & 0x1fffffull;
  return static_cast<uint32_t>(x);
}

LTS_HD inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// IEEE double operations, rounded once each
LTS_HD inline double rn_mul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
LTS_HD inline double rn_add(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}
LTS_HD inline double rn_sub(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}
LTS_HD inline double rn_div(double a, double b) {
#ifdef __CUDA_ARCH__
  return __ddiv_rn(a, b);
#else
  return a / b;
#endif
}
LTS_HD inline double rn_sqrt(double a) {
#ifdef __CUDA_ARCH__
  return __dsqrt_rn(a);
#else
  return std::sqrt(a);
#endif
}

struct Predicate {
  int kind = 0;
  int n = 0;                      // centres
  int l_min = 0, l_max = 0;
  int64_t c[8][3] = {};           // centres in lattice units
  int64_t r2_out = 0;             // squared outer radius (floor)
  int64_t r2_in = 0;              // squared inner radius (ceil), shell only
  double ring_r = 0, ring_b = 0;  // circle: radius and band in lattice units
  // wavelet criterion: the field sum_c exp(-(|x - c| - radius)^2 / band), tolerance eps
  double lo = 0, hi = 0, radius = 0, band = 0, eps = 0;
  double centers[8][3] = {};
};

// squared distances from a point to the nearest and farthest points of a closed box
LTS_HD inline void box_distances(const int64_t lo[3], int64_t edge, const int64_t c[3], int64_t* dmin2,
                                 int64_t* dmax2) {
  int64_t a = 0, b = 0;
  for (int d = 0; d < 3; ++d) {
    const int64_t hi = lo[d] + edge;
    const int64_t below = c[d] < lo[d] ? lo[d] - c[d] : 0;
    const int64_t above = c[d] > hi ? c[d] - hi : 0;
    const int64_t near = below + above;
    a += near * near;
    const int64_t f0 = c[d] - lo[d] < 0 ? lo[d] - c[d] : c[d] - lo[d];
    const int64_t f1 = hi - c[d] < 0 ? c[d] - hi : hi - c[d];
    const int64_t f = f0 > f1 ? f0 : f1;
    b += f * f;
  }
  *dmin2 = a;
  *dmax2 = b;
}

// circle of radius R in the plane z = c_z around the axis through c: the box's distance
// to it is sqrt(drho^2 + dz^2), drho the gap between R and the box's range
// [rho_min, rho_max] of distances from the axis, dz its gap to the plane
LTS_HD inline bool ring_holds(const Predicate& p, const int64_t lo[3], int64_t edge) {
  int64_t near2 = 0, far2 = 0;
  for (int d = 0; d < 2; ++d) {
    const int64_t hi = lo[d] + edge, c = p.c[0][d];
    const int64_t gap = c < lo[d] ? lo[d] - c : (c > hi ? c - hi : 0);
    near2 += gap * gap;
    const int64_t f0 = c - lo[d] < 0 ? lo[d] - c : c - lo[d];
    const int64_t f1 = hi - c < 0 ? c - hi : hi - c;
    const int64_t f = f0 > f1 ? f0 : f1;
    far2 += f * f;
  }
  const int64_t cz = p.c[0][2];
  const int64_t dz = cz < lo[2] ? lo[2] - cz : (cz > lo[2] + edge ? cz - lo[2] - edge : 0);
  const double rho_min = rn_sqrt(static_cast<double>(near2));
  const double rho_max = rn_sqrt(static_cast<double>(far2));
  const double g1 = rn_sub(rho_min, p.ring_r), g2 = rn_sub(p.ring_r, rho_max);
  const double g = g1 > g2 ? g1 : g2;
  const double drho = g > 0.0 ? g : 0.0;
  const double z = static_cast<double>(dz);
  return rn_add(rn_mul(drho, drho), rn_mul(z, z)) <= rn_mul(p.ring_b, p.ring_b);
}

// kinds 0..2 (kind 3 is evaluated by its own kernel: wavelet_coefficient)
LTS_HD inline bool geometric_holds(const Predicate& p, int64_t x, int64_t y, int64_t z, int level) {
  const int64_t lo[3] = {x, y, z};
  const int64_t edge = int64_t(1) << (kDepth - level);
  if (p.kind == 2) return ring_holds(p, lo, edge);
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

// Wavelet criterion field at lattice6 coordinate (6 a + k e / 2) of a box: in a fixed
// order of rounded operations
LTS_HD inline double wavelet_field(const Predicate& p, const int64_t anchor[3], int64_t edge, int kx, int ky, int kz) {
  const int64_t kk[3] = {kx, ky, kz};
  const double lattice6 = 6.0 * double(int64_t(1) << kDepth);
  const double ext = rn_sub(p.hi, p.lo);
  double x[3];
  for (int d = 0; d < 3; ++d) x[d] = rn_add(p.lo, rn_mul(ext, rn_div(double(6 * anchor[d] + kk[d] * (edge / 2)), lattice6)));
  double f = 0.0;
  for (int c = 0; c < p.n; ++c) {
    double d2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double t = rn_sub(x[d], p.centers[c][d]);
      d2 = rn_add(d2, rn_mul(t, t));
    }
    const double r = rn_sub(rn_sqrt(d2), p.radius);
    f = rn_add(f, std::exp(rn_div(-rn_mul(r, r), p.band)));
  }
  return f;
}

// 1-D weights of the wavelet criterion: the degree-6 Lagrange basis on the even
// half-node positions at position k, exact rationals rounded once
LTS_HD inline double wavelet_weight(int k, int j) {
  int64_t num = 1, den = 1;
  for (int m = 0; m < 7; ++m)
    if (m != j) {
      num *= int64_t(k - 2 * m);
      den *= int64_t(2 * j - 2 * m);
    }
  return rn_div(double(num), double(den));
}

Predicate make_predicate(const lts_refine_spec& s);  // thresholds in lattice units (host)

}  // namespace ltsoct
