// Internal declarations shared by the translation units of libltsoct.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ltsoct.h"

namespace ltsoct {

constexpr int kDepth = 20;        // lattice depth: anchors in [0, 2^20)
constexpr int kMaxLevel = 18;     // deepest level a plan accepts
constexpr int kNP = 7;            // nodes per axis (element order 6)
constexpr int kNV = 343;          // nodes per octant
constexpr int kPW = 13;           // padded width (ghost width 3)
constexpr int kNT = 2197;         // padded points per octant

struct Oct {
  int32_t x, y, z, l;
};

// Time-integration tables of one RK scheme (eq. rk_schemes; eqs. rk_crrection,
// fc_1, fc_2).  omega[rel][s][j]: relation 0 same level, 1 finer source
// (theta 0, rho 2), 2 coarser source in step (theta 0, rho 1/2), 3 coarser
// source half-way through its step (theta 1/2, rho 1/2).
struct Tables {
  int p;
  double a[4][4], w[4], c[4];
  double omega[4][4][4];
  double gamma[4][4];  // stage s of a linear problem: u + sum_m gamma[s][m] dt^(m+1) d^(m+1)u/dt^(m+1)
};

bool make_tables(int rk, Tables* t);
void lagrange_7_to_13(double W[13][7]);
void cubic_extrapolation(double E[4][4]);

// Neighbour tables (o2o): nbr[b*27+d] >= 0 leaf covering the same-size box in
// direction d (same size or one level coarser), -1 outside the domain, <= -2:
// the box is split and fine[(-nbr-2)*8 + c] holds child c (-1: not a leaf).
struct Neighbours {
  std::vector<int32_t> nbr;
  std::vector<int32_t> fine;
};

// Sec. 3.2.2 - 3.2.4 on the device (octree.cu): refinement, 2:1 balance, the leaves in
// level order and their o2o table, on the current device.
lts_status device_octree(const lts_refine_spec& spec, std::vector<Oct>* leaves, Neighbours* nb, std::string* err);

void set_last_error(const std::string& msg);

}  // namespace ltsoct

// The opaque octree handle: the leaves and their o2o table, built on the device and
// kept on the host for the plans' set-up.
struct lts_octree {
  lts_refine_spec spec;
  std::vector<ltsoct::Oct> leaves;  // level order
  ltsoct::Neighbours nb;
};
