// CUDA kernels of libltsoct for GB300 (sm_103a).
//
// The LTS substep (Alg. 2, Fig. blk_loop) runs, per RK stage, one launch of
// prolong_kernel and one of stage_kernel over the active octants (a contiguous
// suffix of the level order).
//   prolong_kernel: one CTA per octant with finer neighbours forms its stage
//     inputs as those neighbours see them (eqs. fc_1, fc_2) and interpolates
//     them to the half-node positions they read (Fig. unzip, coarse -> fine).
//   stage_kernel: one CTA per active octant reads the source of each of the
//     2197 points of its padded block from the plan's padding map (Sec. 3.3:
//     coarsest leaf containing the point, ties to the smallest Morton key =
//     smallest level-order index; resolved once per plan by padmap_kernel),
//     gathers the sources' stage inputs into shared memory, fills the physical
//     boundary, evaluates the 4th-order FD right-hand side with Kreiss-Oliger
//     dissipation on the 7^3 interior and writes the stage, the next stage's
//     inputs and, at the last stage, the RK update of eq. rk_schemes into the
//     other half of the double-buffered state.
//
// Precision.  The state u, the RK update and the time corrections are FP64.
// The stage type R (stages, stage inputs, prolonged inputs, the padded tile
// and the right-hand side) is double, or float in the mixed-precision mode.
// FP64 on GB300 issues about 2 DFMA per clock per SM, so the FP64 kernels are
// bound by the FP64 pipe; integer work and memory traffic hide behind it.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "kernels.cuh"

namespace ltsoct {

struct DevTables {
  int p;
  double a[4][4], w[4], omega[4][4][4], gamma[4][4];
};

__constant__ DevTables c_tab[2];  // 0: RK4, 1: SSPRK3
__constant__ double c_W[13][7];   // Lagrange 7 -> 13
__constant__ double c_E[4][4];    // cubic extrapolation weights, rows m = 1..3

constexpr int kThreads = 352;     // 11 warps: the 343 interior nodes in one pass
constexpr int kLatt6 = 6 << kDepth;

// padded points of a sibling-group block tile (19^3) outside its 13^3 nodes, in tile order
__device__ unsigned short g_block_ghost[kBG];

// boundary nodes of an octant (a coordinate 0 or 6), in node order
__device__ unsigned short g_bnode[kBN];

// node of the 13^3 stage tile whose FP32 right-hand side thread t evaluates (-1: none).
// Lane l of every warp takes a node whose tile index c0 is l mod 32, so the 19 loads per
// field of a node hit 32 different banks; in node order, rows of 7 nodes at a row stride
// of 13 put two nodes of a warp on one bank.  (The order is also free of conflicts for
// 8-byte loads, but the FP64 kernel, bound by its FP64 pipe, measured no gain from it.)
__device__ short g_rhs_node[kThreads];


cudaError_t upload_tables(const Tables* rk4, const Tables* rk3, const double W[13][7], const double E[4][4]) {
  {
    unsigned short bn[kBN];
    int n = 0;
    for (int q = 0; q < kNV; ++q) {
      const int i = q % 7, j = (q / 7) % 7, k = q / 49;
      if (i == 0 || i == 6 || j == 0 || j == 6 || k == 0 || k == 6) bn[n++] = static_cast<unsigned short>(q);
    }
    if (n != kBN) return cudaErrorInvalidValue;
    const cudaError_t e = cudaMemcpyToSymbol(g_bnode, bn, sizeof(bn));
    if (e != cudaSuccess) return e;
  }
  {
    // tile nodes by bank (c0 mod 32); warp w takes the w-th node of every bank
    short order[kThreads];
    int taken[32] = {0};
    for (int t = 0; t < kThreads; ++t) order[t] = -1;
    for (int w = 0; w < kThreads / 32; ++w)
      for (int l = 0; l < 32; ++l) {
        int seen = 0;
        for (int q = 0; q < kNV; ++q) {
          const int c0 = (q % 7 + 3) + 13 * ((q / 7) % 7 + 3) + 169 * (q / 49 + 3);
          if (c0 % 32 != l) continue;
          if (seen++ == taken[l]) {
            order[w * 32 + l] = static_cast<short>(q);
            ++taken[l];
            break;
          }
        }
      }
    int placed = 0;
    for (int l = 0; l < 32; ++l) placed += taken[l];
    if (placed != kNV) return cudaErrorInvalidValue;  // 343 nodes over 11 warps: 10 or 11 per bank
    const cudaError_t e = cudaMemcpyToSymbol(g_rhs_node, order, sizeof(order));
    if (e != cudaSuccess) return e;
  }
  {
    unsigned short ghost[kBG];
    int n = 0;
    for (int q = 0; q < kBT; ++q) {
      const int i = q % kBW - 3, j = (q / kBW) % kBW - 3, k = q / (kBW * kBW) - 3;
      if (i < 0 || i > 12 || j < 0 || j > 12 || k < 0 || k > 12) ghost[n++] = static_cast<unsigned short>(q);
    }
    if (n != kBG) return cudaErrorInvalidValue;
    const cudaError_t e = cudaMemcpyToSymbol(g_block_ghost, ghost, sizeof(ghost));
    if (e != cudaSuccess) return e;
  }
  DevTables h[2];
  const Tables* src[2] = {rk4, rk3};
  for (int i = 0; i < 2; ++i) {
    h[i].p = src[i]->p;
    for (int s = 0; s < 4; ++s) {
      for (int j = 0; j < 4; ++j) {
        h[i].a[s][j] = src[i]->a[s][j];
        h[i].gamma[s][j] = src[i]->gamma[s][j];
        for (int r = 0; r < 4; ++r) h[i].omega[r][s][j] = src[i]->omega[r][s][j];
      }
      h[i].w[s] = src[i]->w[s];
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_tab, h, sizeof(h));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_W, W, sizeof(double) * 13 * 7);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_E, E, sizeof(double) * 16);
}

// ---------------------------------------------------------------------------
// Source resolution (Sec. 3.3 / Fig. dg_to_cg ownership): the leaves whose
// closed boxes contain a point of the padded block lie in the same-size
// neighbour boxes whose closure contains it; the source is the one with the
// smallest level-order index (coarsest, then smallest Morton key).
// ---------------------------------------------------------------------------
struct NbrView {
  int nbr[27];
  int kids[27][8];
};

__device__ __forceinline__ void axis_candidates(int i, int& d0, int& d1) {
  if (i < 0) {
    d0 = d1 = -1;
  } else if (i == 0) {
    d0 = -1;
    d1 = 0;
  } else if (i < 6) {
    d0 = d1 = 0;
  } else if (i == 6) {
    d0 = 0;
    d1 = 1;
  } else {
    d0 = d1 = 1;
  }
}

// slot of a source in the neighbour view: d (0..26, 13 = the octant itself) for the
// leaf covering neighbour box d, 27 + 8 d + c for child c of a split box d
constexpr unsigned kSlotNone = 255u;

// (i,j,k) in the octant's node units, i in [-3, 9]; returns -1 outside the domain.
// With `slot`, also reports the source's slot (kSlotNone outside the domain).
__device__ int resolve_source(const NbrView& nv, int i, int j, int k, int self, bool with_self,
                              unsigned* slot = nullptr) {
  int x0, x1, y0, y1, z0, z1;
  axis_candidates(i, x0, x1);
  axis_candidates(j, y0, y1);
  axis_candidates(k, z0, z1);
  int best = INT_MAX;
  unsigned best_slot = kSlotNone;
  for (int dz = z0; dz <= z1; ++dz)
    for (int dy = y0; dy <= y1; ++dy)
      for (int dx = x0; dx <= x1; ++dx) {
        const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        if (d == 13) {
          if (with_self && self < best) {
            best = self;
            best_slot = 13u;
          }
          continue;
        }
        const int e = nv.nbr[d];
        if (e == -1) continue;
        if (e >= 0) {
          if (e < best) {
            best = e;
            best_slot = unsigned(d);
          }
          continue;
        }
        // split neighbour box: children whose closed boxes contain the point
        const int px = i - 6 * dx, py = j - 6 * dy, pz = k - 6 * dz;  // in [0, 6]
        const int hx0 = px <= 3 ? 0 : 1, hx1 = px >= 3 ? 1 : 0;
        const int hy0 = py <= 3 ? 0 : 1, hy1 = py >= 3 ? 1 : 0;
        const int hz0 = pz <= 3 ? 0 : 1, hz1 = pz >= 3 ? 1 : 0;
        for (int hz = hz0; hz <= hz1; ++hz)
          for (int hy = hy0; hy <= hy1; ++hy)
            for (int hx = hx0; hx <= hx1; ++hx) {
              const int leaf = nv.kids[d][hx + 2 * hy + 4 * hz];
              if (leaf >= 0 && leaf < best) {
                best = leaf;
                best_slot = 27u + 8u * unsigned(d) + unsigned(hx + 2 * hy + 4 * hz);
              }
            }
      }
  if (slot) *slot = best_slot;
  return best == INT_MAX ? -1 : best;
}

// the leaf in a slot of the neighbour view (-1 for kSlotNone)
__device__ __forceinline__ int slot_leaf(const NbrView& nv, unsigned slot, int self) {
  if (slot == 13u) return self;
  if (slot < 27u) return nv.nbr[slot];
  if (slot < kSlotNone) return (&nv.kids[0][0])[slot - 27u];
  return -1;
}

// half-node coordinate of lattice6 coordinate P in a source with anchor a, level l
__device__ __forceinline__ int half_node(int P, int a, int l) { return ((P - 6 * a) * 2) >> (kDepth - l); }

// No barrier inside: the children entries read their box's entry from global memory,
// and every caller synchronises before it reads nv.
__device__ void load_neighbours(const DevTree& t, int b, NbrView& nv) {
  for (int d = threadIdx.x; d < 27; d += blockDim.x) nv.nbr[d] = __ldg(t.nbr + b * 27 + d);
  for (int q = threadIdx.x; q < 27 * 8; q += blockDim.x) {
    const int d = q >> 3, c = q & 7;
    const int e = __ldg(t.nbr + b * 27 + d);
    nv.kids[d][c] = e <= -2 ? __ldg(t.fine + (-e - 2) * 8 + c) : -1;
  }
}


// stage input of a source node from its step-start state and RK stages,
// u + dt * sum_t w_t K_(j_t), in FP64 (eq. rk_schemes with the corrected weights
// of eqs. fc_1 / fc_2)
//
// FP32 -> FP64 by bit manipulation, exact like the hardware conversion, on the integer
// pipes: on GB300 conversions execute on the small FP64 pipe, which the mixed-precision
// kernels also need for their FP64 accumulations.  Subnormal, infinite and NaN inputs take
// the hardware conversion.
__device__ __forceinline__ double widen(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 255u;
  if (e - 1u < 254u) {  // normal: exponent rebiased 127 -> 1023, mantissa 23 -> 52 bits
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double(int(hi), int(u << 29));
  }
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double(int(u & 0x80000000u), 0);  // +-0
  return static_cast<double>(x);
}

template <typename T>
__device__ __forceinline__ double to_double(T x) {
  if constexpr (sizeof(T) == sizeof(float)) {
    return widen(x);
  } else {
    return x;
  }
}

//
// C selects the load path: false, the read-only data path (data written by earlier
// launches); true, loads through L2 (ld.global.cg) for data that the same launch may have
// written (the persistent batch round, whose stages follow each other inside one launch).
template <bool C, typename T>
__device__ __forceinline__ T ld_in(const T* p) {
  if constexpr (C) {
    return __ldcg(p);
  } else {
    return __ldg(p);
  }
}

template <typename R, bool C = false>
__device__ __forceinline__ double corrected_value(const double* __restrict__ u, const R* __restrict__ k0,
                                                  long long kstride, const StageTerms& t, double dt) {
  if (t.n == 0) return ld_in<C>(u);  // no correction (stage 0 of a source in its own step)
  double acc = 0.0;
  for (int q = 0; q < t.n; ++q) acc = fma(t.w[q], to_double(ld_in<C>(k0 + t.j[q] * kstride)), acc);
  return fma(dt, acc, ld_in<C>(u));
}

// tensor-product Lagrange interpolation, x then y then z; even coordinates are nodes
template <typename T>
__device__ T interp_tensor(const T* __restrict__ v, const double (*W)[7], int rx, int ry, int rz) {
  const int x0 = (rx & 1) ? 0 : rx >> 1, x1 = (rx & 1) ? 6 : rx >> 1;
  const int y0 = (ry & 1) ? 0 : ry >> 1, y1 = (ry & 1) ? 6 : ry >> 1;
  const int z0 = (rz & 1) ? 0 : rz >> 1, z1 = (rz & 1) ? 6 : rz >> 1;
  T sz = 0;
  for (int c = z0; c <= z1; ++c) {
    T sy = 0;
    for (int bb = y0; bb <= y1; ++bb) {
      T sx = 0;
      for (int a = x0; a <= x1; ++a) sx = fma(T(W[rx][a]), v[a + 7 * bb + 49 * c], sx);
      sy = fma(T(W[ry][bb]), sx, sy);
    }
    sz = fma(T(W[rz][c]), sy, sz);
  }
  return sz;
}

// g^(m)(0), m = 0..5, of g(s) = exp(q0 + q1 s + q2 s^2)
__device__ void expquad(double q0, double q1, double q2, double g[6]) {
  const double G = exp(q0), Q1 = q1, Q2 = 2.0 * q2;
  const double Q1s = Q1 * Q1;
  g[0] = G;
  g[1] = Q1 * G;
  g[2] = (Q2 + Q1s) * G;
  g[3] = (3.0 * Q1 * Q2 + Q1s * Q1) * G;
  g[4] = (3.0 * Q2 * Q2 + 6.0 * Q1s * Q2 + Q1s * Q1s) * G;
  g[5] = (15.0 * Q1 * Q2 * Q2 + 10.0 * Q1s * Q1 * Q2 + Q1s * Q1s * Q1) * G;
}

// closed-form solution and time derivatives d[f][m], m = 0..4, for exact boundary data
__device__ void exact_derivs(int ic, const IcParams& P, const double adv[3], const double x[3], double t,
                             double d[2][5]) {
  if (ic == LTS_IC_ADV_GAUSS) {
    double adot = 0.0, aa = 0.0, dsq = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double dd = x[a] - P.v[a] - adv[a] * t;
      adot += adv[a] * dd;
      aa += adv[a] * adv[a];
      dsq += dd * dd;
    }
    const double w = P.v[3];
    double g[6];
    expquad(-dsq / w, 2.0 * adot / w, -aa / w, g);
    for (int m = 0; m < 5; ++m) {
      d[0][m] = g[m];
      d[1][m] = 0.0;
    }
  } else {  // LTS_IC_WAVE_PLANAR
    const double s0 = P.v[0], w = P.v[1];
    const double sm = x[0] - t - s0, sp = x[0] + t - s0;
    double gm[6], gp[6];
    expquad(-sm * sm / w, -2.0 * sm / w, -1.0 / w, gm);
    expquad(-sp * sp / w, -2.0 * sp / w, -1.0 / w, gp);
    double chi[6];
    for (int m = 0; m < 6; ++m) chi[m] = 0.5 * ((m & 1) ? gp[m] - gm[m] : gp[m] + gm[m]);
    for (int m = 0; m < 5; ++m) {
      d[0][m] = chi[m];
      d[1][m] = chi[m + 1];
    }
  }
}

__device__ __forceinline__ double lattice_to_x(double lo, double ext, int P6) {
  return lo + ext * (static_cast<double>(P6) / (6.0 * static_cast<double>(1 << kDepth)));
}

// ---------------------------------------------------------------------------
// The stage kernel
// ---------------------------------------------------------------------------
// kinds of a slot of the neighbour view, as seen from the octant being stepped
constexpr int kKindCoarser = 0, kKindSame = 1, kKindFiner = 2, kKindNone = 3;
constexpr int kSlots = 256;  // slot values of a padding-map entry (kSlotNone = 255 included)

// Shared memory of the stage kernel: NB tile buffers with their slot tables (the stage
// kernel and the batch kernels use one).
template <int NF, typename R, int NB>
struct StageSmem {
  R T[NB][NF][kNT];               // padded tiles
  int slot[NB][kSlots];           // per slot: base << 2 | kind (the plan's slot map)
  R KV[sizeof(R) == sizeof(float) ? NF : 1][sizeof(R) == sizeof(float) ? kNV : 1];  // FP32: staged right-hand sides
  R orb[NB][2];                   // orbit centre x_1 at the octant's stage time
};

constexpr unsigned kExterior = 1u << 15;  // exterior flag of the 16-bit codes of the block map

// The padding map holds one byte per padded point: the slot of its source in the
// octant's neighbour view (kSlotNone outside the domain).  Where the point lies in the
// source follows from the slot's relation to the octant.  With (i, j, k) the point in
// the octant's node units (each in [-3, 9]):
//   same level, neighbour box d: node (i, j, k) - 6 d of the stage inputs
//                                -> base + lin7,  lin7 = i + 7 j + 49 k
//   finer, child c of the split box d: node 2 ((i, j, k) - 6 d - 3 c), even, whose stage
//                                input the injection pass put at even-node index
//                                (i, j, k) - 6 d - 3 c (4 per axis)
//                                -> base + lin4,  lin4 = i + 4 j + 16 k
//   coarser leaf N: its prolonged 13^3 block, half-node (i, j, k) + 6 (A_b - A_N) / e_b
//                                -> base + q
// q being the point's tile index (i + 3) + 13 (j + 3) + 169 (k + 3); base is fixed per
// slot and octant (the plan's slot map, slotmap_kernel).

constexpr int kPer = (kNT + kThreads - 1) / kThreads;  // padded points per thread of a stage CTA

// A stage CTA's thread t gathers the points of one column (i, j) of the 13^3 tile: column
// t mod 169, tile levels 0..6 for t < 169 and 7..12 for 169 <= t < 338 (threads from 338 on
// take none), so that its point r is q0 + 169 r, at lin7 = l7 + 49 r and lin4 = l4 + 16 r
// in the source numberings above: one division per thread instead of one per
// point, and consecutive threads still read consecutive points.
struct TileColumn {
  int q0, l7, l4, n;  // first point, its offsets, points taken
  __device__ __forceinline__ explicit TileColumn(int t) {
    const int h = t >= 169 ? 1 : 0, c = t - 169 * h;
    const int j = c / 13, i = c - 13 * j, k0 = 7 * h;
    q0 = c + 169 * k0;
    l7 = (i - 3) + 7 * (j - 3) + 49 * (k0 - 3);
    l4 = (i - 3) + 4 * (j - 3) + 16 * (k0 - 3);
    n = t >= 338 ? 0 : 7 - h;
  }
};
static_assert(kPer == 7 && kThreads >= 338, "the tile-column assignment covers 13^3 points with 338 threads");

// exterior padded point of octant (anchor me, edge eb): outside the domain
__device__ __forceinline__ bool exterior_point(int4 me, int eb, int q) {
  const int i = q % 13 - 3, j = (q / 13) % 13 - 3, k = q / 169 - 3;
  const int P[3] = {6 * me.x + i * eb, 6 * me.y + j * eb, 6 * me.z + k * eb};
  return P[0] < 0 || P[1] < 0 || P[2] < 0 || P[0] > kLatt6 || P[1] > kLatt6 || P[2] > kLatt6;
}

// exact boundary data (a reading of the paper): RK stage values of the closed-form solution
template <int NF, typename R>
__device__ __noinline__ void fill_exact(R (*T)[kNT], const StageArgs& A, int4 me, int eb, double dtb) {
  for (int q = threadIdx.x; q < kNT; q += blockDim.x) {
    if (!exterior_point(me, eb, q)) continue;
    const int i = q % 13 - 3, j = (q / 13) % 13 - 3, k = q / 169 - 3;
    const double x[3] = {lattice_to_x(A.lo, A.ext, 6 * me.x + i * eb), lattice_to_x(A.lo, A.ext, 6 * me.y + j * eb),
                         lattice_to_x(A.lo, A.ext, 6 * me.z + k * eb)};
    double d[2][5];
    exact_derivs(A.ic, A.icp, A.adv, x, A.t_b, d);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      double v = d[f][0], dtp = 1.0;
      for (int m = 0; m < A.p; ++m) {
        dtp *= dtb;
        v = fma(A.gamma[m] * dtp, d[f][m + 1], v);
      }
      T[f][q] = static_cast<R>(v);
    }
  }
}

// radiative boundary (a reading of the paper): cubic extrapolation along the outward normal, x then y then z
template <int NF, typename R>
__device__ __noinline__ void fill_extrapolated(R (*T)[kNT], int4 me, int eb) {
  const int anchor[3] = {me.x, me.y, me.z};
  constexpr int kRoot = 1 << kDepth;
  for (int a = 0; a < 3; ++a) {
    const bool lo_b = anchor[a] == 0, hi_b = anchor[a] + eb == kRoot;
    if (lo_b || hi_b) {
      const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
      const int str = a == 0 ? 1 : (a == 1 ? 13 : 169);
      const int str1 = b1 == 0 ? 1 : (b1 == 1 ? 13 : 169);
      const int str2 = b2 == 0 ? 1 : (b2 == 1 ? 13 : 169);
      for (int t = threadIdx.x; t < 169 * 3; t += blockDim.x) {
        const int v1 = t % 13 - 3, v2 = (t / 13) % 13 - 3, m = t / 169 + 1;
        const bool ext1 = (anchor[b1] == 0 && v1 < 0) || (anchor[b1] + eb == kRoot && v1 > 6);
        const bool ext2 = (anchor[b2] == 0 && v2 < 0) || (anchor[b2] + eb == kRoot && v2 > 6);
        if ((b1 > a && ext1) || (b2 > a && ext2)) continue;
        const int base = 3 * str + (v1 + 3) * str1 + (v2 + 3) * str2;  // index 0 along axis a
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (lo_b) {
            R v = 0;
            for (int qq = 0; qq < 4; ++qq) v = fma(R(c_E[m][qq]), T[f][base + qq * str], v);
            T[f][base - m * str] = v;
          }
          if (hi_b) {
            R v = 0;
            for (int qq = 0; qq < 4; ++qq) v = fma(R(c_E[m][qq]), T[f][base + (6 - qq) * str], v);
            T[f][base + (6 + m) * str] = v;
          }
        }
      }
    }
    __syncthreads();
  }
}

// radiative right-hand side at a node on the domain boundary; T[f] are the padded
// tiles (y stride SY, z stride SZ), c0 the node's tile index
template <int NF, typename R, int SY, int SZ>
__device__ __noinline__ void radiative_rhs(const R* const* T, const StageArgs& A, int c0, const int P6[3], R inv12h,
                                           R kv[NF]) {
  const R x[3] = {R(lattice_to_x(A.lo, A.ext, P6[0])), R(lattice_to_x(A.lo, A.ext, P6[1])),
                  R(lattice_to_x(A.lo, A.ext, P6[2]))};
  const R r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const int st[3] = {1, SY, SZ};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const R* Tf = T[f];
    R xd = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R d1 = fma(R(8), Tf[c0 + st[a]] - Tf[c0 - st[a]], Tf[c0 - 2 * st[a]] - Tf[c0 + 2 * st[a]]) * inv12h;
      xd = fma(x[a], d1, xd);
    }
    kv[f] = -(xd + (f == 0 ? R(1) : R(2)) * Tf[c0]) / r;
  }
}

// ---------------------------------------------------------------------------
// FP64 wave right-hand side by exact integer stencil sums.  The 4th-order Laplacian and
// the Kreiss-Oliger operator have integer coefficients (in units of 1/(12 h^2) and of the
// dissipation constant), so at each node the stencil inputs of a field are put on a common
// 2^(E - 1075) grid, E the largest biased exponent among them: input x becomes the integer
// sign(x) trunc(|x| 2^(1075 - E)), |.| < 2^53, exact for every input in E's binade and
// truncated below it (each to within 2^-52 of the largest input, the size of an FP64
// operation's rounding).  Sums and integer combinations are then exact in 64 bits (|.| <
// 192 x 2^53 < 2^61) and each result is rounded once to FP64.  GB300 issues integer
// operations at 32 times its FP64 rate (64 lanes per clock and SM against 2), but a
// conversion costs about a dozen of them, so the work is split between the two pipes:
// chi's Laplacian and dissipation (its 19 stencil inputs) are exact integer sums, phi's
// dissipation stays in FP64 (18 of the 41 FP64 operations of a wave node); of the splits
// that move whole pair sums between the pipes, this one measured fastest.  The result
// depends only on the node's own stencil inputs, so every kernel that evaluates a node
// (stage, block, batch; LTS or GTS) gets the same bits.  Nodes whose largest chi input lies
// outside [2^-968, 2^500) (other than all zero), or whose chi inputs hold an infinity or
// NaN, take the floating-point evaluation instead; subnormal inputs beside normal ones lie
// below a grid unit and truncate to zero.
// ---------------------------------------------------------------------------

// exponent field (bits 20..30 of the high word, in place) of the double at w
__device__ __forceinline__ unsigned fix_expbits(const double* w) {
  return reinterpret_cast<const unsigned*>(w)[1] & 0x7ff00000u;
}

// An exact sum of inputs on the grid 2^(E - 1075): the magnitudes truncated onto the grid
// with their signs applied as one's complements (x ^ s, s = 0 or -1), plus the count of
// negative inputs, which completes the two's complements.
struct FixSum {
  long long ones = 0;
  int neg = 0;
  __device__ __forceinline__ long long value() const { return ones + neg; }
};

// adds x (exponent field <= em, E = em >> 20 in [55, 1523]) to a: sign(x) trunc(|x| 2^(1075 - E)).
// The implicit bit is set for every input: a zero or subnormal input lies at least E >= 55
// binades below the grid's top and is shifted out all the same (a -0 adds ~0 + 1 = 0).
__device__ __forceinline__ void fix_add(FixSum& a, double x, unsigned em) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned lo = static_cast<unsigned>(__double2loint(x));
  const unsigned long long m = (static_cast<unsigned long long>((hi & 0xfffffu) | 0x100000u) << 32) | lo;
  const unsigned sh = (em - (hi & 0x7ff00000u)) >> 20;
  unsigned long long q;
  asm("shr.b64 %0, %1, %2;" : "=l"(q) : "l"(m), "r"(sh));  // amounts above 64 clamp to 64: 0
  a.ones += static_cast<long long>(q) ^ static_cast<long long>(static_cast<int>(hi) >> 31);
  a.neg += static_cast<int>(hi >> 31);
}

// n 2^(E - 1075) rounded once to FP64 (n = 0, or E in [55, 1523] and |n| < 2^62: a normal
// result, no overflow)
__device__ __forceinline__ double fix_value(long long n, unsigned em) {
  if (n == 0) return 0.0;
  const double d = __ll2double_rn(n);
  return __hiloint2double(__double2hiint(d) + ((static_cast<int>(em >> 20) - 1075) << 20), __double2loint(d));
}

// largest exponent field among a node's stencil inputs of one field: the centre and its
// axis neighbours at distance 1..R
template <int SY, int SZ, int R>
__device__ __forceinline__ unsigned fix_emax(const double* T, int c0) {
  unsigned e = fix_expbits(T + c0);
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    e = max(e, max(fix_expbits(T + c0 - m), fix_expbits(T + c0 + m)));
    e = max(e, max(fix_expbits(T + c0 - m * SY), fix_expbits(T + c0 + m * SY)));
    e = max(e, max(fix_expbits(T + c0 - m * SZ), fix_expbits(T + c0 + m * SZ)));
  }
  return e;
}

// the symmetric pair sums at distance m along the three axes, on the grid of em
template <int SY, int SZ>
__device__ __forceinline__ long long fix_ring(const double* T, int c0, int m, unsigned em) {
  FixSum a;
  fix_add(a, T[c0 - m], em);
  fix_add(a, T[c0 + m], em);
  fix_add(a, T[c0 - m * SY], em);
  fix_add(a, T[c0 + m * SY], em);
  fix_add(a, T[c0 - m * SZ], em);
  fix_add(a, T[c0 + m * SZ], em);
  return a.value();
}

__device__ __forceinline__ long long fix_one(double x, unsigned em) {
  FixSum a;
  fix_add(a, x, em);
  return a.value();
}

// every one of those inputs (distance 1..R) is +-0
template <int SY, int SZ, int R>
__device__ __noinline__ bool fix_all_zero(const double* T, int c0) {
  auto bits = [&](int o) {
    const int* w = reinterpret_cast<const int*>(T + c0 + o);
    return (w[1] & 0x7fffffff) | w[0];
  };
  int any = bits(0);
#pragma unroll
  for (int m = 1; m <= R; ++m) any |= bits(-m) | bits(m) | bits(-m * SY) | bits(m * SY) | bits(-m * SZ) | bits(m * SZ);
  return any == 0;
}

// the grid of the largest exponent field em represents those inputs exactly enough:
// E = em >> 20 in [55, 1523] (subnormal inputs then lie below one grid unit), or every input
// zero
template <int SY, int SZ, int R>
__device__ __forceinline__ bool fix_range(unsigned em, const double* T, int c0) {
  return (em >= (55u << 20) && em <= (1523u << 20)) || (em == 0 && fix_all_zero<SY, SZ, R>(T, c0));
}

// the wave right-hand side (chi, phi) at tile index c0 of the FP64 tiles Tc (chi) and Tp
// (phi): chi's Laplacian and dissipation as exact integer sums, phi's dissipation in FP64
// (the association of the floating-point evaluation); false when chi's inputs are out of the
// exact range (nothing written)
template <int SY, int SZ>
__device__ __forceinline__ bool wave_rhs_exact(const double* Tc, const double* Tp, int c0, double kos,
                                               double inv12h2, double& kchi, double& kphi) {
  // phi's dissipation first (FP64 pipe), then chi's integer sums
  const double f0v = Tp[c0];
  const double F1 = (Tp[c0 - 1] + Tp[c0 + 1]) + (Tp[c0 - SY] + Tp[c0 + SY]) + (Tp[c0 - SZ] + Tp[c0 + SZ]);
  const double F2 = (Tp[c0 - 2] + Tp[c0 + 2]) + (Tp[c0 - 2 * SY] + Tp[c0 + 2 * SY]) + (Tp[c0 - 2 * SZ] + Tp[c0 + 2 * SZ]);
  const double F3 = (Tp[c0 - 3] + Tp[c0 + 3]) + (Tp[c0 - 3 * SY] + Tp[c0 + 3 * SY]) + (Tp[c0 - 3 * SZ] + Tp[c0 + 3 * SZ]);
  const double kop = fma(-60.0, f0v, fma(15.0, F1, fma(-6.0, F2, F3)));
  const unsigned ec = fix_emax<SY, SZ, 3>(Tc, c0);
  if (!fix_range<SY, SZ, 3>(ec, Tc, c0)) return false;
  long long lap = 0, koc = 0;  // inputs all zero: zero sums
  if (ec != 0) {
    const long long c = fix_one(Tc[c0], ec);
    const long long c1 = fix_ring<SY, SZ>(Tc, c0, 1, ec);
    const long long c2 = fix_ring<SY, SZ>(Tc, c0, 2, ec);
    lap = 16 * c1 - c2 - 90 * c;
    koc = fix_ring<SY, SZ>(Tc, c0, 3, ec) - 6 * c2 + 15 * c1 - 60 * c;
  }
  kchi = fma(kos, fix_value(koc, ec), f0v);
  kphi = fma(kos, kop, fix_value(lap, ec) * inv12h2);
  return true;
}

// right-hand side at one node from its padded tile: advection (4th-order D1) or the
// wave equation (4th-order Laplacian), plus Kreiss-Oliger dissipation; symmetric pair
// sums at distance 1, 2, 3 are shared by the derivative and the dissipation
template <int NF, typename R, int SY, int SZ>
__device__ __forceinline__ void rhs_node(const R* const* Tt, int c0, const StageArgs& A, R kos, R inv12h, R inv12h2,
                                         R kv[NF]) {
  if (A.pde == LTS_PDE_ADVECTION) {
    const R* T = Tt[0];
    const R uc = T[c0];
    const R P1 = (T[c0 - 1] + T[c0 + 1]) + (T[c0 - SY] + T[c0 + SY]) + (T[c0 - SZ] + T[c0 + SZ]);
    const R P2 = (T[c0 - 2] + T[c0 + 2]) + (T[c0 - 2 * SY] + T[c0 + 2 * SY]) + (T[c0 - 2 * SZ] + T[c0 + 2 * SZ]);
    const R P3 = (T[c0 - 3] + T[c0 + 3]) + (T[c0 - 3 * SY] + T[c0 + 3 * SY]) + (T[c0 - 3 * SZ] + T[c0 + 3 * SZ]);
    R av[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) av[d] = sizeof(R) == sizeof(double) ? R(A.adv[d]) : R(A.cf.adv[d]);
    R d1s = av[0] * fma(R(8), T[c0 + 1] - T[c0 - 1], T[c0 - 2] - T[c0 + 2]);
    d1s = fma(av[1], fma(R(8), T[c0 + SY] - T[c0 - SY], T[c0 - 2 * SY] - T[c0 + 2 * SY]), d1s);
    d1s = fma(av[2], fma(R(8), T[c0 + SZ] - T[c0 - SZ], T[c0 - 2 * SZ] - T[c0 + 2 * SZ]), d1s);
    const R ko = fma(R(-60), uc, fma(R(15), P1, fma(R(-6), P2, P3)));
    kv[0] = fma(kos, ko, -inv12h * d1s);
  } else {
    const R* Tc = Tt[0];
    const R* Tp = Tt[NF - 1];
    if constexpr (sizeof(R) == sizeof(double) && NF == 2) {
      if (wave_rhs_exact<SY, SZ>(Tc, Tp, c0, kos, inv12h2, kv[0], kv[1])) return;
    }
    const R c0v = Tc[c0], f0v = Tp[c0];
    const R C1 = (Tc[c0 - 1] + Tc[c0 + 1]) + (Tc[c0 - SY] + Tc[c0 + SY]) + (Tc[c0 - SZ] + Tc[c0 + SZ]);
    const R C2 = (Tc[c0 - 2] + Tc[c0 + 2]) + (Tc[c0 - 2 * SY] + Tc[c0 + 2 * SY]) + (Tc[c0 - 2 * SZ] + Tc[c0 + 2 * SZ]);
    const R C3 = (Tc[c0 - 3] + Tc[c0 + 3]) + (Tc[c0 - 3 * SY] + Tc[c0 + 3 * SY]) + (Tc[c0 - 3 * SZ] + Tc[c0 + 3 * SZ]);
    const R F1 = (Tp[c0 - 1] + Tp[c0 + 1]) + (Tp[c0 - SY] + Tp[c0 + SY]) + (Tp[c0 - SZ] + Tp[c0 + SZ]);
    const R F2 = (Tp[c0 - 2] + Tp[c0 + 2]) + (Tp[c0 - 2 * SY] + Tp[c0 + 2 * SY]) + (Tp[c0 - 2 * SZ] + Tp[c0 + 2 * SZ]);
    const R F3 = (Tp[c0 - 3] + Tp[c0 + 3]) + (Tp[c0 - 3 * SY] + Tp[c0 + 3 * SY]) + (Tp[c0 - 3 * SZ] + Tp[c0 + 3 * SZ]);
    const R lap = fma(R(-90), c0v, fma(R(16), C1, -C2)) * inv12h2;
    const R koc = fma(R(-60), c0v, fma(R(15), C1, fma(R(-6), C2, C3)));
    const R kop = fma(R(-60), f0v, fma(R(15), F1, fma(R(-6), F2, F3)));
    kv[0] = fma(kos, koc, f0v);
    kv[NF - 1] = fma(kos, kop, lap);
  }
}

// the state as stage input array: FP64 u, or in mixed precision its FP32 copy
template <typename R>
__device__ __forceinline__ const R* state_array(const double* u, const float* us) {
  if constexpr (sizeof(R) == sizeof(double)) {
    return u;
  } else {
    return us;
  }
}

// asynchronous global -> shared copy of one element (cp.async, sm_80+): the gathers of a
// tile go out without staging in registers, and the FP64 correction pass overlaps them
template <typename R>
__device__ __forceinline__ void async_copy(R* smem, const R* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if constexpr (sizeof(R) == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  }
}

__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Stage epilogue of one node-field (o its index in the field arrays): the next stage's
// input u + dt sum_j a[s+1][j] k_j, or after the last stage the new state
// u + dt sum_j w_j k_j, with the products dt a[s+1][j] and dt w_j of the octant's level
// formed on the host (StageArgs::dtw).  FP64: all in FP64, one FMA per term.  Mixed: the
// stage input in FP32 from the FP32 copy of u; the new state accumulates the FP32
// increment sum_j (dt w_j) k_j into FP64 u (and refreshes the FP32 copy).
struct EpilogueOut {
  double unew;
  double uin_d;
  float unew_s;
  float uin_f;
};

template <typename R>
__device__ __forceinline__ EpilogueOut stage_epilogue(const StageArgs& A, const R* K, long long kstride, long long o,
                                                      R kvf, const double* u0, const float* us0, int lb, int s,
                                                      int p) {
  EpilogueOut out{0.0, 0.0, 0.0f, 0.0f};
  if constexpr (sizeof(R) == sizeof(double)) {
    const double kd = kvf;
    if (s < p - 1) {
      double v = u0[o];
      for (int q = 0; q < A.next.n; ++q)
        v = fma(A.dtw.next[lb][q],
                A.next.j[q] == s ? kd : static_cast<double>(K[(long long)A.next.j[q] * kstride + o]), v);
      out.uin_d = v;
    } else if (A.write_update) {
      double v = u0[o];
      for (int q = 0; q < p - 1; ++q) v = fma(A.dtw.upd[lb][q], static_cast<double>(K[(long long)q * kstride + o]), v);
      out.unew = fma(A.dtw.upd[lb][p - 1], kd, v);
    }
  } else {
    if (s < p - 1) {
      float v = us0[o];
      for (int q = 0; q < A.next.n; ++q)
        v = fmaf(A.cf.dtw_next[lb][q], A.next.j[q] == s ? float(kvf) : float(K[(long long)A.next.j[q] * kstride + o]),
                 v);
      out.uin_f = v;
    } else if (A.write_update) {
      float acc = 0.0f;
      for (int q = 0; q < p - 1; ++q) acc = fmaf(A.cf.dtw_upd[lb][q], float(K[(long long)q * kstride + o]), acc);
      acc = fmaf(A.cf.dtw_upd[lb][p - 1], float(kvf), acc);
      out.unew = u0[o] + widen(acc);
      out.unew_s = static_cast<float>(out.unew);
    }
  }
  return out;
}

// source terms of phi_t at one node: -c sin(2 chi)/r^2 (eq. phi, 0 at r = 0) and the
// two orbiting Gaussians centred at +-(cx, cy, 0), cx + i cy = R e^{i W t_s}
template <typename R>
__device__ __noinline__ R wave_source(const StageArgs& A, const int P6[3], R chi, R ax, R ay) {
  constexpr bool f64 = sizeof(R) == sizeof(double);
  R x, y, z;
  if constexpr (f64) {
    x = lattice_to_x(A.lo, A.ext, P6[0]);
    y = lattice_to_x(A.lo, A.ext, P6[1]);
    z = lattice_to_x(A.lo, A.ext, P6[2]);
  } else {
    x = fmaf(A.cf.xscale, float(P6[0]), A.cf.lo);
    y = fmaf(A.cf.xscale, float(P6[1]), A.cf.lo);
    z = fmaf(A.cf.xscale, float(P6[2]), A.cf.lo);
  }
  const R nl_c = f64 ? R(A.nl_c) : R(A.cf.nl_c);
  R src = 0;
  if (nl_c != R(0)) {
    const R r2 = x * x + y * y + z * z;
    if (r2 > R(0)) src = -nl_c * sin(R(2) * chi) / r2;
  }
  if (A.orbit) {
    const R inv_w = R(1) / (f64 ? R(A.orb[2]) : R(A.cf.orb[2]));
    const R d1 = (x - ax) * (x - ax) + (y - ay) * (y - ay) + z * z;
    const R d2 = (x + ax) * (x + ax) + (y + ay) * (y + ay) + z * z;
    src += (f64 ? R(A.orb[3]) : R(A.cf.orb[3])) * (exp(-d1 * inv_w) + exp(-d2 * inv_w));
  }
  return src;
}

// the octant of work item `it` of a stage launch
__device__ __forceinline__ int stage_item(const StageArgs& A, int it) {
  return A.list ? __ldg(A.list + A.first + it) : A.first + it;
}

// padding-map bytes of this thread's points of octant b (TileColumn), four to a register
constexpr int kSlw = (kPer + 3) / 4;
struct Slots {
  unsigned w[kSlw];
  __device__ __forceinline__ unsigned operator[](int r) const { return (w[r >> 2] >> (8 * (r & 3))) & 255u; }
};

template <int TPB>
__device__ __forceinline__ void load_slots(const StageArgs& A, int b, Slots& sl) {
  static_assert(TPB >= 338, "TileColumn needs 338 threads");
  const unsigned char* __restrict__ pm = A.padmap + (long long)b * kNT;
  const TileColumn tc(threadIdx.x);
#pragma unroll
  for (int i = 0; i < kSlw; ++i) sl.w[i] = 0u;
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int q = r < tc.n ? tc.q0 + 169 * r : kNT;
    const unsigned v = q < kNT ? unsigned(__ldg(pm + q)) : kSlotNone;
    sl.w[r >> 2] |= v << (8 * (r & 3));
  }
}

// One RK stage of an octant (Alg. 2 compute_stage, or Alg. 1 when A.gts), in three
// phases over a tile buffer of the CTA:
//   stage_slots    the octant's neighbour view: kind and base of every slot (the plan's
//                  slot map)
//   stage_gather   the padded tile (Sec. 3.3, Fig. unzip): asynchronous copies of the
//                  sources' stage inputs (coarser sources: their prolonged inputs; finer
//                  sources: their injected inputs)
//   stage_compute  physical boundary, right-hand side, RK stage and update
// Between the phases the caller synchronises (stage_octant).

// Per slot of octant b's neighbour view, base << 2 | kind (slotmap_kernel).  No barrier
// inside.
template <int NF, typename R, int NB>
__device__ __forceinline__ void stage_slots(StageSmem<NF, R, NB>& S, int nb, const StageArgs& A, int b) {
  const int* __restrict__ row = A.slotmap + (long long)b * kSlots;
  for (int t = threadIdx.x; t < kSlots; t += blockDim.x) S.slot[nb][t] = __ldg(row + t);
}

// The slot map of one octant (once per plan): for each slot of its neighbour view, the
// kind of its leaf (same level, coarser, finer, none) and the base offset of the array
// the stage kernel reads it from (the numberings above kPer): the stage inputs (same level), the
// prolonged inputs of a coarser source (slot up_slot[leaf]), or the injected inputs of a
// finer source (slot dn_slot[leaf]; a finer leaf that no padding map reads has none).
__global__ void __launch_bounds__(256) slotmap_kernel(const DevTree T, const int* __restrict__ up_slot,
                                                      const int* __restrict__ dn_slot, int nf, int* __restrict__ out,
                                                      int* err) {
  for (int b = blockIdx.x; b < T.n; b += gridDim.x) {
    const int4 me = T.oct[b];
    const int lb = me.w;
    const int sh = kDepth - lb;  // log2 of the octant's edge
    for (int t = threadIdx.x; t < kSlots; t += blockDim.x) {
      int kind = kKindNone;
      long long base = 0;
      if (t == 13) {
        kind = kKindSame;
        base = (long long)b * kNV;
      } else if (t < 27) {
        // the leaf covering the same-size box in direction d = t (same level or coarser),
        // < 0: outside the domain, or a box with children
        const int leaf = T.nbr[(long long)b * 27 + t];
        if (leaf >= 0) {
          const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
          const int4 so = T.oct[leaf];
          if (so.w == lb) {
            kind = kKindSame;
            base = (long long)leaf * kNV - 6 * (dx + 7 * dy + 49 * dz);
          } else if (so.w == lb - 1) {
            const int us = up_slot[leaf];
            if (us >= 0) {
              kind = kKindCoarser;
              const int mx = (me.x - so.x) >> sh, my = (me.y - so.y) >> sh, mz = (me.z - so.z) >> sh;
              base = (long long)us * nf * kNT - 549 + 6 * (mx + 13 * my + 169 * mz);
            } else {
              atomicOr(err, 2);  // a coarser source without prolonged inputs: never on a valid plan
            }
          }
        }
      } else if (t < 27 + 27 * 8) {  // slots 243..255 hold no leaf
        const int d = (t - 27) >> 3, c = (t - 27) & 7;
        const int e = T.nbr[(long long)b * 27 + d];
        const int leaf = e <= -2 ? T.fine[(long long)(-e - 2) * 8 + c] : -1;
        if (leaf >= 0) {
          // dn_slot < 0: no padding map reads this leaf (nor this octant's), the slot stays unused
          const int ds = dn_slot[leaf];
          if (ds >= 0) {
            const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
            const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
            kind = kKindFiner;
            base = (long long)ds * nf * 64 - ((6 * dx + 3 * cx) + 4 * (6 * dy + 3 * cy) + 16 * (6 * dz + 3 * cz));
          }
        }
      }
      out[(long long)b * kSlots + t] = int(base * 4 + kind);  // |base| < 2^29: checked by the plan
    }
  }
}

// The finer sources of the padding maps: mark[leaf] = 1 for every leaf that some octant's
// padding map takes a point from through a child slot (a finer leaf).  Such a leaf need not
// touch the octant: on the face between two finer siblings the padding rule may pick the
// far one.
__global__ void __launch_bounds__(256) finemark_kernel(const DevTree T, const unsigned char* __restrict__ padmap,
                                                       unsigned char* __restrict__ mark) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)T.n * kNT;
       e += (long long)gridDim.x * blockDim.x) {
    const unsigned slot = padmap[e];
    if (slot < 27u || slot >= kSlotNone) continue;
    const long long b = e / kNT;
    const int d = int(slot - 27u) >> 3, c = int(slot - 27u) & 7;
    const int box = T.nbr[b * 27 + d];
    const int leaf = box <= -2 ? T.fine[(long long)(-box - 2) * 8 + c] : -1;
    if (leaf >= 0) mark[leaf] = 1;
  }
}

cudaError_t launch_finemark(const DevTree& t, const unsigned char* padmap, unsigned char* mark, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  finemark_kernel<<<152 * 16, 256, 0, s>>>(t, padmap, mark);
  return cudaGetLastError();
}

cudaError_t launch_slotmap(const DevTree& t, const int* up_slot, const int* dn_slot, int nf, int* out, int* err,
                           cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  slotmap_kernel<<<t.n < 152 * 8 ? t.n : 152 * 8, 256, 0, s>>>(t, up_slot, dn_slot, nf, out, err);
  return cudaGetLastError();
}

// The tile's gathers into buffer nb: same-level (and own) sources read the stage
// inputs, coarser sources their prolonged stage inputs (prolong_kernel), finer sources
// their injected stage inputs (inject_kernel).  At stage 0 the stage input is the state
// u itself.  Points outside the domain are zeroed (the boundary fill overwrites them).
template <int NF, typename R, int NB, int TPB>
__device__ void stage_gather(StageSmem<NF, R, NB>& S, int nb, const StageArgs& A, int lb,
                             const Slots& sl) {
  const double* u0 = A.u[(A.cur_mask >> lb) & 1];
  const float* us0 = A.us[(A.cur_mask >> lb) & 1];
  const R* st_in = A.stage == 0 ? state_array<R>(u0, us0) : static_cast<const R*>(A.Uin);
  const R* up_all = static_cast<const R*>(A.up);
  const R* inj_all = static_cast<const R*>(A.inj);
  const TileColumn tc(threadIdx.x);
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    if (r >= tc.n) break;
    const int q = tc.q0 + 169 * r;
    const int packed = S.slot[nb][sl[r]];
    const int kind = packed & 3;
    const long long base = packed >> 2;  // + q, lin7 or lin4 by kind
    if (kind == kKindCoarser) {
      const R* up = up_all + (base + q);
#pragma unroll
      for (int f = 0; f < NF; ++f) async_copy(&S.T[nb][f][q], up + f * kNT);
    } else if (kind == kKindSame) {
      const R* src = st_in + (base + tc.l7 + 49 * r);
#pragma unroll
      for (int f = 0; f < NF; ++f) async_copy(&S.T[nb][f][q], src + f * A.fstride);
    } else if (kind == kKindFiner) {
      const R* src = inj_all + (base + tc.l4 + 16 * r);
#pragma unroll
      for (int f = 0; f < NF; ++f) async_copy(&S.T[nb][f][q], src + f * 64);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) S.T[nb][f][q] = 0;
    }
  }
}

// Injection pass (Fig. unzip, fine -> coarse) of one finer source b (every thread of a
// CTA, item slot = its position in the plan's list of octants with a coarser neighbour):
// the stage input at each of its 64 even nodes as a coarser neighbour reads it, under LTS
// u + dt_b sum_j omega[1][s][j] k_j of b's own step (the coarse <- fine correction of
// eq. fc_1, FP64), under GTS the stage input itself.
template <int NF, typename R, bool C = false>
__device__ void inject_octant(const InjectArgs& A, const int b, const int slot) {
  const int ls = A.tree.oct[b].w;
  const int cur = (A.cur_mask >> ls) & 1;
  const long long kstride = (long long)A.nf * A.fstride;
  const R* K = static_cast<const R*>(A.K);
  R* out = static_cast<R*>(A.inj) + (long long)slot * NF * 64;
  for (int t = threadIdx.x; t < NF * 64; t += blockDim.x) {
    const int f = t >> 6, e = t & 63;
    const int node = 2 * (e & 3) + 14 * ((e >> 2) & 3) + 98 * (e >> 4);
    const long long off = (long long)b * kNV + node + f * A.fstride;
    R v;
    if (!A.gts) {
      v = static_cast<R>(corrected_value<R, C>(A.u[cur] + off, K + off, kstride, A.om1, A.lc[ls].dt));
    } else if (A.stage == 0) {
      v = sizeof(R) == sizeof(double) ? R(ld_in<C>(A.u[cur] + off)) : R(ld_in<C>(A.us[cur] + off));
    } else {
      v = ld_in<C>(static_cast<const R*>(A.Uin) + off);
    }
    out[f * 64 + e] = v;
  }
}

template <int NF, typename R>
__global__ void __launch_bounds__(128, 16) inject_kernel(const __grid_constant__ InjectArgs A) {
  for (int item = blockIdx.x; item < A.count; item += gridDim.x)
    inject_octant<NF, R>(A, __ldg(A.list + item), A.first + item);
}

template <int NF, typename R>
static cudaError_t launch_inject_t(const InjectArgs& a, cudaStream_t s) {
  const int grid = a.count < 152 * 16 ? a.count : 152 * 16;
  inject_kernel<NF, R><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_inject(const InjectArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  if (a.nf == 1) return a.mixed ? launch_inject_t<1, float>(a, s) : launch_inject_t<1, double>(a, s);
  return a.mixed ? launch_inject_t<2, float>(a, s) : launch_inject_t<2, double>(a, s);
}

// orbit centre x_1 = R (cos W t_s, sin W t_s, 0) at the stage time t_s = t_b + c_s dt of
// level lb (one thread)
template <typename R>
__device__ __forceinline__ void orbit_centre(const StageArgs& A, int lb, R* out) {
  double c, sn;
  sincos(A.orb[1] * fma(A.c_s, A.lc[lb].dt, A.t_b), &sn, &c);
  out[0] = R(A.orb[0] * c);
  out[1] = R(A.orb[0] * sn);
}

// Physical boundary, right-hand side on the 7^3 interior (stage type R), and the stage,
// next stage input and RK update of every node (stage_epilogue), from the complete tile
// in buffer cb.  Barriers inside are uniform over the CTA.
template <int NF, typename R, int NB, int TPB>
__device__ void stage_compute(StageSmem<NF, R, NB>& S, int cb, const StageArgs& A, const int b, const int4 me) {
  const int tid = threadIdx.x;
  const int p = A.p;
  const int s = A.stage;
  const int lb = me.w;
  const int eb = 1 << (kDepth - lb);
  const long long kstride = (long long)A.nf * A.fstride;
  R* __restrict__ K = static_cast<R*>(A.K);
  const double* u0 = A.u[(A.cur_mask >> lb) & 1];
  const float* us0 = A.us[(A.cur_mask >> lb) & 1];
  R(*T)[kNT] = S.T[cb];

  // physical boundary
  const LevelConst lc = A.lc[lb];
  constexpr int kRoot = 1 << kDepth;
  const bool touches = me.x == 0 || me.y == 0 || me.z == 0 || me.x + eb == kRoot || me.y + eb == kRoot ||
                       me.z + eb == kRoot;
  if (touches) {  // uniform over the CTA
    if (A.bc == LTS_BC_EXACT)
      fill_exact<NF, R>(T, A, me, eb, lc.dt);
    else
      fill_extrapolated<NF, R>(T, me, eb);
    __syncthreads();
  }

  auto rhs_at = [&](int n, R (&kv)[NF]) {
    const int i = n % 7, j = (n / 7) % 7, k = n / 49;
    const int c0 = (i + 3) + 13 * (j + 3) + 169 * (k + 3);
    const R kos = sizeof(R) == sizeof(double) ? R(lc.kos) : R(A.cf.lc[lb][0]);
    const R inv12h = sizeof(R) == sizeof(double) ? R(lc.inv12h) : R(A.cf.lc[lb][1]);
    const R inv12h2 = sizeof(R) == sizeof(double) ? R(lc.inv12h2) : R(A.cf.lc[lb][2]);
    const R* Tt[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) Tt[f] = T[f];
    rhs_node<NF, R, 13, 169>(Tt, c0, A, kos, inv12h, inv12h2, kv);
    if (A.pde != LTS_PDE_ADVECTION) {
      if (A.cf.sources) {
        const int P6[3] = {6 * me.x + i * eb, 6 * me.y + j * eb, 6 * me.z + k * eb};
        kv[NF - 1] += wave_source<R>(A, P6, Tt[0][c0], S.orb[cb][0], S.orb[cb][1]);
      }
      if (A.bc == LTS_BC_RADIATIVE && touches) {
        const int P6[3] = {6 * me.x + i * eb, 6 * me.y + j * eb, 6 * me.z + k * eb};
        const bool on_bnd = P6[0] == 0 || P6[1] == 0 || P6[2] == 0 || P6[0] == kLatt6 || P6[1] == kLatt6 ||
                            P6[2] == kLatt6;
        if (on_bnd) radiative_rhs<NF, R, 13, 169>(Tt, A, c0, P6, inv12h, kv);
      }
    }
  };
  auto finish = [&](int n, const R (&kv)[NF]) {
    const long long node = (long long)b * kNV + n;
    R* Uout = static_cast<R*>(A.Uout);
    const int nx = ((A.cur_mask >> lb) & 1) ^ 1;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long o = f * A.fstride + node;
      K[(long long)s * kstride + o] = kv[f];
      const EpilogueOut e = stage_epilogue<R>(A, K, kstride, o, kv[f], u0, us0, lb, s, p);
      if (s < p - 1) {
        Uout[o] = sizeof(R) == sizeof(double) ? R(e.uin_d) : R(e.uin_f);
      } else if (A.write_update) {
        A.u[nx][o] = e.unew;
        if (sizeof(R) != sizeof(double)) A.us[nx][o] = e.unew_s;
      }
    }
  };
  if constexpr (sizeof(R) == sizeof(double)) {
    // FP64: node order; the FP64 pipe, not shared memory, bounds this kernel
    for (int n = tid; n < kNV; n += TPB) {
      R kv[NF];
      rhs_at(n, kv);
      finish(n, kv);
    }
  } else {
    static_assert(TPB == kThreads, "g_rhs_node is laid out for kThreads threads");
    // FP32: right-hand sides in the bank-conflict-free order of g_rhs_node, staged in
    // shared memory, then the epilogue in node order (coalesced stores)
    const int n = g_rhs_node[tid];
    if (n >= 0) {
      R kv[NF];
      rhs_at(n, kv);
#pragma unroll
      for (int f = 0; f < NF; ++f) S.KV[f][n] = kv[f];
    }
    __syncthreads();
    for (int m = tid; m < kNV; m += TPB) {
      R kv[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) kv[f] = S.KV[f][m];
      finish(m, kv);
    }
  }
}

// One RK stage of octant b by a CTA of TPB threads with one tile buffer (the stage and batch
// kernels): the four phases in sequence.  The caller separates consecutive calls by a
// barrier.
template <int NF, typename R, int TPB = kThreads>
__device__ void stage_octant(StageSmem<NF, R, 1>& S, const StageArgs& A, const int b) {
  const int4 me = __ldg(A.tree.oct + b);
  Slots sl;
  load_slots<TPB>(A, b, sl);
  stage_slots<NF, R, 1>(S, 0, A, b);
  if (threadIdx.x == 0 && A.orbit) orbit_centre<R>(A, me.w, S.orb[0]);
  __syncthreads();
  stage_gather<NF, R, 1, TPB>(S, 0, A, me.w, sl);
  async_wait_all();
  __syncthreads();
  stage_compute<NF, R, 1, TPB>(S, 0, A, b, me);
}

// Threads per CTA and CTAs per SM of the stage kernel: 352 threads (the 343 interior
// nodes in one pass) and 5 CTAs per SM (1,760 of 2,048 threads; 37 KB of shared memory
// each in FP64, 20 KB in mixed precision).  Measured slower: mixed precision with 128
// threads and 10 CTAs per SM (13%); FP64 with 320 threads and 6 CTAs per SM (1%: the
// 23 nodes of a second pass); persistent CTAs stepping their octants with two tile
// buffers, the next octant's gathers in flight during the current one's right-hand sides
// (FP64 25%: 3 CTAs per SM fit; mixed 27%: the slot table's loads stall the whole CTA);
// mixed precision with two octants per CTA, their maps, slot tables and gathers in
// flight together (12%: the second octant's slot registers spill at 32 registers); FP64
// at 4 CTAs per SM with 40 registers, its spills nearly gone (6%).
template <typename R> struct StageShape {
  static constexpr int kTPB = kThreads;
  static constexpr int kMinBlocks = 5;
};

// The stage kernel: CTA x steps octant list[first + x] (or first + x).
template <int NF, typename R>
__global__ void __launch_bounds__(StageShape<R>::kTPB, StageShape<R>::kMinBlocks)
    stage_kernel(const __grid_constant__ StageArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StageSmem<NF, R, 1>& S = *reinterpret_cast<StageSmem<NF, R, 1>*>(smem_raw);
  stage_octant<NF, R, StageShape<R>::kTPB>(S, A, stage_item(A, blockIdx.x));
}

// ---------------------------------------------------------------------------
// Block kernel: one RK stage of a complete sibling group (the 8 children of one
// parent, all leaves of the same level), stepped as one block of 13^3 nodes with a
// 19^3 padded tile (the octree-to-block decomposition of Sec. 3.2.5).  Every padded
// point takes the value the children's own padded tiles would take (the padding
// rule is a property of the point), and shared face nodes of siblings hold equal
// values, so each node is computed once and written to each of its 1, 2, 4 or 8
// octant copies: the results equal those of stage_kernel bit for bit, with 2.5
// instead of 6.4 gathered points and 0.8 instead of 1 right-hand side per node.
// ---------------------------------------------------------------------------
constexpr int kBlockThreads = 448;  // 14 warps: the 2197 block nodes in five passes; 2 CTAs/SM in FP64, 4 in mixed

template <int NF, typename R>
struct BlockSmem {
  R T[NF][kBT];
  StageTerms om[4];
  R orb[2];
  int any_finer;  // some ghost point has a finer source
};

constexpr int kBPer = (kBG + kBlockThreads - 1) / kBlockThreads;  // ghost points per thread
constexpr int kBChunk = 4;  // ghost-map entries loaded together before their copies are issued

// exact boundary data at the exterior points of the block tile (as fill_exact)
template <int NF, typename R>
__device__ __noinline__ void block_fill_exact(BlockSmem<NF, R>& S, const StageArgs& A, int4 me, int eb, double dtb) {
  for (int q = threadIdx.x; q < kBT; q += blockDim.x) {
    const int i = q % kBW - 3, j = (q / kBW) % kBW - 3, k = q / (kBW * kBW) - 3;
    const int P6[3] = {6 * me.x + i * eb, 6 * me.y + j * eb, 6 * me.z + k * eb};
    bool ext = false;
    for (int a = 0; a < 3; ++a) ext = ext || P6[a] < 0 || P6[a] > kLatt6;
    if (!ext) continue;
    const double x[3] = {lattice_to_x(A.lo, A.ext, P6[0]), lattice_to_x(A.lo, A.ext, P6[1]),
                         lattice_to_x(A.lo, A.ext, P6[2])};
    double d[2][5];
    exact_derivs(A.ic, A.icp, A.adv, x, A.t_b, d);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      double v = d[f][0], dtp = 1.0;
      for (int m = 0; m < A.p; ++m) {
        dtp *= dtb;
        v = fma(A.gamma[m] * dtp, d[f][m + 1], v);
      }
      S.T[f][q] = static_cast<R>(v);
    }
  }
}

// cubic extrapolation along the outward normal, x then y then z (as fill_extrapolated)
template <int NF, typename R>
__device__ __noinline__ void block_fill_extrapolated(BlockSmem<NF, R>& S, int4 me, int eb2) {
  const int anchor[3] = {me.x, me.y, me.z};
  constexpr int kRoot = 1 << kDepth;
  constexpr int kLast = 12;  // last node of the block
  for (int a = 0; a < 3; ++a) {
    const bool lo_b = anchor[a] == 0, hi_b = anchor[a] + eb2 == kRoot;
    if (lo_b || hi_b) {
      const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
      const int str = a == 0 ? 1 : (a == 1 ? kBW : kBW * kBW);
      const int str1 = b1 == 0 ? 1 : (b1 == 1 ? kBW : kBW * kBW);
      const int str2 = b2 == 0 ? 1 : (b2 == 1 ? kBW : kBW * kBW);
      for (int t = threadIdx.x; t < kBW * kBW * 3; t += blockDim.x) {
        const int v1 = t % kBW - 3, v2 = (t / kBW) % kBW - 3, m = t / (kBW * kBW) + 1;
        const bool ext1 = (anchor[b1] == 0 && v1 < 0) || (anchor[b1] + eb2 == kRoot && v1 > kLast);
        const bool ext2 = (anchor[b2] == 0 && v2 < 0) || (anchor[b2] + eb2 == kRoot && v2 > kLast);
        if ((b1 > a && ext1) || (b2 > a && ext2)) continue;
        const int base = 3 * str + (v1 + 3) * str1 + (v2 + 3) * str2;  // index 0 along axis a
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (lo_b) {
            R v = 0;
            for (int qq = 0; qq < 4; ++qq) v = fma(R(c_E[m][qq]), S.T[f][base + qq * str], v);
            S.T[f][base - m * str] = v;
          }
          if (hi_b) {
            R v = 0;
            for (int qq = 0; qq < 4; ++qq) v = fma(R(c_E[m][qq]), S.T[f][base + (kLast - qq) * str], v);
            S.T[f][base + (kLast + m) * str] = v;
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int NF, typename R>
__global__ void __launch_bounds__(kBlockThreads, (sizeof(R) == 8 ? 2 : 4))
    block_kernel(const __grid_constant__ StageArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSmem<NF, R>& S = *reinterpret_cast<BlockSmem<NF, R>*>(smem_raw);
  const int tid = threadIdx.x;
  const int g = A.first + blockIdx.x;
  const int b0 = A.grp[g];
  const int p = A.p;
  const int s = A.stage;
  const int4 me = A.tree.oct[b0];  // child 0: its anchor is the parent's
  const int lb = me.w;
  const int eb = 1 << (kDepth - lb);
  const long long kstride = (long long)A.nf * A.fstride;
  R* __restrict__ K = static_cast<R*>(A.K);
  if (tid < 4) S.om[tid] = A.om[tid];
  if (tid == 4) S.any_finer = 0;
  if (tid == 0 && A.orbit) {
    double c, sn;
    sincos(A.orb[1] * fma(A.c_s, A.lc[lb].dt, A.t_b), &sn, &c);
    S.orb[0] = R(A.orb[0] * c);
    S.orb[1] = R(A.orb[0] * sn);
  }
  __syncthreads();  // S.om is read by the correction pass

  // 1a. the block's own 13^3 nodes: the stage inputs of the 8 children (a node shared by
  //     siblings is read from the lowest of them; their copies are equal)
  const int* __restrict__ gs = A.gsrc + (long long)g * kBG;
  const unsigned short* __restrict__ gc = A.gcode + (long long)g * kBG;
  const R* Uin = static_cast<const R*>(A.Uin);
  const double* u0 = A.u[(A.cur_mask >> lb) & 1];
  const float* us0 = A.us[(A.cur_mask >> lb) & 1];
  const R* up_all = static_cast<const R*>(A.up);
  const R* st_in = s == 0 ? state_array<R>(u0, us0) : Uin;
  for (int n = tid; n < 13 * 13 * 13; n += kBlockThreads) {
    const int i = n % 13, j = (n / 13) % 13, k = n / 169;
    const int cx = i > 6, cy = j > 6, cz = k > 6;
    const long long off = (long long)(b0 + cx + 2 * cy + 4 * cz) * kNV + (i - 6 * cx) + 7 * (j - 6 * cy) +
                          49 * (k - 6 * cz);
    const int q = (i + 3) + kBW * (j + 3) + kBW * kBW * (k + 3);
#pragma unroll
    for (int f = 0; f < NF; ++f) async_copy(&S.T[f][q], st_in + f * A.fstride + off);
  }

  // 1b. ghost points (as stage_kernel step 2), their map entries loaded kBChunk at a
  //     time ahead of the copies that depend on them
  for (int r0 = 0; r0 < kBPer; r0 += kBChunk) {
    unsigned cv[kBChunk];
    int sv[kBChunk];
#pragma unroll
    for (int r = 0; r < kBChunk; ++r) {
      const int gi = tid + (r0 + r) * kBlockThreads;
      const bool ok = r0 + r < kBPer && gi < kBG;
      cv[r] = ok ? __ldg(gc + gi) : 0xffffu;
      sv[r] = ok ? __ldg(gs + gi) : -1;
    }
#pragma unroll
    for (int r = 0; r < kBChunk; ++r) {
      const int gi = tid + (r0 + r) * kBlockThreads;
      const unsigned code = cv[r];
      if (code == 0xffffu) continue;  // past the end
      const int q = g_block_ghost[gi];
      if (code & kExterior) {
#pragma unroll
        for (int f = 0; f < NF; ++f) S.T[f][q] = 0;  // the boundary fill overwrites it
        continue;
      }
      const int rx = code & 15, ry = (code >> 4) & 15, rz = (code >> 8) & 15;
      const int rel_code = (code >> 12) & 3;  // 0 coarser, 1 same, 2 finer
      const int src = sv[r];
      if (rel_code == 0) {
        const R* up = up_all + (long long)__ldg(A.up_slot + src) * NF * kNT + rx + 13 * ry + 169 * rz;
#pragma unroll
        for (int f = 0; f < NF; ++f) async_copy(&S.T[f][q], up + f * kNT);
      } else if (rel_code == 1 || A.gts) {
        // under GTS a finer source's stage-0 input is its own level's state (levels may sit in
        // different halves of the double-buffered state after LTS substeps)
        const R* sin = (rel_code == 2 && s == 0)
                           ? state_array<R>(A.u[(A.cur_mask >> (lb + 1)) & 1], A.us[(A.cur_mask >> (lb + 1)) & 1])
                           : st_in;
        const long long off = (long long)src * kNV + (rx >> 1) + 7 * (ry >> 1) + 49 * (rz >> 1);
#pragma unroll
        for (int f = 0; f < NF; ++f) async_copy(&S.T[f][q], sin + f * A.fstride + off);
      } else {
        S.any_finer = 1;
      }
    }
  }
  __syncthreads();  // S.any_finer

  // 2. finer sources with the coarse<-fine correction of eq. fc_1 (FP64)
  if (!A.gts && S.any_finer) {
    for (int gi = tid; gi < kBG; gi += blockDim.x) {
      const unsigned code = __ldg(gc + gi);
      if ((code & kExterior) || ((code >> 12) & 3) != 2) continue;
      const int rx = code & 15, ry = (code >> 4) & 15, rz = (code >> 8) & 15;
      const int ls = lb + 1;
      const double* ub = A.u[(A.cur_mask >> ls) & 1];
      const long long off = (long long)__ldg(gs + gi) * kNV + (rx >> 1) + 7 * (ry >> 1) + 49 * (rz >> 1);
      const int q = g_block_ghost[gi];
#pragma unroll
      for (int f = 0; f < NF; ++f)
        S.T[f][q] = static_cast<R>(corrected_value<R>(ub + f * A.fstride + off, K + f * A.fstride + off, kstride,
                                                      S.om[1], A.lc[ls].dt));
    }
  }
  async_wait_all();
  __syncthreads();

  // 3. physical boundary
  const LevelConst lc = A.lc[lb];
  constexpr int kRoot = 1 << kDepth;
  const int eb2 = 2 * eb;
  const bool touches = me.x == 0 || me.y == 0 || me.z == 0 || me.x + eb2 == kRoot || me.y + eb2 == kRoot ||
                       me.z + eb2 == kRoot;
  if (touches) {  // uniform over the CTA
    if (A.bc == LTS_BC_EXACT)
      block_fill_exact<NF, R>(S, A, me, eb, lc.dt);
    else
      block_fill_extrapolated<NF, R>(S, me, eb2);
    __syncthreads();
  }

  // 4. right-hand side at the 13^3 block nodes; stage, next stage input and RK update
  //    (FP64) written to every octant copy of the node
  const R kos = sizeof(R) == sizeof(double) ? R(lc.kos) : R(A.cf.lc[lb][0]);
  const R inv12h = sizeof(R) == sizeof(double) ? R(lc.inv12h) : R(A.cf.lc[lb][1]);
  const R inv12h2 = sizeof(R) == sizeof(double) ? R(lc.inv12h2) : R(A.cf.lc[lb][2]);
  const R* Tt[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) Tt[f] = S.T[f];
  R* Uout = static_cast<R*>(A.Uout);
  for (int n = tid; n < 13 * 13 * 13; n += kBlockThreads) {
    const int i = n % 13, j = (n / 13) % 13, k = n / 169;
    const int c0 = (i + 3) + kBW * (j + 3) + kBW * kBW * (k + 3);
    R kv[NF];
    rhs_node<NF, R, kBW, kBW * kBW>(Tt, c0, A, kos, inv12h, inv12h2, kv);
    if (A.pde != LTS_PDE_ADVECTION) {
      if (A.cf.sources) {
        const int P6[3] = {6 * me.x + i * eb, 6 * me.y + j * eb, 6 * me.z + k * eb};
        kv[NF - 1] += wave_source<R>(A, P6, Tt[0][c0], S.orb[0], S.orb[1]);
      }
      if (A.bc == LTS_BC_RADIATIVE && touches) {
        const int P6[3] = {6 * me.x + i * eb, 6 * me.y + j * eb, 6 * me.z + k * eb};
        const bool on_bnd = P6[0] == 0 || P6[1] == 0 || P6[2] == 0 || P6[0] == kLatt6 || P6[1] == kLatt6 ||
                            P6[2] == kLatt6;
        if (on_bnd) radiative_rhs<NF, R, kBW, kBW * kBW>(Tt, A, c0, P6, inv12h, kv);
      }
    }
    // octant copies of the node: child c = cx + 2 cy + 4 cz with local node (i - 6 cx, ...);
    // a coordinate of 6 lies on the face shared by children 0 and 1 of that axis
    const int cx0 = i > 6, cx1 = i >= 6, cy0 = j > 6, cy1 = j >= 6, cz0 = k > 6, cz1 = k >= 6;
    const long long own = (long long)(b0 + cx0 + 2 * cy0 + 4 * cz0) * kNV + (i - 6 * cx0) + 7 * (j - 6 * cy0) +
                          49 * (k - 6 * cz0);
    const int nx = ((A.cur_mask >> lb) & 1) ^ 1;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long fo = f * A.fstride;
      const EpilogueOut e = stage_epilogue<R>(A, K, kstride, fo + own, kv[f], u0, us0, lb, s, p);
      const R uout = sizeof(R) == sizeof(double) ? R(e.uin_d) : R(e.uin_f);
      for (int cz = cz0; cz <= cz1; ++cz)
        for (int cy = cy0; cy <= cy1; ++cy)
          for (int cx = cx0; cx <= cx1; ++cx) {
            const long long o = fo + (long long)(b0 + cx + 2 * cy + 4 * cz) * kNV + (i - 6 * cx) + 7 * (j - 6 * cy) +
                                49 * (k - 6 * cz);
            K[(long long)s * kstride + o] = kv[f];
            if (s < p - 1) {
              Uout[o] = uout;
            } else if (A.write_update) {
              A.u[nx][o] = e.unew;
              if (sizeof(R) != sizeof(double)) A.us[nx][o] = e.unew_s;
            }
          }
    }
  }
}

template <int NF, typename R>
static cudaError_t launch_block_t(const StageArgs& a, int count, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(block_kernel<NF, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(BlockSmem<NF, R>));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  block_kernel<NF, R><<<count, kBlockThreads, sizeof(BlockSmem<NF, R>), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_block(const StageArgs& a, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (a.nf == 1) return a.mixed ? launch_block_t<1, float>(a, count, s) : launch_block_t<1, double>(a, count, s);
  return a.mixed ? launch_block_t<2, float>(a, count, s) : launch_block_t<2, double>(a, count, s);
}

// Padding of the ghost points of every sibling group's block tile: a point p in [-3, 15]^3 (child node
// units from the parent's anchor) lies in the padded tile of child c (c_a = 1 iff
// p_a > 6) at local coordinate p - 6 c in [-3, 9]; its source is given by that child's
// padding-map slot, and its code holds its half-node coordinates in the source.
__global__ void __launch_bounds__(256) groupmap_kernel(const DevTree T, const int* __restrict__ grp, int count,
                                                       const unsigned char* __restrict__ padmap, int* __restrict__ gsrc,
                                                       unsigned short* __restrict__ gcode) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)count * kBG;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = int(e / kBG), q = g_block_ghost[e - (long long)g * kBG];
    const int px = q % kBW - 3, py = (q / kBW) % kBW - 3, pz = q / (kBW * kBW) - 3;
    const int cx = px > 6, cy = py > 6, cz = pz > 6;
    const int c = grp[g] + cx + 2 * cy + 4 * cz;
    const int li = px - 6 * cx, lj = py - 6 * cy, lk = pz - 6 * cz;
    const int lq = (li + 3) + 13 * (lj + 3) + 169 * (lk + 3);
    const unsigned slot = padmap[(long long)c * kNT + lq];
    int src = -1;
    if (slot == 13u) {
      src = c;
    } else if (slot < 27u) {
      src = T.nbr[(long long)c * 27 + slot];
    } else if (slot < kSlotNone) {
      const int d = int(slot - 27u) >> 3, ch = int(slot - 27u) & 7;
      const int box = T.nbr[(long long)c * 27 + d];
      src = box <= -2 ? T.fine[(long long)(-box - 2) * 8 + ch] : -1;
    }
    unsigned code = kExterior;
    if (src >= 0) {
      const int4 co = T.oct[c], so = T.oct[src];
      const int ec = 1 << (kDepth - co.w);
      const int rx = half_node(6 * co.x + li * ec, so.x, so.w);
      const int ry = half_node(6 * co.y + lj * ec, so.y, so.w);
      const int rz = half_node(6 * co.z + lk * ec, so.z, so.w);
      const int rel = so.w - co.w + 1;
      code = unsigned(rx) | unsigned(ry) << 4 | unsigned(rz) << 8 | unsigned(rel) << 12;
    }
    gsrc[e] = src;
    gcode[e] = static_cast<unsigned short>(code);
  }
}

cudaError_t launch_groupmap(const DevTree& t, const int* grp, int count, const unsigned char* padmap, int* gsrc,
                            unsigned short* gcode, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  groupmap_kernel<<<152 * 8, 256, 0, s>>>(t, grp, count, padmap, gsrc, gcode);
  return cudaGetLastError();
}

template <int NF, typename R>
static cudaError_t launch_stage_t(const StageArgs& a, int count, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<NF, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(StageSmem<NF, R, 1>));
    if (e != cudaSuccess) return e;
    // all of the unified L1 / shared memory as shared memory: the occupancy above needs it
    e = cudaFuncSetAttribute(stage_kernel<NF, R>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  stage_kernel<NF, R><<<count, StageShape<R>::kTPB, sizeof(StageSmem<NF, R, 1>), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stage(const StageArgs& a, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (a.nf == 1) return a.mixed ? launch_stage_t<1, float>(a, count, s) : launch_stage_t<1, double>(a, count, s);
  return a.mixed ? launch_stage_t<2, float>(a, count, s) : launch_stage_t<2, double>(a, count, s);
}

// ---------------------------------------------------------------------------
// Prolongation of coarser sources (Fig. unzip, coarse -> fine).  One CTA per
// octant with finer neighbours forms its stage inputs as those neighbours see
// them (eqs. fc_1 / fc_2, FP64) and interpolates them, sum-factorised x, then y,
// then z (stage type), to every half-node position of the box its finer
// neighbours read.  Each finer neighbour then gathers these values as copies.
// ---------------------------------------------------------------------------
template <int NF, typename R>
struct ProlongSmem {
  R V[NF][kNV];
  R X1[NF][13 * 49];      // [ra][jc][jb] in the frame of the pass axes a, b, c
  R X2[NF][13 * 13 * 7];  // [ra][rb][jc]
  R E[3][4];              // symmetric-part weights of the mirrored pairs (1, 11), (3, 9), (5, 7)
  R O[3][3];              // antisymmetric-part weights
  R W[6][7];              // Lagrange weights of the odd positions 1, 3, ..., 11 (row k >> 1)
  int Ec[3][4];           // integer pair weights of the exact FP64 lines (interp_line_exact)
  int Oc[3][3];
};


// Division by a divisor fixed per CTA: q = floor(t / d) = umulhi(t, ceil(2^32 / d)), exact
// while t * d < 2^32 (here t < 2 * 2197 and d <= 2 * 2197).
struct FastDiv {
  unsigned d, m;
  __device__ explicit FastDiv(unsigned dv) : d(dv), m(dv > 1u ? 0xffffffffu / dv + 1u : 0u) {}
  __device__ __forceinline__ unsigned div(unsigned t) const { return d > 1u ? __umulhi(t, m) : t; }
};

// class of a half-node coordinate: 0 for [0,3], 1 for [4,8], 2 for [9,12]
__device__ __forceinline__ int half_class(int r) { return r <= 3 ? 0 : (r >= 9 ? 2 : 1); }

// lowest / highest coordinate of the classes in a 3-bit set
__device__ __forceinline__ int class_lo(unsigned m) { return (m & 1u) ? 0 : ((m & 2u) ? 4 : 9); }
__device__ __forceinline__ int class_hi(unsigned m) { return (m & 4u) ? 12 : ((m & 2u) ? 8 : 3); }

// ---------------------------------------------------------------------------
// FP64 prolongation lines by exact integer sums.  With D = 46080 = 2^6 x 720 every Lagrange
// weight of the 7 -> 13 interpolation is an integer over D (c_rj = D W_rj; at odd r,
// c_rj = C(6, j) (-1)^(6 - j) prod_{m != j} (r - 2m)), and sum_j |c_rj| <= 196,470 < 2^17.6.
// A line's 7 values are put on a grid 8 bits below their largest biased exponent E
// (x = floor(M 2^(e - E + 8)), |x| < 2^61: exact for the inputs within 2^8 of the largest,
// each within 2^-60 of the largest), a mirrored pair of odd positions is formed exactly as
// (E' +- O') / 2 from the sums and differences of mirrored values (products of 32-bit halves
// on the FMA pipe, mad.wide; sums below 2^49.4 per half), kept as floor(. / 2^18) < 2^62.3
// and rounded to FP64 with the scale 2^(E - 1065) / (2 D): within a unit of the last place of
// the line's largest weighted term, as the floating-point evaluation, with two FP64
// operations per odd position instead of 5.5.
// Even positions are copies.  Lines whose largest value lies outside [2^-968, 2^876) (other
// than all zero), or is an infinity or NaN, take the floating-point evaluation.
// ---------------------------------------------------------------------------

// x = M 2^(e - 1075) exactly: (M, e) = (0, 0) for +-0, (+-fraction, 1) for subnormal numbers,
// (+-(2^52 + fraction), biased exponent) for normal ones; infinities and NaNs (their bits,
// 2047)
__device__ __forceinline__ long long fix_split(double x, unsigned& e) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned lo = static_cast<unsigned>(__double2loint(x));
  const unsigned eb = (hi >> 20) & 0x7ffu;
  const unsigned fh = hi & 0xfffffu;
  if (eb == 0x7ffu) {
    e = 0x7ffu;
    return __double_as_longlong(x);
  }
  e = eb != 0u ? eb : ((fh | lo) != 0u ? 1u : 0u);
  const long long m =
      static_cast<long long>((static_cast<unsigned long long>(fh | (eb != 0u ? 0x100000u : 0u)) << 32) | lo);
  return static_cast<int>(hi) < 0 ? -m : m;
}

// the exponent fix_split gives x
__device__ __forceinline__ unsigned fix_exp_of(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned eb = (hi >> 20) & 0x7ffu;
  if (eb != 0u) return eb;
  return ((hi & 0xfffffu) | static_cast<unsigned>(__double2loint(x))) != 0u ? 1u : 0u;
}

// floor(m / 2^sh); amounts above 64 clamp to 64 (0 or -1)
__device__ __forceinline__ long long fix_shr(long long m, unsigned sh) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(m), "r"(sh));
  return r;
}

// a * b + c, 32 x 32 -> 64 bits (one FMA-pipe instruction)
__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// floor((h 2^31 + l) / 2^k), 1 <= k <= 31
__device__ __forceinline__ long long hl_shift(long long h, long long l, int k) {
  return h * (1ll << (31 - k)) + (l >> k);  // (a product: h may be negative)
}

// the halves of |v| < 2^62: v = h 2^31 + l, 0 <= l < 2^31
__device__ __forceinline__ int fix_hi(long long v) { return static_cast<int>(v >> 31); }
__device__ __forceinline__ int fix_lo(long long v) { return static_cast<int>(v & 0x7fffffffll); }

// One line of the interpolation as above: the 7 node values v to the half-node positions
// r in [r0, r0 + n) whose class is in cls; put(r, value).  Ec and Oc are the integer pair
// weights (sums and differences of the pair's weights over D, Ec_3 = 2 c_k3).  False, with
// nothing written, for a line out of range.
template <typename Put>
__device__ __forceinline__ bool interp_line_exact(const double (&v)[7], int r0, int n, unsigned cls,
                                                  const int (*Ec)[4], const int (*Oc)[3], Put put) {
  auto needed = [&](int r) { return r >= r0 && r < r0 + n && ((cls >> half_class(r)) & 1u); };
  unsigned em = fix_exp_of(v[0]);
#pragma unroll
  for (int j = 1; j < 7; ++j) em = max(em, fix_exp_of(v[j]));
  if (!(em == 0u || (em >= 55u && em <= 1900u))) return false;
#pragma unroll
  for (int r = 0; r <= 12; r += 2)
    if (needed(r)) put(r, v[r >> 1]);
  long long x[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    unsigned e;
    const long long m = fix_split(v[j], e);
    x[j] = fix_shr(m * 256, em - e);
  }
  const long long s[3] = {x[0] + x[6], x[1] + x[5], x[2] + x[4]};
  const long long d[3] = {x[0] - x[6], x[1] - x[5], x[2] - x[4]};
  // 2^(18 - 8 + E - 1075) / (2 D): a power of two times the rounded 1 / 92160 (exact product)
  const double scale = __hiloint2double((static_cast<int>(em == 0u ? 55u : em) - 42) << 20, 0) * (1.0 / 92160.0);
#pragma unroll
  for (int pr = 0; pr < 3; ++pr) {
    const int kk = 2 * pr + 1;
    const bool nk = needed(kk), nm = needed(12 - kk);
    if (!(nk || nm)) continue;
    long long eh = mad_wide(Ec[pr][3], fix_hi(x[3]), 0), el = mad_wide(Ec[pr][3], fix_lo(x[3]), 0);
    long long oh = 0, ol = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      eh = mad_wide(Ec[pr][j], fix_hi(s[j]), eh);
      el = mad_wide(Ec[pr][j], fix_lo(s[j]), el);
      oh = mad_wide(Oc[pr][j], fix_hi(d[j]), oh);
      ol = mad_wide(Oc[pr][j], fix_lo(d[j]), ol);
    }
    if (nk) put(kk, __ll2double_rn(hl_shift(eh + oh, el + ol, 18)) * scale);
    if (nm) put(12 - kk, __ll2double_rn(hl_shift(eh - oh, el - ol, 18)) * scale);
  }
  return true;
}

// One line of the interpolation: the 7 node values v of a line to the half-node
// positions r in [r0, r0 + n) whose class is in the 3-bit set cls; put(r, value).
// Even positions are nodes (copies).  Odd positions come in mirrored pairs (k, 12 - k):
// the Lagrange weights satisfy W[12 - k][j] = W[k][6 - j], so with s_j = v_j + v_{6-j}
// and d_j = v_j - v_{6-j} the pair is E + O and E - O, E = sum_j E[p][j] s_j (s_3 = v_3)
// and O = sum_j O[p][j] d_j: 9 operations for the pair once the 6 sums and differences
// are formed, against 7 for one position as a direct dot product with W.  The form is
// chosen per pair from the set all (a superset of cls, uniform over the CTA's lines of a
// pass, so that a warp's lines take one path): pairs needed whole take the symmetric form
// when there are at least two of them, every other odd position the direct one; a whole
// line costs 33 operations instead of 42, a one-sided face slab 14 instead of 22.
template <typename R, typename Put>
__device__ __forceinline__ void interp_line(const R (&v)[7], int r0, int n, unsigned cls, unsigned all,
                                            const R (*E)[4], const R (*O)[3], const R (*W)[7], const int (*Ec)[4],
                                            const int (*Oc)[3], Put put) {
  if constexpr (sizeof(R) == sizeof(double)) {
    if (interp_line_exact(v, r0, n, cls, Ec, Oc, put)) return;
  }
  auto in_set = [&](int r, unsigned set) { return r >= r0 && r < r0 + n && ((set >> half_class(r)) & 1u); };
  auto needed = [&](int r) { return in_set(r, cls); };
#pragma unroll
  for (int r = 0; r <= 12; r += 2)
    if (needed(r)) put(r, v[r >> 1]);
  bool pair[3];
  int pairs = 0;
#pragma unroll
  for (int pr = 0; pr < 3; ++pr) {
    pair[pr] = in_set(2 * pr + 1, all) && in_set(11 - 2 * pr, all);
    pairs += pair[pr];
  }
  if (pairs < 2) {
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) pair[pr] = false;
  }
  auto direct = [&](int r) {
    const R* w = W[r >> 1];
    R x = w[0] * v[0];
#pragma unroll
    for (int j = 1; j < 7; ++j) x = fma(w[j], v[j], x);
    put(r, x);
  };
  R s0 = 0, s1 = 0, s2 = 0, d0 = 0, d1 = 0, d2 = 0;
  if (pairs >= 2) {
    s0 = v[0] + v[6], s1 = v[1] + v[5], s2 = v[2] + v[4];
    d0 = v[0] - v[6], d1 = v[1] - v[5], d2 = v[2] - v[4];
  }
#pragma unroll
  for (int pr = 0; pr < 3; ++pr) {
    const int k = 2 * pr + 1;
    const bool nk = needed(k), nm = needed(12 - k);
    if (pair[pr]) {
      if (!(nk || nm)) continue;
      const R e = fma(E[pr][0], s0, fma(E[pr][1], s1, fma(E[pr][2], s2, E[pr][3] * v[3])));
      const R o = fma(O[pr][0], d0, fma(O[pr][1], d1, O[pr][2] * d2));
      if (nk) put(k, e + o);
      if (nm) put(12 - k, e - o);
    } else {
      if (nk) direct(k);
      if (nm) direct(12 - k);
    }
  }
}

// Prolongation of octant b for one stage; called by every thread of a CTA.  The
// passes run along axes a, b, c (a permutation of x, y, z chosen per source on the
// host); V, X1 and X2 hold the source's values in that frame, and only positions
// whose class box is in the source's set (or its projections) are computed.
template <int NF, typename R, bool C = false>
__device__ void prolong_octant(ProlongSmem<NF, R>& S, const ProlongArgs& A, const int b) {
  const int tid = threadIdx.x;
  const int slot = A.up_slot[b];
  const int lb = A.tree.oct[b].w;
  const int rel = A.gts ? 0 : (lb >= A.lstar ? 2 : 3);
  const unsigned word = unsigned(A.box[slot]);
  const unsigned m = word & 0x7ffffffu;  // class mask, bit ca + 3 cb + 9 cc
  const int order = int(word >> 27);
  // pass axes (0 = x, 1 = y, 2 = z) of kProlongOrders[order]
  const int pa = order >> 1, pb = (order == 0 || order == 5) ? 1 : (order == 1 || order == 3) ? 2 : 0;
  const int pc = 3 - pa - pb;
  // node strides 1, 7, 49 and half-node strides 1, 13, 169 of the pass axes
  const int sna = pa == 0 ? 1 : (pa == 1 ? 7 : 49), snb = pb == 0 ? 1 : (pb == 1 ? 7 : 49);
  const int snc = pc == 0 ? 1 : (pc == 1 ? 7 : 49);
  // projections of the set: classes of a, and of (a, b) pairs
  unsigned mab = 0;
  for (int cc = 0; cc < 3; ++cc) mab |= (m >> (9 * cc)) & 0x1ffu;
  const unsigned ma = (mab | mab >> 3 | mab >> 6) & 7u;
  unsigned mb = 0, mc = 0;
  for (int q = 0; q < 9; ++q) {
    if (mab >> q & 1u) mb |= 1u << (q / 3);
  }
  for (int q = 0; q < 27; ++q) {
    if (m >> q & 1u) mc |= 1u << (q / 9);
  }
  const int a0 = class_lo(ma), na = class_hi(ma) - a0 + 1;
  const int b0 = class_lo(mb), nb = class_hi(mb) - b0 + 1;
  const int c0 = class_lo(mc), nc = class_hi(mc) - c0 + 1;
  const long long kstride = (long long)A.nf * A.fstride;
  const R* K = static_cast<const R*>(A.K);
  if (tid < 21) {  // pair weights of the symmetric evaluation (interp_line), from the FP64 table
    const int pr = tid / 7, q = tid % 7, k = 2 * pr + 1;
    if (q < 4) {
      S.E[pr][q] = R(q < 3 ? 0.5 * (c_W[k][q] + c_W[k][6 - q]) : c_W[k][3]);
    } else {
      const int j = q - 4;
      S.O[pr][j] = R(0.5 * (c_W[k][j] - c_W[k][6 - j]));
    }
  } else if (tid >= 32 && tid < 32 + 42) {  // the odd rows for the direct evaluation
    const int q = tid - 32;
    S.W[q / 7][q % 7] = R(c_W[2 * (q / 7) + 1][q % 7]);
  } else if (tid >= 96 && tid < 96 + 21) {  // integer pair weights (46080 W is an integer)
    const int pr = (tid - 96) / 7, q = (tid - 96) % 7, k = 2 * pr + 1;
    if (q < 4) {
      S.Ec[pr][q] = __double2int_rn(46080.0 * (q < 3 ? c_W[k][q] + c_W[k][6 - q] : 2.0 * c_W[k][3]));
    } else {
      const int j = q - 4;
      S.Oc[pr][j] = __double2int_rn(46080.0 * (c_W[k][j] - c_W[k][6 - j]));
    }
  }
  const int cur = (A.cur_mask >> lb) & 1;
  const R* Uin = static_cast<const R*>(A.Uin);
  const double* ub = A.u[cur ^ (rel == 3 ? 1 : 0)];
  for (int t = tid; t < NF * kNV; t += blockDim.x) {
    const int f = t / kNV, n = t - f * kNV;  // n = ja + 7 jb + 49 jc in the pass frame
    const int ja = n % 7, jb = (n / 7) % 7, jc = n / 49;
    const long long off = (long long)b * kNV + ja * sna + jb * snb + jc * snc;
    R v;
    if (rel != 0)
      v = static_cast<R>(corrected_value<R, C>(ub + f * A.fstride + off, K + f * A.fstride + off, kstride, A.om[rel],
                                               A.lc[lb].dt));
    else if (A.stage == 0)
      v = static_cast<R>(ld_in<C>(A.u[cur] + f * A.fstride + off));
    else
      v = ld_in<C>(Uin + f * A.fstride + off);
    S.V[f][n] = v;
  }
  __syncthreads();
  // pass 1 (axis a): one thread per line (f, jb, jc), X1[ra][jb + 7 jc]
  for (int t = tid; t < NF * 49; t += blockDim.x) {
    const int f = t / 49, bc = t - f * 49;
    R v[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] = S.V[f][7 * bc + q];
    R* x1 = S.X1[f] + bc;
    interp_line<R>(v, a0, na, ma, ma, S.E, S.O, S.W, S.Ec, S.Oc, [&](int r, R val) { x1[r * 49] = val; });
  }
  __syncthreads();
  // pass 2 (axis b): one thread per line (f, ra, jc), X2[ra][rb][jc]
  const FastDiv by_a7{unsigned(na * 7)};
  for (int t = tid; t < NF * na * 7; t += blockDim.x) {
    const int f = int(by_a7.div(unsigned(t))), rem = t - f * na * 7;
    const int rai = rem / 7, jc = rem - rai * 7;
    const int ra = a0 + rai, ca = half_class(ra);
    const unsigned cls = ((mab >> ca) & 1u) | ((mab >> (ca + 3)) & 1u) << 1 | ((mab >> (ca + 6)) & 1u) << 2;
    if (!cls) continue;
    R v[7];
    const R* x1 = S.X1[f] + ra * 49 + 7 * jc;  // [jb]
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] = x1[q];
    R* x2 = S.X2[f] + ra * 13 * 7 + jc;
    interp_line<R>(v, b0, nb, cls, mb, S.E, S.O, S.W, S.Ec, S.Oc, [&](int r, R val) { x2[r * 7] = val; });
  }
  __syncthreads();
  // pass 3 (axis c): one thread per line (f, ra, rb), every position of the set written
  // at rx + 13 ry + 169 rz
  R* out = static_cast<R*>(A.up) + (long long)slot * NF * kNT;
  const int soa = pa == 0 ? 1 : (pa == 1 ? 13 : 169), sob = pb == 0 ? 1 : (pb == 1 ? 13 : 169);
  const int soc = pc == 0 ? 1 : (pc == 1 ? 13 : 169);
  const FastDiv by_ab{unsigned(na * nb)}, by_a{unsigned(na)};
  for (int t = tid; t < NF * na * nb; t += blockDim.x) {
    const int f = int(by_ab.div(unsigned(t))), rab = t - f * na * nb;
    const int rbi = int(by_a.div(unsigned(rab))), rai = rab - rbi * na;
    const int ra = a0 + rai, rb = b0 + rbi;
    const unsigned sh = unsigned(half_class(ra) + 3 * half_class(rb));
    const unsigned cls = ((m >> sh) & 1u) | ((m >> (sh + 9)) & 1u) << 1 | ((m >> (sh + 18)) & 1u) << 2;
    if (!cls) continue;
    R v[7];
    const R* x2 = S.X2[f] + (ra * 13 + rb) * 7;  // [jc]
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] = x2[q];
    R* o = out + f * kNT + ra * soa + rb * sob;
    interp_line<R>(v, c0, nc, cls, mc, S.E, S.O, S.W, S.Ec, S.Oc, [&](int r, R val) { o[r * soc] = val; });
  }
}

template <int NF, typename R>
__global__ void __launch_bounds__(256, 6) prolong_kernel(const __grid_constant__ ProlongArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ProlongSmem<NF, R>& S = *reinterpret_cast<ProlongSmem<NF, R>*>(smem_raw);
  prolong_octant<NF, R>(S, A, A.list[blockIdx.x]);
}

template <int NF, typename R>
static cudaError_t launch_prolong_t(const ProlongArgs& a, cudaStream_t s) {
  prolong_kernel<NF, R><<<a.count, 256, sizeof(ProlongSmem<NF, R>), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const ProlongArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  if (a.nf == 1) return a.mixed ? launch_prolong_t<1, float>(a, s) : launch_prolong_t<1, double>(a, s);
  return a.mixed ? launch_prolong_t<2, float>(a, s) : launch_prolong_t<2, double>(a, s);
}

// ---------------------------------------------------------------------------
// GTS step update (Alg. 1 compute_step) from the synchronised stages, FP64
// ---------------------------------------------------------------------------
template <typename R>
__global__ void update_kernel(UpdateArgs A) {
  const long long total = (long long)A.nf * A.fstride;
  const long long kstride = (long long)A.nf * A.fstride;
  const R* K = static_cast<const R*>(A.K);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long inf = e % A.fstride;
    const int b = int(inf / kNV);
    const int cur = (A.cur_mask >> A.oct[b].w) & 1;
    // as the stage epilogue (the same products dt w_j, the same order), so that GTS on a
    // one-level tree equals LTS bit for bit
    if constexpr (sizeof(R) == sizeof(double)) {
      double v = A.u[cur][e];
      for (int q = 0; q < A.p; ++q) v = fma(A.dtw[q], static_cast<double>(K[q * kstride + e]), v);
      A.u[cur ^ 1][e] = v;
    } else {
      // FP32 increment accumulated into FP64 u
      float acc = 0.0f;
      for (int q = 0; q < A.p; ++q) acc = fmaf(A.dtwf[q], float(K[q * kstride + e]), acc);
      const double un = A.u[cur][e] + widen(acc);
      A.u[cur ^ 1][e] = un;
      A.us[cur ^ 1][e] = static_cast<float>(un);
    }
  }
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  const long long total = (long long)a.nf * a.fstride;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (a.mixed)
    update_kernel<float><<<(int)blocks, threads, 0, s>>>(a);
  else
    update_kernel<double><<<(int)blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-node synchronisation (zip + unzip, Fig. dg_to_cg), in place
// ---------------------------------------------------------------------------
struct SyncSmem {
  NbrView nv;
  double W[13][7];  // interpolation weights (divergent row indices: shared, not constant memory)
};

__device__ __forceinline__ bool is_boundary_node(int i, int j, int k) {
  return i == 0 || i == 6 || j == 0 || j == 6 || k == 0 || k == 6;
}

// zip: every non-hanging node takes its owner's value (owners keep theirs)
template <typename T>
__device__ void sync_zip_octant(SyncSmem& S, const SyncArgs& A, const int b) {
  load_neighbours(A.tree, b, S.nv);
  __syncthreads();
  const int4 me = A.tree.oct[b];
  const int eb = 1 << (kDepth - me.w);
  for (int n = threadIdx.x; n < kNV; n += blockDim.x) {
    const int i = n % 7, j = (n / 7) % 7, k = n / 49;
    if (!is_boundary_node(i, j, k)) continue;
    const int src = resolve_source(S.nv, i, j, k, b, true);
    if (src == b) continue;
    const int4 so = A.tree.oct[src];
    const int rx = half_node(6 * me.x + i * eb, so.x, so.w);
    const int ry = half_node(6 * me.y + j * eb, so.y, so.w);
    const int rz = half_node(6 * me.z + k * eb, so.z, so.w);
    if (unsigned(rx) > 12u || unsigned(ry) > 12u || unsigned(rz) > 12u) {
      atomicOr(A.err, 1);
      continue;
    }
    if ((rx | ry | rz) & 1) continue;
    const T* vs = static_cast<const T*>(A.vb[(A.sel_mask >> so.w) & 1]);
    T* vd = static_cast<T*>(A.vb[(A.sel_mask >> me.w) & 1]);
    float* sd = A.shadow[(A.sel_mask >> me.w) & 1];
    for (int f = 0; f < A.nf; ++f) {
      const T v = vs[f * A.fstride + (long long)src * kNV + (rx >> 1) + 7 * (ry >> 1) + 49 * (rz >> 1)];
      vd[f * A.fstride + (long long)b * kNV + n] = v;
      if (sd) sd[f * A.fstride + (long long)b * kNV + n] = static_cast<float>(v);
    }
  }
}

// unzip of hanging nodes of the listed octants (all of one level, whose coarser
// sources are final)
template <typename T>
__device__ void sync_hanging_octant(SyncSmem& S, const SyncArgs& A, const int b) {
  load_neighbours(A.tree, b, S.nv);
  for (int q = threadIdx.x; q < 91; q += blockDim.x) S.W[q / 7][q % 7] = c_W[q / 7][q % 7];
  __syncthreads();
  const int4 me = A.tree.oct[b];
  const int eb = 1 << (kDepth - me.w);
  for (int n = threadIdx.x; n < kNV; n += blockDim.x) {
    const int i = n % 7, j = (n / 7) % 7, k = n / 49;
    if (!is_boundary_node(i, j, k)) continue;
    const int src = resolve_source(S.nv, i, j, k, b, true);
    if (src == b) continue;
    const int4 so = A.tree.oct[src];
    const int rx = half_node(6 * me.x + i * eb, so.x, so.w);
    const int ry = half_node(6 * me.y + j * eb, so.y, so.w);
    const int rz = half_node(6 * me.z + k * eb, so.z, so.w);
    if (unsigned(rx) > 12u || unsigned(ry) > 12u || unsigned(rz) > 12u) {
      atomicOr(A.err, 1);
      continue;
    }
    if (!((rx | ry | rz) & 1)) continue;
    const T* vs = static_cast<const T*>(A.vb[(A.sel_mask >> so.w) & 1]);
    T* vd = static_cast<T*>(A.vb[(A.sel_mask >> me.w) & 1]);
    float* sd = A.shadow[(A.sel_mask >> me.w) & 1];
    for (int f = 0; f < A.nf; ++f) {
      const T v = interp_tensor<T>(vs + f * A.fstride + (long long)src * kNV, S.W, rx, ry, rz);
      vd[f * A.fstride + (long long)b * kNV + n] = v;
      if (sd) sd[f * A.fstride + (long long)b * kNV + n] = static_cast<float>(v);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128) sync_zip_kernel(const __grid_constant__ SyncArgs A) {
  __shared__ SyncSmem S;
  sync_zip_octant<T>(S, A, A.list ? A.list[blockIdx.x] : blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(128) sync_hanging_kernel(const __grid_constant__ SyncArgs A) {
  __shared__ SyncSmem S;
  sync_hanging_octant<T>(S, A, A.list[blockIdx.x]);
}

// The same two passes from the plan's compact node maps (built once from nodemap_kernel's
// output): one thread per copied or hanging node, so every lane of a warp does work.
template <typename T>
__global__ void __launch_bounds__(256) zipmap_kernel(const __grid_constant__ SyncArgs A) {
  for (long long e = A.map_first + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < A.map_first + A.map_count;
       e += (long long)gridDim.x * blockDim.x) {
    const int dst = __ldg(A.map_dst + e), src = __ldg(A.map_src + e);
    const int ld = A.tree.oct[dst / kNV].w, ls = A.tree.oct[src / kNV].w;
    const T* vs = static_cast<const T*>(A.vb[(A.sel_mask >> ls) & 1]);
    T* vd = static_cast<T*>(A.vb[(A.sel_mask >> ld) & 1]);
    float* sd = A.shadow[(A.sel_mask >> ld) & 1];
    for (int f = 0; f < A.nf; ++f) {
      const T v = vs[f * A.fstride + src];
      vd[f * A.fstride + dst] = v;
      if (sd) sd[f * A.fstride + dst] = static_cast<float>(v);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) hangmap_kernel(const __grid_constant__ SyncArgs A) {
  // the interpolation weights in shared memory: threads of a warp index different rows,
  // which the constant cache would serialise
  __shared__ double W[13][7];
  for (int q = threadIdx.x; q < 91; q += blockDim.x) W[q / 7][q % 7] = c_W[q / 7][q % 7];
  __syncthreads();
  for (long long e = A.map_first + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < A.map_first + A.map_count;
       e += (long long)gridDim.x * blockDim.x) {
    const int dst = __ldg(A.map_dst + e), src = __ldg(A.map_src + e);
    const unsigned code = __ldg(A.map_code + e);
    const int ld = A.tree.oct[dst / kNV].w, ls = A.tree.oct[src].w;
    const T* vs = static_cast<const T*>(A.vb[(A.sel_mask >> ls) & 1]);
    T* vd = static_cast<T*>(A.vb[(A.sel_mask >> ld) & 1]);
    float* sd = A.shadow[(A.sel_mask >> ld) & 1];
    const int rx = code & 15, ry = (code >> 4) & 15, rz = (code >> 8) & 15;
    for (int f = 0; f < A.nf; ++f) {
      const T v = interp_tensor<T>(vs + f * A.fstride + (long long)src * kNV, W, rx, ry, rz);
      vd[f * A.fstride + dst] = v;
      if (sd) sd[f * A.fstride + dst] = static_cast<float>(v);
    }
  }
}

static int map_blocks(long long work) {
  long long b = (work + 255) / 256;
  return int(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_sync_zip(const SyncArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  if (a.map_dst) {
    if (a.map_count <= 0) return cudaSuccess;
    const int nb = map_blocks(a.map_count);
    if (a.elem == 4)
      zipmap_kernel<float><<<nb, 256, 0, s>>>(a);
    else
      zipmap_kernel<double><<<nb, 256, 0, s>>>(a);
  } else if (a.elem == 4) {
    sync_zip_kernel<float><<<a.count, 128, 0, s>>>(a);
  } else {
    sync_zip_kernel<double><<<a.count, 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_sync_hanging(const SyncArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  if (a.map_dst) {
    if (a.map_count <= 0) return cudaSuccess;
    const int nb = map_blocks(a.map_count);
    if (a.elem == 4)
      hangmap_kernel<float><<<nb, 256, 0, s>>>(a);
    else
      hangmap_kernel<double><<<nb, 256, 0, s>>>(a);
  } else if (a.elem == 4) {
    sync_hanging_kernel<float><<<a.count, 128, 0, s>>>(a);
  } else {
    sync_hanging_kernel<double><<<a.count, 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Node maps of a plan: for every boundary node of every octant, its owner (the coarsest
// octant having the node, ties to the smallest Morton key, the octant itself included)
// and whether it is a copy (all half-node coordinates even) or a hanging node to
// interpolate.
__global__ void __launch_bounds__(128) nodemap_kernel(const DevTree T, const int* __restrict__ hang_pos,
                                                       int* __restrict__ zipmap, int* __restrict__ hang_src,
                                                       unsigned short* __restrict__ hang_code, int* err) {
  __shared__ NbrView nv;
  for (int b = blockIdx.x; b < T.n; b += gridDim.x) {
    __syncthreads();
    load_neighbours(T, b, nv);
    __syncthreads();
    const int4 me = T.oct[b];
    const int eb = 1 << (kDepth - me.w);
    const int hp = hang_pos[b];
    for (int k = threadIdx.x; k < kBN; k += blockDim.x) {
      const int n = g_bnode[k];
      const int i = n % 7, j = (n / 7) % 7, kk = n / 49;
      int zsrc = -1, hsrc = -1;
      unsigned code = 0;
      const int src = resolve_source(nv, i, j, kk, b, true);
      if (src != b && src >= 0) {
        const int4 so = T.oct[src];
        const int rx = half_node(6 * me.x + i * eb, so.x, so.w);
        const int ry = half_node(6 * me.y + j * eb, so.y, so.w);
        const int rz = half_node(6 * me.z + kk * eb, so.z, so.w);
        if (unsigned(rx) > 12u || unsigned(ry) > 12u || unsigned(rz) > 12u) {
          atomicOr(err, 1);
        } else if (!((rx | ry | rz) & 1)) {
          zsrc = src * kNV + (rx >> 1) + 7 * (ry >> 1) + 49 * (rz >> 1);
        } else if (hp >= 0) {
          hsrc = src;
          code = unsigned(rx) | unsigned(ry) << 4 | unsigned(rz) << 8;
        } else {
          atomicOr(err, 2);  // a hanging node outside the hanging list: never on a balanced tree
        }
      }
      zipmap[(long long)b * kBN + k] = zsrc;
      if (hp >= 0) {
        hang_src[(long long)hp * kBN + k] = hsrc;
        hang_code[(long long)hp * kBN + k] = static_cast<unsigned short>(code);
      }
    }
  }
}

cudaError_t launch_nodemap(const DevTree& t, const int* hang_pos, int* zipmap, int* hang_src,
                           unsigned short* hang_code, int* err, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  nodemap_kernel<<<t.n < 152 * 8 ? t.n : 152 * 8, 128, 0, s>>>(t, hang_pos, zipmap, hang_src, hang_code, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batches (many instances advanced together).  A round advances every instance
// with substeps left by one substep of its own schedule (Fig. blk_loop): one
// persistent launch per stage covers the active octants of all instances.
// ---------------------------------------------------------------------------
template <bool C = false>
__device__ __forceinline__ int batch_find(const int* pre, int n, int item) {
  // largest i with pre[i] <= item (pre is non-decreasing, pre[0] = 0)
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ld_in<C>(pre + mid) <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Start of a round (one CTA): each instance's active level l* and argument blocks for
// this substep, prefix sums of the work items over instances, work counters zeroed.
__device__ void round_begin_body(const BatchArgs& B) {
  for (int i = threadIdx.x; i < B.n; i += blockDim.x) {
    BatchInst& I = B.inst[i];
    I.reconcile = 0;
    I.active = I.remaining > 0;
    int lstar = I.lmax;
    for (int l = I.lmin; l <= I.lmax; ++l)
      if (I.n_sub % (1ll << (I.lmax - l)) == 0) {
        lstar = l;
        break;
      }
    I.lstar = lstar;
    const double t_b = I.t_macro + double(I.n_sub) * I.dt_f;
    const int lo = max(lstar - 1, I.lmin), hi = I.lmax - 1;
    for (int s = 0; s < 4; ++s) {
      StageArgs& A = I.st[s];
      A.first = I.off[lstar];
      A.lstar = lstar;
      A.cur_mask = I.cur_mask;
      A.t_b = t_b;
      ProlongArgs& P = I.pr[s];
      P.list = I.up_list + I.up_off[lo];
      P.count = hi >= lo ? I.up_off[hi + 1] - I.up_off[lo] : 0;
      P.lstar = lstar;
      P.cur_mask = I.cur_mask;
      // finer sources of the active octants: the padding maps' finer leaves on levels > l*
      InjectArgs& J = I.in[s];
      J.first = I.dn_off[lstar + 1];
      J.list = I.dn_list + J.first;
      J.count = I.dn_off[I.lmax + 1] - J.first;
      J.cur_mask = I.cur_mask;
    }
  }
  __syncthreads();
  if (threadIdx.x < 12) B.next_item[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 4; ++s) {
      int* sp = B.stage_pre + s * (kMaxBatch + 1);
      int* pp = B.prol_pre + s * (kMaxBatch + 1);
      int* ip = B.inj_pre + s * (kMaxBatch + 1);
      sp[0] = pp[0] = ip[0] = 0;
      for (int k = 0; k < B.n; ++k) {
        const BatchInst& I = B.inst[k];
        const bool on = I.active && s < I.p;
        sp[k + 1] = sp[k] + (on ? I.n - I.off[I.lstar] : 0);
        pp[k + 1] = pp[k] + (on ? I.pr[s].count : 0);
        ip[k + 1] = ip[k] + (on ? I.in[s].count : 0);
      }
    }
  }
}

// End of a round (one CTA): schedules advanced, instances that finish a macro step marked
// for the reconcile, prefix sums of its work items.
__device__ void round_end_body(const BatchArgs& B) {
  for (int i = threadIdx.x; i < B.n; i += blockDim.x) {
    BatchInst& I = B.inst[i];
    if (I.active) {
      for (int l = I.lstar; l <= I.lmax; ++l) I.cur_mask ^= 1u << l;
      I.n_sub++;
      I.remaining--;
      if (I.n_sub == I.nsub_macro) {
        I.reconcile = 1;
        I.t_macro += double(I.n_sub) * I.dt_f;
        I.n_sub = 0;
      }
    }
    I.zip.sel_mask = I.cur_mask;
    I.hang.sel_mask = I.cur_mask;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    B.zip_pre[0] = 0;
    for (int k = 0; k < B.n; ++k) B.zip_pre[k + 1] = B.zip_pre[k] + (B.inst[k].reconcile ? B.inst[k].n : 0);
    for (int l = 0; l <= kMaxLevel + 1; ++l) {
      int* hp = B.hang_pre + l * (kMaxBatch + 1);
      hp[0] = 0;
      for (int k = 0; k < B.n; ++k) {
        const BatchInst& I = B.inst[k];
        const int c = (I.reconcile && l <= 32) ? I.hang_off[l + 1] - I.hang_off[l] : 0;
        hp[k + 1] = hp[k] + c;
      }
    }
  }
}

__global__ void batch_round_begin(BatchArgs B) { round_begin_body(B); }

__global__ void batch_round_end(BatchArgs B) { round_end_body(B); }

// copies an argument block into shared memory (all threads of the CTA)
template <bool C = false, typename T>
__device__ __forceinline__ void copy_args(T* dst, const T* src) {
  static_assert(sizeof(T) % 8 == 0, "argument blocks are 8-byte multiples");
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int q = threadIdx.x; q < int(sizeof(T) / 8); q += blockDim.x) d[q] = ld_in<C>(s + q);
}

// Work items (octant-stages of all instances, in instance order) are claimed one at
// a time from a counter, so that CTAs that drew expensive octants (level interfaces,
// the boundary) do not hold up the launch; a CTA re-reads an instance's arguments
// into shared memory only when its next item belongs to another instance.
__device__ __forceinline__ int claim_item(int* counter, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
  __syncthreads();
  return *slot;
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 4) batch_stage_kernel(const __grid_constant__ BatchArgs B, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ StageArgs args;  // the current instance's arguments
  __shared__ int s_item;
  const int* pre = B.stage_pre + stage * (kMaxBatch + 1);
  const int total = pre[B.n];
  int cur = -1;
  for (;;) {
    const int item = claim_item(B.next_item + 4 + stage, &s_item);
    if (item >= total) break;
    const int i = batch_find(pre, B.n + 1, item);
    if (i != cur) {
      copy_args(&args, &B.inst[i].st[stage]);
      __syncthreads();
      cur = i;
    }
    const int b = args.first + (item - pre[i]);
    if (args.nf == 1)
      stage_octant<1, R>(*reinterpret_cast<StageSmem<1, R, 1>*>(smem_raw), args, b);
    else
      stage_octant<2, R>(*reinterpret_cast<StageSmem<2, R, 1>*>(smem_raw), args, b);
  }
}

template <typename R>
__global__ void __launch_bounds__(256, 4) batch_prolong_kernel(const __grid_constant__ BatchArgs B, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ProlongArgs args;
  __shared__ int s_item;
  const int* pre = B.prol_pre + stage * (kMaxBatch + 1);
  const int total = pre[B.n];
  int cur = -1;
  for (;;) {
    const int item = claim_item(B.next_item + stage, &s_item);
    if (item >= total) break;
    const int i = batch_find(pre, B.n + 1, item);
    if (i != cur) {
      copy_args(&args, &B.inst[i].pr[stage]);
      __syncthreads();
      cur = i;
    }
    const int b = args.list[item - pre[i]];
    if (args.nf == 1)
      prolong_octant<1, R>(*reinterpret_cast<ProlongSmem<1, R>*>(smem_raw), args, b);
    else
      prolong_octant<2, R>(*reinterpret_cast<ProlongSmem<2, R>*>(smem_raw), args, b);
  }
}

template <typename R>
__global__ void __launch_bounds__(128, 16) batch_inject_kernel(const __grid_constant__ BatchArgs B, int stage) {
  __shared__ InjectArgs args;
  __shared__ int s_item;
  const int* pre = B.inj_pre + stage * (kMaxBatch + 1);
  const int total = pre[B.n];
  int cur = -1;
  for (;;) {
    const int item = claim_item(B.next_item + 8 + stage, &s_item);
    if (item >= total) break;
    const int i = batch_find(pre, B.n + 1, item);
    if (i != cur) {
      copy_args(&args, &B.inst[i].in[stage]);
      __syncthreads();
      cur = i;
    }
    const int k = item - pre[i];
    if (args.nf == 1)
      inject_octant<1, R>(args, __ldg(args.list + k), args.first + k);
    else
      inject_octant<2, R>(args, __ldg(args.list + k), args.first + k);
  }
}

__global__ void __launch_bounds__(128) batch_zip_kernel(const __grid_constant__ BatchArgs B) {
  __shared__ SyncSmem S;
  const int total = B.zip_pre[B.n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int i = batch_find(B.zip_pre, B.n + 1, item);
    sync_zip_octant<double>(S, B.inst[i].zip, item - B.zip_pre[i]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(128) batch_hanging_kernel(const __grid_constant__ BatchArgs B, int level) {
  __shared__ SyncSmem S;
  const int* pre = B.hang_pre + level * (kMaxBatch + 1);
  const int total = pre[B.n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int i = batch_find(pre, B.n + 1, item);
    const BatchInst& I = B.inst[i];
    sync_hanging_octant<double>(S, I.hang, I.hang_list[I.hang_off[level] + (item - pre[i])]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The persistent round: one cooperative launch per substep of all instances.  Its
// phases (round start, per RK stage the prolongation and the stage over the work items
// of every instance, round end, reconcile) are separated by a grid-wide barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a launch whose CTAs are all resident (a cooperative launch):
// bar[0] counts the CTAs that arrived, bar[1] is the barrier's generation.  Thread 0 of
// each CTA arrives after a fence (its CTA's writes are published); the last to arrive
// resets the count and advances the generation; the others poll the generation.  A CTA
// that polls longer than limit_ns, or finds kErrTimeout set in the error word, sets it
// and returns false, and so does every later barrier of the launch: all CTAs then leave
// the launch within about limit_ns, and the host reads kErrTimeout.  After the barrier
// every thread fences, so that its later loads see what the other CTAs wrote before it.
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* verr = err;
    int ok = (*verr & kErrTimeout) == 0;
    if (ok) {
      volatile unsigned* gen = bar + 1;
      const unsigned g = *gen;
      __threadfence();
      if (atomicAdd(bar, 1u) == gridDim.x - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        const unsigned long long t0 = global_ns();
        while (*gen == g) {
          if ((*verr & kErrTimeout) || global_ns() - t0 > limit_ns) {
            atomicOr(err, kErrTimeout);
            ok = 0;
            break;
          }
          __nanosleep(128);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  const int ok = s_ok;
  __threadfence();
  return ok != 0;
}

template <typename R>
union BatchSmem {
  StageSmem<2, R, 1> st;
  ProlongSmem<2, R> pr;
  SyncSmem sy;
};

// One round of a batch in one launch: grid-stride work claiming as in the per-stage
// kernels above, the phases separated by grid_barrier.  Every load of data that an
// earlier phase of the launch wrote goes through L2 (C = true) or is ordered by the
// barrier's fences (the asynchronous gathers, plain loads).
template <typename R>
__global__ void __launch_bounds__(kThreads, 3)
    batch_substep_kernel(const __grid_constant__ BatchArgs B, int pmax, int lmax_all, unsigned* bar, int* err,
                         unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem<R>& S = *reinterpret_cast<BatchSmem<R>*>(smem_raw);
  __shared__ StageArgs sargs;
  __shared__ ProlongArgs pargs;
  __shared__ InjectArgs jargs;
  __shared__ SyncArgs yargs;
  __shared__ int s_item;
  if (blockIdx.x == 0) round_begin_body(B);
  if (!grid_barrier(bar, err, limit_ns)) return;
  for (int st = 0; st < pmax; ++st) {
    {  // prolongation of the coarser sources of every instance
      const int* pre = B.prol_pre + st * (kMaxBatch + 1);
      const int total = __ldcg(pre + B.n);  // the same value in every CTA
      if (total > 0) {
        int cur = -1;
        for (;;) {
          const int item = claim_item(B.next_item + st, &s_item);
          if (item >= total) break;
          const int i = batch_find<true>(pre, B.n + 1, item);
          if (i != cur) {
            copy_args<true>(&pargs, &B.inst[i].pr[st]);
            __syncthreads();
            cur = i;
          }
          const int b = __ldg(pargs.list + (item - __ldcg(pre + i)));
          if (pargs.nf == 1)
            prolong_octant<1, R, true>(*reinterpret_cast<ProlongSmem<1, R>*>(&S.pr), pargs, b);
          else
            prolong_octant<2, R, true>(S.pr, pargs, b);
        }
      }
      // injection of the finer sources of every instance, in the same phase
      const int* ipre = B.inj_pre + st * (kMaxBatch + 1);
      const int itotal = __ldcg(ipre + B.n);
      if (itotal > 0) {
        int cur = -1;
        for (;;) {
          const int item = claim_item(B.next_item + 8 + st, &s_item);
          if (item >= itotal) break;
          const int i = batch_find<true>(ipre, B.n + 1, item);
          if (i != cur) {
            copy_args<true>(&jargs, &B.inst[i].in[st]);
            __syncthreads();
            cur = i;
          }
          const int k = item - __ldcg(ipre + i);
          if (jargs.nf == 1)
            inject_octant<1, R, true>(jargs, __ldg(jargs.list + k), jargs.first + k);
          else
            inject_octant<2, R, true>(jargs, __ldg(jargs.list + k), jargs.first + k);
        }
      }
      if (total > 0 || itotal > 0)
        if (!grid_barrier(bar, err, limit_ns)) return;
    }
    {  // the stage over the active octants of every instance
      const int* pre = B.stage_pre + st * (kMaxBatch + 1);
      const int total = __ldcg(pre + B.n);
      if (total > 0) {
        int cur = -1;
        for (;;) {
          const int item = claim_item(B.next_item + 4 + st, &s_item);
          if (item >= total) break;
          const int i = batch_find<true>(pre, B.n + 1, item);
          if (i != cur) {
            copy_args<true>(&sargs, &B.inst[i].st[st]);
            __syncthreads();
            cur = i;
          }
          const int b = sargs.first + (item - __ldcg(pre + i));
          if (sargs.nf == 1)
            stage_octant<1, R, kThreads>(*reinterpret_cast<StageSmem<1, R, 1>*>(&S.st), sargs, b);
          else
            stage_octant<2, R, kThreads>(S.st, sargs, b);
        }
        if (!grid_barrier(bar, err, limit_ns)) return;
      }
    }
  }
  if (blockIdx.x == 0) round_end_body(B);
  if (!grid_barrier(bar, err, limit_ns)) return;
  {  // reconcile of the instances that finished a macro step: zip, then hanging nodes by level
    const int total = __ldcg(B.zip_pre + B.n);
    if (total > 0) {
      int cur = -1;
      for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = batch_find<true>(B.zip_pre, B.n + 1, item);
        if (i != cur) {
          __syncthreads();
          copy_args<true>(&yargs, &B.inst[i].zip);
          __syncthreads();
          cur = i;
        }
        sync_zip_octant<double>(S.sy, yargs, item - __ldcg(B.zip_pre + i));
        __syncthreads();
      }
      if (!grid_barrier(bar, err, limit_ns)) return;
    }
  }
  for (int l = 1; l <= lmax_all; ++l) {
    const int* pre = B.hang_pre + l * (kMaxBatch + 1);
    const int total = __ldcg(pre + B.n);
    if (total == 0) continue;
    int cur = -1;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      const int i = batch_find<true>(pre, B.n + 1, item);
      if (i != cur) {
        __syncthreads();
        copy_args<true>(&yargs, &B.inst[i].hang);
        __syncthreads();
        cur = i;
      }
      const BatchInst& I = B.inst[i];
      sync_hanging_octant<double>(S.sy, yargs, __ldg(I.hang_list + I.hang_off[l] + (item - __ldcg(pre + i))));
      __syncthreads();
    }
    if (!grid_barrier(bar, err, limit_ns)) return;
  }
}

// The barrier alone, for its time limit: CTA `absent` returns without arriving (-1: all
// arrive), so that the other CTAs' waits run out and set kErrTimeout.
__global__ void barrier_probe_kernel(unsigned* bar, int* err, unsigned long long limit_ns, int absent) {
  if (int(blockIdx.x) == absent) return;
  grid_barrier(bar, err, limit_ns);
}

cudaError_t prepare_batch_kernels() {
  cudaError_t e = cudaFuncSetAttribute(batch_stage_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(StageSmem<2, double, 1>));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(batch_stage_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(StageSmem<2, float, 1>));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(batch_substep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(BatchSmem<double>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(batch_substep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(BatchSmem<float>));
}

cudaError_t batch_substep_resident(int mixed, int* per_sm, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  return mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_substep_kernel<float>, kThreads,
                                                               sizeof(BatchSmem<float>))
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_substep_kernel<double>, kThreads,
                                                               sizeof(BatchSmem<double>));
}

template <typename R>
static cudaError_t batch_round_t(const BatchArgs& a, int pmax, int lmax_all, int gs, int gp, int gy, cudaStream_t s) {
  const size_t smem_stage = sizeof(StageSmem<2, R, 1>);
  const size_t smem_prol = sizeof(ProlongSmem<2, R>);
  batch_round_begin<<<1, kMaxBatch, 0, s>>>(a);
  for (int st = 0; st < pmax; ++st) {
    batch_prolong_kernel<R><<<gp, 256, smem_prol, s>>>(a, st);
    batch_inject_kernel<R><<<gp, 128, 0, s>>>(a, st);
    batch_stage_kernel<R><<<gs, kThreads, smem_stage, s>>>(a, st);
  }
  batch_round_end<<<1, kMaxBatch, 0, s>>>(a);
  batch_zip_kernel<<<gy, 128, 0, s>>>(a);
  for (int l = 1; l <= lmax_all; ++l) batch_hanging_kernel<<<gy, 128, 0, s>>>(a, l);
  return cudaGetLastError();
}

cudaError_t launch_batch_round(const BatchArgs& a, int pmax, int lmax_all, int grid_stage, int grid_prolong,
                               int grid_sync, int mixed, cudaStream_t s) {
  return mixed ? batch_round_t<float>(a, pmax, lmax_all, grid_stage, grid_prolong, grid_sync, s)
               : batch_round_t<double>(a, pmax, lmax_all, grid_stage, grid_prolong, grid_sync, s);
}

template <typename R>
static cudaError_t batch_substep_t(const BatchArgs& a, int pmax, int lmax_all, int grid, unsigned* bar, int* err,
                                   unsigned long long limit_ns, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = sizeof(BatchSmem<R>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_substep_kernel<R>, a, pmax, lmax_all, bar, err, limit_ns);
}

cudaError_t launch_batch_substep(const BatchArgs& a, int pmax, int lmax_all, int grid, int mixed, unsigned* bar,
                                 int* err, unsigned long long limit_ns, cudaStream_t s) {
  return mixed ? batch_substep_t<float>(a, pmax, lmax_all, grid, bar, err, limit_ns, s)
               : batch_substep_t<double>(a, pmax, lmax_all, grid, bar, err, limit_ns, s);
}

cudaError_t launch_barrier_probe(int grid, unsigned* bar, int* err, unsigned long long limit_ns, int absent,
                                 cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, barrier_probe_kernel, bar, err, limit_ns, absent);
}

// ---------------------------------------------------------------------------
// Initial data
// ---------------------------------------------------------------------------
__global__ void init_kernel(InitArgs A) {
  const long long total = (long long)A.tree.n * kNV;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = int(e / kNV), n = int(e - (long long)b * kNV);
    const int4 o = A.tree.oct[b];
    const int eb = 1 << (kDepth - o.w);
    const int i = n % 7, j = (n / 7) % 7, k = n / 49;
    const double x[3] = {lattice_to_x(A.lo, A.ext, 6 * o.x + i * eb), lattice_to_x(A.lo, A.ext, 6 * o.y + j * eb),
                         lattice_to_x(A.lo, A.ext, 6 * o.z + k * eb)};
    double v0 = 0.0, v1 = 0.0;
    if (A.ic == LTS_IC_WAVE_SHELL) {
      const double R = A.icp.v[0], w = A.icp.v[1], amp = A.icp.v[2], ks = A.icp.v[4];
      const int nm = int(A.icp.v[3]);
      const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      double pert = 0.0;
      for (int m = 0; m < nm; ++m) {
        const double* md = A.icp.v + 5 + 5 * m;
        pert += md[0] * sin(ks * (md[1] * x[0] + md[2] * x[1] + md[3] * x[2]) + md[4]);
      }
      const double z = r - R;
      v0 = exp(-z * z / w) * (1.0 + amp * pert);
      v1 = 0.0;
    } else if (A.ic != LTS_IC_WAVE_REST) {
      double d[2][5];
      exact_derivs(A.ic, A.icp, A.adv, x, A.t0, d);
      v0 = d[0][0];
      v1 = d[1][0];
    }
    A.u[e] = v0;
    if (A.nf == 2) A.u[A.fstride + e] = v1;
  }
}

cudaError_t launch_init(const InitArgs& a, cudaStream_t s) {
  const long long total = (long long)a.tree.n * kNV;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  init_kernel<<<(int)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Padding map (Fig. unzip): for every octant and padded point, the slot of its source in
// the octant's neighbour view (one byte; kSlotNone outside the domain).  The tree is
// static, so this is resolved once per plan instead of at every stage; where the point
// lies in the source follows from the slot (stage_slots).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) padmap_kernel(const DevTree T, unsigned char* __restrict__ out, int* err) {
  __shared__ NbrView nv;
  for (int b = blockIdx.x; b < T.n; b += gridDim.x) {
    __syncthreads();
    load_neighbours(T, b, nv);
    __syncthreads();
    const int4 me = T.oct[b];
    const int lb = me.w;
    const int eb = 1 << (kDepth - lb);
    for (int q = threadIdx.x; q < kNT; q += blockDim.x) {
      const int i = q % 13 - 3, j = (q / 13) % 13 - 3, k = q / 169 - 3;
      unsigned entry;
      if (i >= 0 && i <= 6 && j >= 0 && j <= 6 && k >= 0 && k <= 6) {
        entry = 13u;
      } else {
        unsigned slot;
        const int src = resolve_source(nv, i, j, k, b, false, &slot);
        if (src < 0) {
          entry = kSlotNone;
        } else {
          const int4 so = T.oct[src];
          const int rx = half_node(6 * me.x + i * eb, so.x, so.w);
          const int ry = half_node(6 * me.y + j * eb, so.y, so.w);
          const int rz = half_node(6 * me.z + k * eb, so.z, so.w);
          const bool coarser = so.w < lb;
          // same-level and finer sources hold the point as a node (even coordinates)
          const bool odd = !coarser && ((rx | ry | rz) & 1);
          if (unsigned(rx) > 12u || unsigned(ry) > 12u || unsigned(rz) > 12u || unsigned(so.w - lb + 1) > 2u || odd) {
            atomicOr(err, 1);  // never on a balanced tree: reported, and the point becomes a zero ghost
            entry = kSlotNone;
          } else {
            entry = slot;
          }
        }
      }
      out[(long long)b * kNT + q] = static_cast<unsigned char>(entry);
    }
  }
}

cudaError_t launch_padmap(const DevTree& t, unsigned char* out, int* err, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  const int blocks = t.n < 152 * 8 ? t.n : 152 * 8;
  padmap_kernel<<<blocks, 256, 0, s>>>(t, out, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Map export (parity checks).  Padding maps are decoded from the plan's padding
// map (what the stage kernel reads); node maps use the resolver of the sync kernels.
// ---------------------------------------------------------------------------
__global__ void maps_kernel(MapArgs A) {
  __shared__ SyncSmem S;
  const int b = A.octs[blockIdx.x];
  load_neighbours(A.tree, b, S.nv);
  __syncthreads();
  const int4 me = A.tree.oct[b];
  const int eb = 1 << (kDepth - me.w);
  const int npts = A.nodes ? kNV : kNT;
  if (!A.nodes && A.padmap) {
    for (int q = threadIdx.x; q < kNT; q += blockDim.x) {
      const int src = slot_leaf(S.nv, A.padmap[(long long)b * kNT + q], b);
      const int i = q % 13 - 3, j = (q / 13) % 13 - 3, k = q / 169 - 3;
      const long long o = (long long)blockIdx.x * kNT + q;
      A.src[o] = src;
      int r[3] = {-1, -1, -1};
      if (src >= 0) {
        const int4 so = A.tree.oct[src];
        r[0] = half_node(6 * me.x + i * eb, so.x, so.w);
        r[1] = half_node(6 * me.y + j * eb, so.y, so.w);
        r[2] = half_node(6 * me.z + k * eb, so.z, so.w);
      }
      for (int a = 0; a < 3; ++a) A.r[o * 3 + a] = r[a];
    }
    return;
  }
  for (int q = threadIdx.x; q < npts; q += blockDim.x) {
    int i, j, k;
    if (A.nodes) {
      i = q % 7;
      j = (q / 7) % 7;
      k = q / 49;
    } else {
      i = q % 13 - 3;
      j = (q / 13) % 13 - 3;
      k = q / 169 - 3;
    }
    const bool inside = i >= 0 && i <= 6 && j >= 0 && j <= 6 && k >= 0 && k <= 6;
    int src = (inside && !A.nodes) ? b : resolve_source(S.nv, i, j, k, b, A.nodes != 0);
    int r[3] = {-1, -1, -1};
    if (src >= 0) {
      const int4 so = A.tree.oct[src];
      r[0] = half_node(6 * me.x + i * eb, so.x, so.w);
      r[1] = half_node(6 * me.y + j * eb, so.y, so.w);
      r[2] = half_node(6 * me.z + k * eb, so.z, so.w);
    }
    const long long o = (long long)blockIdx.x * npts + q;
    A.src[o] = src;
    for (int a = 0; a < 3; ++a) A.r[o * 3 + a] = r[a];
  }
}

__global__ void widen_kernel(const float* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = static_cast<double>(in[e]);
}

__global__ void narrow_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = static_cast<float>(in[e]);
}

cudaError_t launch_narrow(const double* in, float* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  narrow_kernel<<<(int)blocks, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_widen(const float* in, double* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  widen_kernel<<<(int)blocks, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_maps(const MapArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  maps_kernel<<<a.count, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed device staging area of lts_export_pad_map_static: room for the octant
// list and the padding sources of kStaticMapOctants octants.  It lives in the
// library image, so every GPU that loads the library holds it (about 1.1 MB)
// until the process exits, and no call allocates.
// ---------------------------------------------------------------------------
static __device__ __align__(256) int g_static_map_scratch[kStaticMapOctants * (1 + 4 * kNT)];

// Device address of the staging area on the current device.  Host code cannot
// use the symbol itself (it names a host-side stand-in), so the address is
// looked up once per device, with that device current, and cached.
cudaError_t static_map_scratch(int** out) {
  static std::mutex mu;
  static int* cached[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!cached[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_map_scratch);
    if (e != cudaSuccess) return e;
    cached[dev] = static_cast<int*>(ptr);
  }
  *out = cached[dev];
  return cudaSuccess;
}

}  // namespace ltsoct
