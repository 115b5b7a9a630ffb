// CUDA kernels of libltsoct for GB300 (sm_103a).
//
// The LTS substep (Alg. 2, Fig. blk_loop) runs one launch of stage_kernel per
// RK stage over the active octants, which are a contiguous suffix of the level
// order.  One CTA owns one octant: it resolves the source of each of the 2197
// points of its padded block (Sec. 3.3: coarsest leaf containing the point, ties
// to the smallest Morton key = smallest level-order index), forms the time-
// corrected stage inputs of the sources (eqs. fc_1, fc_2), interpolates from
// coarser sources in shared memory (Fig. unzip), fills the physical boundary,
// evaluates the 4th-order FD right-hand side with Kreiss-Oliger dissipation on
// the 7^3 interior and writes the stage (and, at the last stage, the RK update
// of eq. rk_schemes into the other half of the double-buffered state).
//
// FP64 on GB300 issues about 2 DFMA per clock per SM, so these kernels are
// bound by the FP64 pipe; integer work (source resolution) and memory traffic
// hide behind it.  The FD formulas are arranged to share the symmetric sums
// between the Laplacian and the dissipation.
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

cudaError_t upload_tables(const Tables* rk4, const Tables* rk3, const double W[13][7], const double E[4][4]) {
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

// (i,j,k) in the octant's node units, i in [-3, 9]; returns -1 outside the domain
__device__ int resolve_source(const NbrView& nv, int i, int j, int k, int self, bool with_self) {
  int x0, x1, y0, y1, z0, z1;
  axis_candidates(i, x0, x1);
  axis_candidates(j, y0, y1);
  axis_candidates(k, z0, z1);
  int best = INT_MAX;
  for (int dz = z0; dz <= z1; ++dz)
    for (int dy = y0; dy <= y1; ++dy)
      for (int dx = x0; dx <= x1; ++dx) {
        const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        if (d == 13) {
          if (with_self) best = min(best, self);
          continue;
        }
        const int e = nv.nbr[d];
        if (e == -1) continue;
        if (e >= 0) {
          best = min(best, e);
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
              if (leaf >= 0) best = min(best, leaf);
            }
      }
  return best == INT_MAX ? -1 : best;
}

// half-node coordinate of lattice6 coordinate P in a source with anchor a, level l
__device__ __forceinline__ int half_node(int P, int a, int l) { return ((P - 6 * a) * 2) >> (kDepth - l); }

__device__ void load_neighbours(const DevTree& t, int b, NbrView& nv) {
  for (int d = threadIdx.x; d < 27; d += blockDim.x) nv.nbr[d] = t.nbr[b * 27 + d];
  __syncthreads();
  for (int q = threadIdx.x; q < 27 * 8; q += blockDim.x) {
    const int d = q >> 3, c = q & 7;
    const int e = nv.nbr[d];
    nv.kids[d][c] = e <= -2 ? t.fine[(-e - 2) * 8 + c] : -1;
  }
}

// stage input of a source node from its step-start state and RK stages,
// u + dt * sum_t w_t K_(j_t)  (eq. rk_schemes with the corrected weights of
// eqs. fc_1 / fc_2)
__device__ __forceinline__ double corrected_value(const double* __restrict__ u, const double* __restrict__ k0,
                                                  long long kstride, const StageTerms& t, double dt) {
  double acc = 0.0;
  for (int q = 0; q < t.n; ++q) acc = fma(t.w[q], __ldg(k0 + t.j[q] * kstride), acc);
  return fma(dt, acc, __ldg(u));
}

// tensor-product Lagrange interpolation, x then y then z; even coordinates are nodes
__device__ double interp_tensor(const double* __restrict__ v, const double (*W)[7], int rx, int ry, int rz) {
  const int x0 = (rx & 1) ? 0 : rx >> 1, x1 = (rx & 1) ? 6 : rx >> 1;
  const int y0 = (ry & 1) ? 0 : ry >> 1, y1 = (ry & 1) ? 6 : ry >> 1;
  const int z0 = (rz & 1) ? 0 : rz >> 1, z1 = (rz & 1) ? 6 : rz >> 1;
  double sz = 0.0;
  for (int c = z0; c <= z1; ++c) {
    double sy = 0.0;
    for (int bb = y0; bb <= y1; ++bb) {
      double sx = 0.0;
      for (int a = x0; a <= x1; ++a) sx = fma(W[rx][a], v[a + 7 * bb + 49 * c], sx);
      sy = fma(W[ry][bb], sx, sy);
    }
    sz = fma(W[rz][c], sy, sz);
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
template <int NF>
struct StageSmem {
  double T[NF][kNT];         // padded tiles
  StageTerms om[4];          // correction terms of this stage per relation
  int src[kNT];
  unsigned short code[kNT];  // rx | ry << 4 | rz << 8 | (level diff + 1) << 12 | exterior << 15
  NbrView nv;
};

constexpr unsigned kExterior = 1u << 15;
constexpr int kPer = (kNT + kThreads - 1) / kThreads;  // padded points per thread

// exact boundary data (reading R10): RK stage values of the closed-form solution
template <int NF>
__device__ __noinline__ void fill_exact(StageSmem<NF>& S, const StageArgs& A, int4 me, int eb, double dtb) {
  for (int q = threadIdx.x; q < kNT; q += blockDim.x) {
    if (!(S.code[q] & kExterior)) continue;
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
      S.T[f][q] = v;
    }
  }
}

// radiative boundary (reading R11): cubic extrapolation along the outward normal, x then y then z
template <int NF>
__device__ __noinline__ void fill_extrapolated(StageSmem<NF>& S, int4 me, int eb) {
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
            double v = 0.0;
            for (int qq = 0; qq < 4; ++qq) v = fma(c_E[m][qq], S.T[f][base + qq * str], v);
            S.T[f][base - m * str] = v;
          }
          if (hi_b) {
            double v = 0.0;
            for (int qq = 0; qq < 4; ++qq) v = fma(c_E[m][qq], S.T[f][base + (6 - qq) * str], v);
            S.T[f][base + (6 + m) * str] = v;
          }
        }
      }
    }
    __syncthreads();
  }
}

// radiative right-hand side at a node on the domain boundary
template <int NF>
__device__ __noinline__ void radiative_rhs(const StageSmem<NF>& S, const StageArgs& A, int c0, const int P6[3],
                                           double inv12h, double kv[NF]) {
  const double x[3] = {lattice_to_x(A.lo, A.ext, P6[0]), lattice_to_x(A.lo, A.ext, P6[1]),
                       lattice_to_x(A.lo, A.ext, P6[2])};
  const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const int st[3] = {1, 13, 169};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double* T = S.T[f];
    double xd = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double d1 = fma(8.0, T[c0 + st[a]] - T[c0 - st[a]], T[c0 - 2 * st[a]] - T[c0 + 2 * st[a]]) * inv12h;
      xd = fma(x[a], d1, xd);
    }
    kv[f] = -(xd + (f == 0 ? 1.0 : 2.0) * T[c0]) / r;
  }
}

template <int NF>
__global__ void __launch_bounds__(kThreads, 4) stage_kernel(StageArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StageSmem<NF>& S = *reinterpret_cast<StageSmem<NF>*>(smem_raw);
  const int b = A.first + blockIdx.x;
  const int tid = threadIdx.x;
  const int p = A.p;
  const int s = A.stage;
  const int4 me = A.tree.oct[b];
  const int lb = me.w;
  const int eb = 1 << (kDepth - lb);
  const long long kstride = (long long)A.nf * A.fstride;

  load_neighbours(A.tree, b, S.nv);
  if (tid < 4) S.om[tid] = A.om[tid];
  __syncthreads();

  // 1. source of every padded point (coarsest leaf containing it, then smallest Morton key)
  for (int q = tid; q < kNT; q += blockDim.x) {
    const int i = q % 13 - 3, j = (q / 13) % 13 - 3, k = q / 169 - 3;
    int src;
    unsigned code;
    if (i >= 0 && i <= 6 && j >= 0 && j <= 6 && k >= 0 && k <= 6) {
      src = b;
      code = unsigned(2 * i) | unsigned(2 * j) << 4 | unsigned(2 * k) << 8 | 1u << 12;
    } else {
      src = resolve_source(S.nv, i, j, k, b, false);
      if (src < 0) {
        code = kExterior;
      } else {
        const int4 so = A.tree.oct[src];
        const int rx = half_node(6 * me.x + i * eb, so.x, so.w);
        const int ry = half_node(6 * me.y + j * eb, so.y, so.w);
        const int rz = half_node(6 * me.z + k * eb, so.z, so.w);
        if (unsigned(rx) > 12u || unsigned(ry) > 12u || unsigned(rz) > 12u || unsigned(so.w - lb + 1) > 2u) {
          atomicOr(A.err, 1);  // never on a balanced tree: report and use a zero ghost
          src = -1;
          code = kExterior;
        } else {
          code = unsigned(rx) | unsigned(ry) << 4 | unsigned(rz) << 8 | unsigned(so.w - lb + 1) << 12;
        }
      }
    }
    S.src[q] = src;
    S.code[q] = static_cast<unsigned short>(code);
  }
  __syncthreads();

  // 2. gathers, batched for memory parallelism: own interior and same-level sources
  //    read the stage inputs; coarser sources read their prolonged stage inputs
  //    (Fig. unzip, prepared by prolong_kernel); under GTS every source is read directly
  const double* direct = s == 0 ? A.u[(A.cur_mask >> lb) & 1] : A.Uin;
  {
    double v[kPer][NF];
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
      const int q = tid + it * kThreads;
#pragma unroll
      for (int f = 0; f < NF; ++f) v[it][f] = 0.0;
      if (q < kNT) {
        const unsigned code = S.code[q];
        if (!(code & kExterior)) {
          const int rx = code & 15, ry = (code >> 4) & 15, rz = (code >> 8) & 15;
          const int rel_code = (code >> 12) & 3;  // 0 coarser, 1 same, 2 finer
          const int src = S.src[q];
          if (rel_code == 0) {
            const double* up = A.up + (long long)__ldg(A.up_slot + src) * NF * kNT + rx + 13 * ry + 169 * rz;
#pragma unroll
            for (int f = 0; f < NF; ++f) v[it][f] = __ldg(up + f * kNT);
          } else if (rel_code == 1 || A.gts) {
            const long long off = (long long)src * kNV + (rx >> 1) + 7 * (ry >> 1) + 49 * (rz >> 1);
#pragma unroll
            for (int f = 0; f < NF; ++f) v[it][f] = __ldg(direct + f * A.fstride + off);
          }
        }
      }
    }
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
      const int q = tid + it * kThreads;
      if (q < kNT) {
#pragma unroll
        for (int f = 0; f < NF; ++f) S.T[f][q] = v[it][f];
      }
    }
  }

  // 3. finer sources (injection) with the coarse<-fine correction of eq. fc_1
  if (!A.gts) {
    for (int q = tid; q < kNT; q += blockDim.x) {
      const unsigned code = S.code[q];
      if ((code & kExterior) || ((code >> 12) & 3) != 2) continue;
      const int rx = code & 15, ry = (code >> 4) & 15, rz = (code >> 8) & 15;
      const int ls = lb + 1;
      const double* ub = A.u[(A.cur_mask >> ls) & 1];
      const long long off = (long long)S.src[q] * kNV + (rx >> 1) + 7 * (ry >> 1) + 49 * (rz >> 1);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        S.T[f][q] = corrected_value(ub + f * A.fstride + off, A.K + f * A.fstride + off, kstride, S.om[1],
                                    A.lc[ls].dt);
    }
  }
  __syncthreads();

  // 5. physical boundary
  const LevelConst lc = A.lc[lb];
  constexpr int kRoot = 1 << kDepth;
  const bool touches = me.x == 0 || me.y == 0 || me.z == 0 || me.x + eb == kRoot || me.y + eb == kRoot ||
                       me.z + eb == kRoot;
  if (touches) {
    if (A.bc == LTS_BC_EXACT)
      fill_exact<NF>(S, A, me, eb, lc.dt);
    else
      fill_extrapolated<NF>(S, me, eb);
  }
  __syncthreads();

  // 6. right-hand side on the 7^3 interior; stage, next stage input, fused RK update
  if (tid < kNV) {
    const int i = tid % 7, j = (tid / 7) % 7, k = tid / 49;
    const int c0 = (i + 3) + 13 * (j + 3) + 169 * (k + 3);
    double kv[NF];
    if (A.pde == LTS_PDE_ADVECTION) {
      const double* T = S.T[0];
      const double u0 = T[c0];
      // symmetric pair sums at distance 1, 2, 3 (Kreiss-Oliger) and the D1 differences
      const double P1 = (T[c0 - 1] + T[c0 + 1]) + (T[c0 - 13] + T[c0 + 13]) + (T[c0 - 169] + T[c0 + 169]);
      const double P2 = (T[c0 - 2] + T[c0 + 2]) + (T[c0 - 26] + T[c0 + 26]) + (T[c0 - 338] + T[c0 + 338]);
      const double P3 = (T[c0 - 3] + T[c0 + 3]) + (T[c0 - 39] + T[c0 + 39]) + (T[c0 - 507] + T[c0 + 507]);
      double d1s = A.adv[0] * fma(8.0, T[c0 + 1] - T[c0 - 1], T[c0 - 2] - T[c0 + 2]);
      d1s = fma(A.adv[1], fma(8.0, T[c0 + 13] - T[c0 - 13], T[c0 - 26] - T[c0 + 26]), d1s);
      d1s = fma(A.adv[2], fma(8.0, T[c0 + 169] - T[c0 - 169], T[c0 - 338] - T[c0 + 338]), d1s);
      const double ko = fma(-60.0, u0, fma(15.0, P1, fma(-6.0, P2, P3)));
      kv[0] = fma(lc.kos, ko, -lc.inv12h * d1s);
    } else {
      const double* Tc = S.T[0];
      const double* Tp = S.T[NF - 1];
      const double c0v = Tc[c0], f0v = Tp[c0];
      const double C1 = (Tc[c0 - 1] + Tc[c0 + 1]) + (Tc[c0 - 13] + Tc[c0 + 13]) + (Tc[c0 - 169] + Tc[c0 + 169]);
      const double C2 = (Tc[c0 - 2] + Tc[c0 + 2]) + (Tc[c0 - 26] + Tc[c0 + 26]) + (Tc[c0 - 338] + Tc[c0 + 338]);
      const double C3 = (Tc[c0 - 3] + Tc[c0 + 3]) + (Tc[c0 - 39] + Tc[c0 + 39]) + (Tc[c0 - 507] + Tc[c0 + 507]);
      const double F1 = (Tp[c0 - 1] + Tp[c0 + 1]) + (Tp[c0 - 13] + Tp[c0 + 13]) + (Tp[c0 - 169] + Tp[c0 + 169]);
      const double F2 = (Tp[c0 - 2] + Tp[c0 + 2]) + (Tp[c0 - 26] + Tp[c0 + 26]) + (Tp[c0 - 338] + Tp[c0 + 338]);
      const double F3 = (Tp[c0 - 3] + Tp[c0 + 3]) + (Tp[c0 - 39] + Tp[c0 + 39]) + (Tp[c0 - 507] + Tp[c0 + 507]);
      const double lap = fma(-90.0, c0v, fma(16.0, C1, -C2)) * lc.inv12h2;
      const double koc = fma(-60.0, c0v, fma(15.0, C1, fma(-6.0, C2, C3)));
      const double kop = fma(-60.0, f0v, fma(15.0, F1, fma(-6.0, F2, F3)));
      kv[0] = fma(lc.kos, koc, f0v);
      kv[NF - 1] = fma(lc.kos, kop, lap);
      if (A.bc == LTS_BC_RADIATIVE && touches) {
        const int P6[3] = {6 * me.x + i * eb, 6 * me.y + j * eb, 6 * me.z + k * eb};
        const bool on_bnd = P6[0] == 0 || P6[1] == 0 || P6[2] == 0 || P6[0] == kLatt6 || P6[1] == kLatt6 ||
                            P6[2] == kLatt6;
        if (on_bnd) radiative_rhs<NF>(S, A, c0, P6, lc.inv12h, kv);
      }
    }
    const long long node = (long long)b * kNV + tid;
    const double* ucur = A.u[(A.cur_mask >> lb) & 1];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long o = f * A.fstride + node;
      A.K[(long long)s * kstride + o] = kv[f];
      if (s < p - 1) {
        // stage input of the next stage: u + dt sum_j a[s+1][j] k_j
        double acc = 0.0;
        for (int q = 0; q < A.next.n; ++q)
          acc = fma(A.next.w[q], A.next.j[q] == s ? kv[f] : A.K[(long long)A.next.j[q] * kstride + o], acc);
        A.Uout[o] = fma(lc.dt, acc, ucur[o]);
      } else if (A.write_update) {
        double acc = 0.0;
        for (int q = 0; q < p - 1; ++q) acc = fma(A.w[q], A.K[(long long)q * kstride + o], acc);
        acc = fma(A.w[p - 1], kv[f], acc);
        A.u[((A.cur_mask >> lb) & 1) ^ 1][o] = fma(lc.dt, acc, ucur[o]);
      }
    }
  }
}

template <int NF>
static size_t stage_smem() {
  return sizeof(StageSmem<NF>);
}

cudaError_t launch_stage(const StageArgs& a, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_smem<1>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(stage_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_smem<2>());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (a.nf == 1)
    stage_kernel<1><<<count, kThreads, stage_smem<1>(), s>>>(a);
  else
    stage_kernel<2><<<count, kThreads, stage_smem<2>(), s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prolongation of coarser sources (Fig. unzip, coarse -> fine).  One CTA per
// octant with finer neighbours forms its stage inputs as those neighbours see
// them (eqs. fc_1 / fc_2) and interpolates them, sum-factorised x, then y, then z,
// to every half-node position of the box its finer neighbours read.  Each finer
// neighbour then gathers these values as plain copies.
// ---------------------------------------------------------------------------
template <int NF>
struct ProlongSmem {
  double V[NF][kNV];
  double X1[NF][13 * 49];      // [rx][z][y]
  double X2[NF][13 * 13 * 7];  // [rx][ry][z]
  double W[13][7];
};

template <int NF>
__global__ void __launch_bounds__(256) prolong_kernel(ProlongArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ProlongSmem<NF>& S = *reinterpret_cast<ProlongSmem<NF>*>(smem_raw);
  const int tid = threadIdx.x;
  const int b = A.list[blockIdx.x];
  const int slot = A.up_slot[b];
  const int lb = A.tree.oct[b].w;
  const int rel = A.gts ? 0 : (lb >= A.lstar ? 2 : 3);
  const int bx = A.box[slot];
  const int rx0 = bx & 15, ry0 = (bx >> 8) & 15, rz0 = (bx >> 16) & 15;
  const int nrx = ((bx >> 4) & 15) - rx0 + 1, nry = ((bx >> 12) & 15) - ry0 + 1, nrz = ((bx >> 20) & 15) - rz0 + 1;
  const long long kstride = (long long)A.nf * A.fstride;
  for (int q = tid; q < 91; q += blockDim.x) S.W[q / 7][q % 7] = c_W[q / 7][q % 7];
  const int cur = (A.cur_mask >> lb) & 1;
  const double* direct = A.stage == 0 ? A.u[cur] : A.Uin;
  const double* ub = A.u[cur ^ (rel == 3 ? 1 : 0)];
  for (int t = tid; t < NF * kNV; t += blockDim.x) {
    const int f = t / kNV, n = t - f * kNV;
    const long long off = (long long)b * kNV + n;
    S.V[f][n] = rel == 0 ? __ldg(direct + f * A.fstride + off)
                         : corrected_value(ub + f * A.fstride + off, A.K + f * A.fstride + off, kstride, A.om[rel],
                                           A.lc[lb].dt);
  }
  __syncthreads();
  for (int t = tid; t < NF * nrx * 49; t += blockDim.x) {
    const int f = t / (nrx * 49), rem = t - f * nrx * 49;
    const int rxi = rem / 49, yz = rem - rxi * 49;  // yz = y + 7 z
    const int rx = rx0 + rxi;
    const double* v = S.V[f] + 7 * yz;
    double acc;
    if (rx & 1) {
      acc = 0.0;
#pragma unroll
      for (int a = 0; a < 7; ++a) acc = fma(S.W[rx][a], v[a], acc);
    } else {
      acc = v[rx >> 1];
    }
    S.X1[f][rem] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NF * nrx * nry * 7; t += blockDim.x) {
    const int f = t / (nrx * nry * 7), rem = t - f * nrx * nry * 7;
    const int z = rem % 7, ryi = (rem / 7) % nry, rxi = rem / (7 * nry);
    const int ry = ry0 + ryi;
    const double* x1 = S.X1[f] + rxi * 49 + 7 * z;  // [y]
    double acc;
    if (ry & 1) {
      acc = 0.0;
#pragma unroll
      for (int bb = 0; bb < 7; ++bb) acc = fma(S.W[ry][bb], x1[bb], acc);
    } else {
      acc = x1[ry >> 1];
    }
    S.X2[f][rem] = acc;
  }
  __syncthreads();
  double* out = A.up + (long long)slot * NF * kNT;
  for (int t = tid; t < NF * nrx * nry * nrz; t += blockDim.x) {
    const int f = t / (nrx * nry * nrz), rem = t - f * nrx * nry * nrz;
    const int rxi = rem % nrx, ryi = (rem / nrx) % nry, rzi = rem / (nrx * nry);
    const int rz = rz0 + rzi;
    const double* x2 = S.X2[f] + (rxi * nry + ryi) * 7;  // [z]
    double acc;
    if (rz & 1) {
      acc = 0.0;
#pragma unroll
      for (int cc = 0; cc < 7; ++cc) acc = fma(S.W[rz][cc], x2[cc], acc);
    } else {
      acc = x2[rz >> 1];
    }
    out[f * kNT + (rx0 + rxi) + 13 * (ry0 + ryi) + 169 * rz] = acc;
  }
}

cudaError_t launch_prolong(const ProlongArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  if (a.nf == 1)
    prolong_kernel<1><<<a.count, 256, sizeof(ProlongSmem<1>), s>>>(a);
  else
    prolong_kernel<2><<<a.count, 256, sizeof(ProlongSmem<2>), s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// GTS step update (Alg. 1 compute_step) from the synchronised stages
// ---------------------------------------------------------------------------
__global__ void update_kernel(UpdateArgs A) {
  const long long total = (long long)A.nf * A.fstride;
  const DevTables& tab = c_tab[A.scheme];
  const long long kstride = (long long)A.nf * A.fstride;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long inf = e % A.fstride;
    const int b = int(inf / kNV);
    const int cur = (A.cur_mask >> A.oct[b].w) & 1;
    double acc = 0.0;
    for (int q = 0; q < A.p - 1; ++q) acc = fma(tab.w[q], A.K[q * kstride + e], acc);
    acc = fma(tab.w[A.p - 1], A.K[(A.p - 1) * kstride + e], acc);
    A.u[cur ^ 1][e] = fma(A.dt_f, acc, A.u[cur][e]);
  }
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  const long long total = (long long)a.nf * a.fstride;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  update_kernel<<<(int)blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-node synchronisation (zip + unzip, Fig. dg_to_cg), in place
// ---------------------------------------------------------------------------
struct SyncSmem {
  NbrView nv;
};

__device__ __forceinline__ bool is_boundary_node(int i, int j, int k) {
  return i == 0 || i == 6 || j == 0 || j == 6 || k == 0 || k == 6;
}

// zip: every non-hanging node takes its owner's value (owners keep theirs)
__global__ void __launch_bounds__(128) sync_zip_kernel(SyncArgs A) {
  __shared__ SyncSmem S;
  const int b = A.list ? A.list[blockIdx.x] : blockIdx.x;
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
    const double* vs = A.vb[(A.sel_mask >> so.w) & 1];
    double* vd = A.vb[(A.sel_mask >> me.w) & 1];
    for (int f = 0; f < A.nf; ++f)
      vd[f * A.fstride + (long long)b * kNV + n] =
          vs[f * A.fstride + (long long)src * kNV + (rx >> 1) + 7 * (ry >> 1) + 49 * (rz >> 1)];
  }
}

// unzip of hanging nodes of the listed octants (all of one level, whose coarser
// sources are final)
__global__ void __launch_bounds__(128) sync_hanging_kernel(SyncArgs A) {
  __shared__ SyncSmem S;
  const int b = A.list[blockIdx.x];
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
    if (!((rx | ry | rz) & 1)) continue;
    const double* vs = A.vb[(A.sel_mask >> so.w) & 1];
    double* vd = A.vb[(A.sel_mask >> me.w) & 1];
    for (int f = 0; f < A.nf; ++f)
      vd[f * A.fstride + (long long)b * kNV + n] = interp_tensor(vs + f * A.fstride + (long long)src * kNV, c_W, rx, ry, rz);
  }
}

cudaError_t launch_sync_zip(const SyncArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  sync_zip_kernel<<<a.count, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sync_hanging(const SyncArgs& a, cudaStream_t s) {
  if (a.count <= 0) return cudaSuccess;
  sync_hanging_kernel<<<a.count, 128, 0, s>>>(a);
  return cudaGetLastError();
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
    } else {
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
// Map export (parity checks): the same resolver the stage and sync kernels use
// ---------------------------------------------------------------------------
__global__ void maps_kernel(MapArgs A) {
  __shared__ SyncSmem S;
  const int b = A.octs[blockIdx.x];
  load_neighbours(A.tree, b, S.nv);
  __syncthreads();
  const int4 me = A.tree.oct[b];
  const int eb = 1 << (kDepth - me.w);
  const int npts = A.nodes ? kNV : kNT;
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
