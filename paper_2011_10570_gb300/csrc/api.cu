// C ABI of libltsoct (include/ltsoct.h): plan lifecycle, the LTS substep
// schedule (Alg. 2, Fig. blk_loop), GTS (Alg. 1), the shared-node sync and the
// parity exports.  All device work is enqueued on the plan's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "ltsoct_internal.h"

namespace ltsoct {
const char* last_error_cstr();
}

using ltsoct::kNV;

// Algorithmic work of one node-stage (FMA = 2 flops, add/mul = 1), counted from
// the stage kernel's formulas.  Wave: six symmetric pair sums per field (30), the
// Laplacian (5), two dissipation combinations (12), two outputs (4), the next
// stage input (3 over four stages) and the RK update's share (5) = 59.
// Advection: pair sums (15), D1 differences and a.grad (17), dissipation (6),
// output (3), next stage input (1.5), update share (2.5) = 45.
static double flops_per_node_stage(int pde) { return pde == LTS_PDE_ADVECTION ? 45.0 : 59.0; }
// Algorithmic HBM bytes of one node-stage per field: own stage input (8), own
// step-start state (8), the stage (8), the next stage input (6 over four
// stages), the update's share of stage reads and state write (6 + 2) = 38.
// Ghost reads of neighbours are expected to hit L2 and are not counted.  Mixed
// precision (FP32 stage type): 4 + 8 + 4 + 3 + (3 + 2) = 24 bytes per field.
static double bytes_per_node_stage(int nf, int mixed) { return (mixed ? 24.0 : 38.0) * nf; }

struct lts_plan {
  lts_problem prob;
  lts_refine_spec spec;
  ltsoct::Tables tab;
  int scheme = 0;
  int64_t N = 0;
  int nf = 1, p = 4, lmin = 0, lmax = 0;
  int64_t count[33] = {};
  int64_t off[34] = {};
  double dt_f = 0.0, t_macro = 0.0;
  int64_t n_sub = 0;
  unsigned cur_mask = 0;
  std::vector<ltsoct::Oct> octs;
  ltsoct::Neighbours nb;
  std::vector<int32_t> hang;           // octants with hanging nodes, level order
  int64_t hang_off[34] = {};           // per level ranges in hang
  int4* d_oct = nullptr;
  int* d_nbr = nullptr;
  int* d_fine = nullptr;
  int* d_hang = nullptr;
  double* d_u[2] = {nullptr, nullptr};
  float* d_us[2] = {nullptr, nullptr};  // mixed precision: FP32 copies of d_u
  void* d_K = nullptr;                  // RK stages, stage type
  void* d_U[2] = {nullptr, nullptr};    // stage inputs of the current and the next stage, stage type
  int mixed = 0;                        // 1: FP32 stage type
  size_t es = 8;                        // bytes per stage-type element
  std::vector<int32_t> up_list;         // octants with finer neighbours (coarser sources), level order
  int64_t up_off[34] = {};              // per level ranges in up_list
  std::vector<int32_t> up_box, up_slot;
  int* d_up_list = nullptr;
  int* d_up_box = nullptr;
  int* d_up_slot = nullptr;
  void* d_up = nullptr;                 // prolonged stage inputs [slot][nf][2197], stage type
  int* d_err = nullptr;
  unsigned char* d_padmap = nullptr;  // [N][2197] padding map (source slots), built once by padmap_kernel
  int* d_slotmap = nullptr;             // [N][256] per octant and slot: base << 2 | kind (slotmap_kernel)
  // finer sources: the leaves some padding map takes a point from through a child slot
  std::vector<int32_t> dn_list;         // level order
  int64_t dn_off[34] = {};              // per level ranges in dn_list
  int* d_dn_list = nullptr;
  int* d_dn_slot = nullptr;             // per octant: its position in dn_list, or -1
  void* d_inj = nullptr;                // injected stage inputs of finer sources [dn][nf][64], stage type
  // compact shared-node maps (zip: copied nodes; hanging: interpolated nodes, per level)
  int* d_zl_dst = nullptr;
  int* d_zl_src = nullptr;
  int64_t n_zip = 0;
  int* d_hl_dst = nullptr;
  int* d_hl_src = nullptr;
  unsigned short* d_hl_code = nullptr;
  int64_t hl_off[34] = {};
  // octree-to-block decomposition (Sec. 3.2.5): complete sibling groups are stepped as
  // one 13^3-node block by block_kernel, the other octants one by one by stage_kernel
  bool blocking = true;
  std::vector<int32_t> grp, single;     // first octant of each group / the other octants, level order
  int64_t grp_off[34] = {}, single_off[34] = {};
  int* d_grp = nullptr;
  int* d_single = nullptr;
  int* d_gsrc = nullptr;                // [G][kBG]: ghost points of the block tiles
  unsigned short* d_gcode = nullptr;    // [G][kBG]
  int64_t launches = 0;               // every kernel launched by the plan
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  int device = -1;                      // CUDA device current when the plan was created
  std::vector<void*> allocations;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  std::vector<int64_t> event_nodes;
  int64_t prof_launches = 0, prof_node_stages = 0;
  double prof_ms = 0.0;
  // prolongation launches under profiling: events, FP64-equivalent flops and sources
  std::vector<int64_t> up_cost;  // prefix sums over up_list of the interpolation multiply-adds per field
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pevents;
  std::vector<double> pevent_flops;
  std::vector<int64_t> pevent_sources;
  int64_t pprof_launches = 0, pprof_sources = 0;
  double pprof_ms = 0.0, pprof_flops = 0.0;
  double w_lts = 0.0, w_gts = 0.0;
};

namespace {

lts_status fail(lts_status s, const std::string& msg) {
  ltsoct::set_last_error(msg);
  return s;
}

lts_status cuda_fail(cudaError_t e, const char* where) {
  return fail(LTS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                       \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

void* dev_alloc(lts_plan* P, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* ptr = nullptr;
  if (P->prob.dev_alloc) {
    ptr = P->prob.dev_alloc(bytes, P->prob.alloc_ctx);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (ptr) {
    P->allocations.push_back(ptr);
    P->bytes += bytes;
  }
  return ptr;
}

void release(lts_plan* P) {
  if (P->stream) cudaStreamSynchronize(P->stream);
  for (auto& ev : P->events) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  P->events.clear();
  for (auto& ev : P->pevents) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  P->pevents.clear();
  for (void* ptr : P->allocations) {
    if (P->prob.dev_free)
      P->prob.dev_free(ptr, P->prob.alloc_ctx);
    else
      cudaFree(ptr);
  }
  P->allocations.clear();
}

ltsoct::DevTree dev_tree(const lts_plan* P) {
  return ltsoct::DevTree{P->d_oct, P->d_nbr, P->d_fine, int(P->N)};
}

int cur_of(const lts_plan* P, int l) { return (P->cur_mask >> l) & 1; }

// in-place shared-node sync of the arrays vb (level l uses vb[(sel >> l) & 1])
// Compact shared-node maps: nodemap_kernel resolves the owner of every boundary node of
// every octant once (dense, temporary); the copies and the hanging nodes are gathered
// into lists on the host, the hanging ones per level and within a level ordered by the
// number of odd half-node coordinates (uniform work across a warp).
lts_status build_node_maps(lts_plan* P) {
  const size_t nb = size_t(P->N) * ltsoct::kBN, nh = std::max<size_t>(P->hang.size(), 1) * ltsoct::kBN;
  std::vector<int32_t> hang_pos(P->N, -1);
  for (size_t h = 0; h < P->hang.size(); ++h) hang_pos[P->hang[h]] = int32_t(h);
  int *t_pos = nullptr, *t_zip = nullptr, *t_hsrc = nullptr;
  unsigned short* t_hcode = nullptr;
  auto cleanup = [&]() {
    cudaFree(t_pos);
    cudaFree(t_zip);
    cudaFree(t_hsrc);
    cudaFree(t_hcode);
  };
  cudaError_t e = cudaMalloc(&t_pos, sizeof(int) * P->N);
  if (e == cudaSuccess) e = cudaMalloc(&t_zip, sizeof(int) * nb);
  if (e == cudaSuccess) e = cudaMalloc(&t_hsrc, sizeof(int) * nh);
  if (e == cudaSuccess) e = cudaMalloc(&t_hcode, sizeof(unsigned short) * nh);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t_pos, hang_pos.data(), sizeof(int) * P->N, cudaMemcpyHostToDevice, P->stream);
  if (e == cudaSuccess) e = ltsoct::launch_nodemap(dev_tree(P), t_pos, t_zip, t_hsrc, t_hcode, P->d_err, P->stream);
  std::vector<int32_t> zip(nb), hsrc(nh);
  std::vector<uint16_t> hcode(nh);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(zip.data(), t_zip, sizeof(int) * nb, cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hsrc.data(), t_hsrc, sizeof(int) * nh, cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hcode.data(), t_hcode, sizeof(uint16_t) * nh, cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "lts_plan_create: node maps");
  if (herr) return fail(LTS_EINTERNAL, "lts_plan_create: node maps: a shared node without a valid owner");
  P->launches++;
  // boundary nodes in node order (the table of the kernels)
  int bnode[ltsoct::kBN], nbn = 0;
  for (int q = 0; q < kNV; ++q) {
    const int i = q % 7, j = (q / 7) % 7, k = q / 49;
    if (i == 0 || i == 6 || j == 0 || j == 6 || k == 0 || k == 6) bnode[nbn++] = q;
  }
  std::vector<int32_t> zl_dst, zl_src;
  for (int64_t b = 0; b < P->N; ++b)
    for (int k = 0; k < ltsoct::kBN; ++k) {
      const int32_t src = zip[size_t(b) * ltsoct::kBN + k];
      if (src < 0) continue;
      zl_dst.push_back(int32_t(b * kNV + bnode[k]));
      zl_src.push_back(src);
    }
  // hanging nodes: per level, then by the number of odd coordinates
  std::vector<int32_t> hl_dst, hl_src;
  std::vector<uint16_t> hl_code;
  for (int l = 0; l <= 32; ++l) {
    P->hl_off[l] = int64_t(hl_dst.size());
    for (int odd = 1; odd <= 3; ++odd)
      for (int64_t h = P->hang_off[l]; h < P->hang_off[l + 1]; ++h)
        for (int k = 0; k < ltsoct::kBN; ++k) {
          const size_t x = size_t(h) * ltsoct::kBN + k;
          if (hsrc[x] < 0) continue;
          const unsigned c = hcode[x];
          const int n_odd = int(c & 1u) + int((c >> 4) & 1u) + int((c >> 8) & 1u);
          if (n_odd != odd) continue;
          hl_dst.push_back(int32_t(int64_t(P->hang[h]) * kNV + bnode[k]));
          hl_src.push_back(hsrc[x]);
          hl_code.push_back(uint16_t(c));
        }
  }
  P->hl_off[33] = int64_t(hl_dst.size());
  P->n_zip = int64_t(zl_dst.size());
  P->d_zl_dst = static_cast<int*>(dev_alloc(P, sizeof(int) * std::max<size_t>(zl_dst.size(), 1)));
  P->d_zl_src = static_cast<int*>(dev_alloc(P, sizeof(int) * std::max<size_t>(zl_src.size(), 1)));
  P->d_hl_dst = static_cast<int*>(dev_alloc(P, sizeof(int) * std::max<size_t>(hl_dst.size(), 1)));
  P->d_hl_src = static_cast<int*>(dev_alloc(P, sizeof(int) * std::max<size_t>(hl_src.size(), 1)));
  P->d_hl_code = static_cast<unsigned short*>(dev_alloc(P, sizeof(uint16_t) * std::max<size_t>(hl_code.size(), 1)));
  if (!P->d_zl_dst || !P->d_zl_src || !P->d_hl_dst || !P->d_hl_src || !P->d_hl_code)
    return fail(LTS_ENOMEM, "lts_plan_create: node map allocation failed");
  if (!zl_dst.empty()) {
    CK(cudaMemcpyAsync(P->d_zl_dst, zl_dst.data(), sizeof(int) * zl_dst.size(), cudaMemcpyHostToDevice, P->stream), "copy");
    CK(cudaMemcpyAsync(P->d_zl_src, zl_src.data(), sizeof(int) * zl_src.size(), cudaMemcpyHostToDevice, P->stream), "copy");
  }
  if (!hl_dst.empty()) {
    CK(cudaMemcpyAsync(P->d_hl_dst, hl_dst.data(), sizeof(int) * hl_dst.size(), cudaMemcpyHostToDevice, P->stream), "copy");
    CK(cudaMemcpyAsync(P->d_hl_src, hl_src.data(), sizeof(int) * hl_src.size(), cudaMemcpyHostToDevice, P->stream), "copy");
    CK(cudaMemcpyAsync(P->d_hl_code, hl_code.data(), sizeof(uint16_t) * hl_code.size(), cudaMemcpyHostToDevice,
                       P->stream), "copy");
  }
  CK(cudaStreamSynchronize(P->stream), "cudaStreamSynchronize");
  return LTS_OK;
}

lts_status sync_fields(lts_plan* P, void* vb0, void* vb1, unsigned sel, int elem) {
  ltsoct::SyncArgs a{};
  a.tree = dev_tree(P);
  a.vb[0] = vb0;
  a.vb[1] = vb1;
  if (P->d_us[0] && vb0 == P->d_u[0]) {  // the FP64 state: keep its FP32 copies equal
    a.shadow[0] = P->d_us[0];
    a.shadow[1] = vb1 == P->d_u[1] ? P->d_us[1] : P->d_us[0];
  }
  a.elem = elem;
  a.sel_mask = sel;
  a.fstride = P->N * kNV;
  a.nf = P->nf;
  a.list = nullptr;
  a.count = int(P->N);
  a.err = P->d_err;
  a.map_dst = P->d_zl_dst;
  a.map_src = P->d_zl_src;
  a.map_first = 0;
  a.map_count = P->n_zip;
  CK(ltsoct::launch_sync_zip(a, P->stream), "sync (zip)");
  P->launches++;
  for (int l = P->lmin + 1; l <= P->lmax; ++l) {
    const int64_t n = P->hang_off[l + 1] - P->hang_off[l];
    if (!n) continue;
    a.list = P->d_hang + P->hang_off[l];
    a.count = int(n);
    a.map_dst = P->d_hl_dst;
    a.map_src = P->d_hl_src;
    a.map_code = P->d_hl_code;
    a.map_first = P->hl_off[l];
    a.map_count = P->hl_off[l + 1] - P->hl_off[l];
    CK(ltsoct::launch_sync_hanging(a, P->stream), "sync (hanging nodes)");
    P->launches++;
  }
  return LTS_OK;
}

// Prolongation plan of one coarser source: the class mask `cls` (bit cx + 3 cy + 9 cz)
// re-expressed in the frame of the cheapest pass order, with the order's index in
// bits 27-29 (orders as in ltsoct::kProlongOrders).  Cost model: pass 1 interpolates
// 7 x 7 source lines at each odd position of its axis, pass 2 7 lines per odd
// position of the plane it needs, pass 3 every odd point of the set, 7 multiply-adds
// each; a class spans 4 / 5 / 4 positions, two of them odd.
uint32_t prolong_plan_word(uint32_t cls, int64_t* cost_out = nullptr) {
  static const int kN[3] = {4, 5, 4}, kOdd[3] = {2, 2, 2};
  int64_t best_cost = INT64_MAX;
  uint32_t best = 0;
  for (int o = 0; o < 6; ++o) {
    const int* ax = ltsoct::kProlongOrders[o];  // pass axes a, b, c
    uint32_t m = 0;                             // mask in the (a, b, c) frame
    for (int c2 = 0; c2 < 3; ++c2)
      for (int c1 = 0; c1 < 3; ++c1)
        for (int c0 = 0; c0 < 3; ++c0) {
          int c[3];
          c[ax[0]] = c0;
          c[ax[1]] = c1;
          c[ax[2]] = c2;
          if (cls >> (c[0] + 3 * c[1] + 9 * c[2]) & 1u) m |= 1u << (c0 + 3 * c1 + 9 * c2);
        }
    int64_t cost = 0;
    for (int ca = 0; ca < 3; ++ca) {
      bool any_a = false;
      for (int cb = 0; cb < 3; ++cb) {
        bool any_ab = false;
        for (int cc = 0; cc < 3; ++cc)
          if (m >> (ca + 3 * cb + 9 * cc) & 1u) {
            any_ab = true;
            cost += int64_t(kN[ca]) * kN[cb] * kOdd[cc] * 7;
          }
        if (any_ab) cost += int64_t(kN[ca]) * kOdd[cb] * 49;
        any_a = any_a || any_ab;
      }
      if (any_a) cost += int64_t(kOdd[ca]) * 343;
    }
    if (cost < best_cost) {
      best_cost = cost;
      best = m | uint32_t(o) << 27;
    }
  }
  if (cost_out) *cost_out = best_cost;
  return best;
}

ltsoct::StageTerms terms_of(const double* row, int p) {
  ltsoct::StageTerms t{};
  for (int j = 0; j < p; ++j)
    if (row[j] != 0.0) {
      t.j[t.n] = j;
      t.w[t.n] = row[j];
      t.n++;
    }
  return t;
}

ltsoct::StageArgs stage_args(const lts_plan* P, int stage, int first, int lstar, int gts) {
  ltsoct::StageArgs a{};
  a.tree = dev_tree(P);
  a.u[0] = P->d_u[0];
  a.u[1] = P->d_u[1];
  a.us[0] = P->d_us[0];
  a.us[1] = P->d_us[1];
  a.K = P->d_K;
  a.Uin = P->d_U[stage & 1];
  a.Uout = P->d_U[(stage + 1) & 1];
  a.mixed = P->mixed;
  a.fstride = P->N * kNV;
  a.nf = P->nf;
  a.p = P->p;
  a.stage = stage;
  a.first = first;
  a.lstar = lstar;
  a.lmax = P->lmax;
  a.cur_mask = P->cur_mask;
  a.gts = gts;
  a.write_update = gts ? 0 : 1;
  a.t_b = P->t_macro + double(P->n_sub) * P->dt_f;
  a.lo = P->spec.lo;
  a.ext = P->spec.hi - P->spec.lo;
  a.pde = P->prob.pde;
  a.bc = P->prob.bc;
  a.ic = P->prob.ic;
  for (int d = 0; d < 3; ++d) a.adv[d] = P->prob.adv[d];
  for (int l = 0; l < 32; ++l) {
    const double h = a.ext / (6.0 * std::ldexp(1.0, l));
    a.lc[l].dt = gts ? P->dt_f : std::ldexp(P->dt_f, P->lmax - l);
    a.lc[l].inv12h = 1.0 / (12.0 * h);
    a.lc[l].inv12h2 = 1.0 / (12.0 * h * h);
    a.lc[l].kos = P->prob.ko_sigma / (64.0 * h);
  }
  a.om[0] = terms_of(P->tab.a[stage], P->p);
  for (int r = 1; r < 4; ++r) a.om[r] = terms_of(P->tab.omega[r][stage], P->p);
  if (stage + 1 < P->p) a.next = terms_of(P->tab.a[stage + 1], P->p);
  for (int j = 0; j < 4; ++j) {
    a.w[j] = P->tab.w[j];
    a.gamma[j] = P->tab.gamma[stage][j];
  }
  for (int i = 0; i < 32; ++i) a.icp.v[i] = P->prob.ic_params[i];
  a.err = P->d_err;
  a.up = P->d_up;
  a.up_slot = P->d_up_slot;
  a.padmap = P->d_padmap;
  a.slotmap = P->d_slotmap;
  a.inj = P->d_inj;
  a.grp = P->d_grp;
  a.gsrc = P->d_gsrc;
  a.gcode = P->d_gcode;
  a.nl_c = P->prob.nl_c;
  a.orbit = P->prob.orbit;
  for (int i = 0; i < 4; ++i) a.orb[i] = P->prob.orbit_params[i];
  a.c_s = P->tab.c[stage];
  // FP32 copies of the constants for the mixed-precision kernels
  for (int l = 0; l < 32; ++l) {
    a.cf.lc[l][0] = float(a.lc[l].kos);
    a.cf.lc[l][1] = float(a.lc[l].inv12h);
    a.cf.lc[l][2] = float(a.lc[l].inv12h2);
    a.cf.dt[l] = float(a.lc[l].dt);
  }
  for (int l = 0; l < 32; ++l)
    for (int q = 0; q < 4; ++q) {
      a.dtw.next[l][q] = q < a.next.n ? a.lc[l].dt * a.next.w[q] : 0.0;
      a.dtw.upd[l][q] = q < P->p ? a.lc[l].dt * a.w[q] : 0.0;
      a.cf.dtw_next[l][q] = float(a.dtw.next[l][q]);
      a.cf.dtw_upd[l][q] = float(a.dtw.upd[l][q]);
    }
  for (int q = 0; q < 4; ++q) {
    a.cf.w[q] = float(a.w[q]);
    a.cf.orb[q] = float(a.orb[q]);
  }
  for (int d = 0; d < 3; ++d) a.cf.adv[d] = float(a.adv[d]);
  a.cf.nl_c = float(a.nl_c);
  a.cf.lo = float(a.lo);
  a.cf.xscale = float(a.ext / (6.0 * double(int64_t(1) << ltsoct::kDepth)));
  a.cf.sources = (a.nl_c != 0.0 || a.orbit) ? 1 : 0;
  return a;
}

// prolongation of the coarser sources needed by the octants stepping in this stage:
// octants of levels [max(l* - 1, l_min), l_max - 1] with finer neighbours
lts_status launch_prolong_for(lts_plan* P, const ltsoct::StageArgs& sa, int lstar) {
  const int lo = std::max(lstar - 1, P->lmin), hi = P->lmax - 1;
  if (hi < lo) return LTS_OK;
  const int64_t first = P->up_off[lo], count = P->up_off[hi + 1] - first;
  if (count <= 0) return LTS_OK;
  ltsoct::ProlongArgs a{};
  a.tree = sa.tree;
  a.list = P->d_up_list + first;
  a.count = int(count);
  a.box = P->d_up_box;
  a.up_slot = P->d_up_slot;
  a.up = P->d_up;
  a.u[0] = sa.u[0];
  a.u[1] = sa.u[1];
  a.K = sa.K;
  a.Uin = sa.Uin;
  a.fstride = sa.fstride;
  a.nf = sa.nf;
  a.stage = sa.stage;
  a.lstar = lstar;
  a.cur_mask = sa.cur_mask;
  a.gts = sa.gts;
  a.mixed = sa.mixed;
  for (int l = 0; l < 32; ++l) a.lc[l] = sa.lc[l];
  for (int r = 0; r < 4; ++r) a.om[r] = sa.om[r];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (P->profiling) {
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    CK(cudaEventCreate(&e1), "cudaEventCreate");
    CK(cudaEventRecord(e0, P->stream), "cudaEventRecord");
  }
  CK(ltsoct::launch_prolong(a, P->stream), "prolongation kernel launch");
  P->launches++;
  if (P->profiling) {
    CK(cudaEventRecord(e1, P->stream), "cudaEventRecord");
    P->pevents.emplace_back(e0, e1);
    // FP64-equivalent work as directly evaluated: the interpolation's multiply-adds (the
    // plan's cost model, 7 per odd position) and the corrected stage inputs (one
    // multiply-add per stage term and one for the step, 343 nodes), 2 flops each
    double fma = double(P->nf) * double(P->up_cost[first + count] - P->up_cost[first]);
    if (!sa.gts) {
      for (int l = lo; l <= hi; ++l) {
        const int rel = l >= lstar ? 2 : 3;
        fma += double(P->up_off[l + 1] - P->up_off[l]) * P->nf * kNV * (sa.om[rel].n + 1);
      }
    }
    P->pevent_flops.push_back(2.0 * fma);
    P->pevent_sources.push_back(count);
  }
  return LTS_OK;
}

// the injection arguments of a stage (InjectArgs), all but the octant range
ltsoct::InjectArgs inject_args(const lts_plan* P, const ltsoct::StageArgs& sa) {
  ltsoct::InjectArgs a{};
  a.tree = sa.tree;
  a.inj = P->d_inj;
  a.u[0] = sa.u[0];
  a.u[1] = sa.u[1];
  a.us[0] = sa.us[0];
  a.us[1] = sa.us[1];
  a.K = sa.K;
  a.Uin = sa.Uin;
  a.fstride = sa.fstride;
  a.nf = sa.nf;
  a.stage = sa.stage;
  a.gts = sa.gts;
  a.mixed = sa.mixed;
  a.cur_mask = sa.cur_mask;
  for (int l = 0; l < 32; ++l) a.lc[l] = sa.lc[l];
  a.om1 = sa.om[1];
  return a;
}

// the stage inputs of the finer sources read in this stage: those on levels > lstar (a
// finer source of an active octant is on an active level; all of them under GTS)
lts_status launch_inject_for(lts_plan* P, const ltsoct::StageArgs& sa, int lstar) {
  const int lo = std::min(lstar + 1, 33);
  const int64_t first = P->dn_off[lo], count = int64_t(P->dn_list.size()) - first;
  if (count <= 0) return LTS_OK;
  ltsoct::InjectArgs a = inject_args(P, sa);
  a.list = P->d_dn_list + first;
  a.first = int(first);
  a.count = int(count);
  CK(ltsoct::launch_inject(a, P->stream), "injection kernel launch");
  P->launches++;
  return LTS_OK;
}

// one RK stage of the octants of levels >= lstar: complete sibling groups by the
// block kernel, the other octants by the stage kernel (or every octant by the stage
// kernel when blocking is off)
lts_status launch_stage_timed(lts_plan* P, const ltsoct::StageArgs& a, int lstar) {
  const int count = int(P->N - P->off[lstar]);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (P->profiling) {
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    CK(cudaEventCreate(&e1), "cudaEventCreate");
    CK(cudaEventRecord(e0, P->stream), "cudaEventRecord");
  }
  if (P->blocking) {
    ltsoct::StageArgs ab = a;
    ab.first = int(P->grp_off[lstar]);
    const int ng = int(int64_t(P->grp.size()) - P->grp_off[lstar]);
    CK(ltsoct::launch_block(ab, ng, P->stream), "block kernel launch");
    if (ng > 0) P->launches++;
    ltsoct::StageArgs as = a;
    as.list = P->d_single;
    as.first = int(P->single_off[lstar]);
    const int ns = int(int64_t(P->single.size()) - P->single_off[lstar]);
    CK(ltsoct::launch_stage(as, ns, P->stream), "stage kernel launch");
    if (ns > 0) P->launches++;
  } else {
    CK(ltsoct::launch_stage(a, count, P->stream), "stage kernel launch");
    if (count > 0) P->launches++;
  }
  if (P->profiling) {
    CK(cudaEventRecord(e1, P->stream), "cudaEventRecord");
    P->events.emplace_back(e0, e1);
    P->event_nodes.push_back(int64_t(count) * kNV);
  }
  return LTS_OK;
}

int active_level(const lts_plan* P, int64_t n) {
  for (int l = P->lmin; l <= P->lmax; ++l)
    if (n % (int64_t(1) << (P->lmax - l)) == 0) return l;
  return P->lmax;
}

lts_status lts_substep(lts_plan* P) {
  const int lstar = active_level(P, P->n_sub);
  const int first = int(P->off[lstar]);
  for (int s = 0; s < P->p; ++s) {
    const ltsoct::StageArgs sa = stage_args(P, s, first, lstar, 0);
    lts_status st = launch_prolong_for(P, sa, lstar);
    if (st != LTS_OK) return st;
    st = launch_inject_for(P, sa, lstar);
    if (st != LTS_OK) return st;
    st = launch_stage_timed(P, sa, lstar);
    if (st != LTS_OK) return st;
  }
  // the active levels completed a step: their state now lives in the other buffer
  for (int l = lstar; l <= P->lmax; ++l) P->cur_mask ^= 1u << l;
  P->n_sub++;
  if (P->n_sub == (int64_t(1) << (P->lmax - P->lmin))) {
    lts_status st = sync_fields(P, P->d_u[0], P->d_u[1], P->cur_mask, 8);
    if (st != LTS_OK) return st;
    P->t_macro += double(P->n_sub) * P->dt_f;
    P->n_sub = 0;
  }
  return LTS_OK;
}

lts_status gts_step(lts_plan* P) {
  const size_t kstride_bytes = P->es * size_t(P->nf) * P->N * kNV;
  for (int s = 0; s < P->p; ++s) {
    const ltsoct::StageArgs sa = stage_args(P, s, 0, P->lmin, 1);
    lts_status st = launch_prolong_for(P, sa, P->lmin);
    if (st != LTS_OK) return st;
    st = launch_inject_for(P, sa, P->lmin);
    if (st != LTS_OK) return st;
    st = launch_stage_timed(P, sa, P->lmin);
    if (st != LTS_OK) return st;
    void* Ks = static_cast<char*>(P->d_K) + s * kstride_bytes;
    st = sync_fields(P, Ks, Ks, 0u, int(P->es));
    if (st != LTS_OK) return st;
    if (s + 1 < P->p) {
      // the next stage's inputs were formed from the unsynchronised stage: sync them too
      void* Un = P->d_U[(s + 1) & 1];
      st = sync_fields(P, Un, Un, 0u, int(P->es));
      if (st != LTS_OK) return st;
    }
  }
  ltsoct::UpdateArgs ua{};
  ua.u[0] = P->d_u[0];
  ua.u[1] = P->d_u[1];
  ua.us[0] = P->d_us[0];
  ua.us[1] = P->d_us[1];
  ua.K = P->d_K;
  ua.mixed = P->mixed;
  ua.fstride = P->N * kNV;
  ua.nf = P->nf;
  ua.p = P->p;
  ua.scheme = P->scheme;
  ua.n = int(P->N);
  ua.oct = P->d_oct;
  ua.cur_mask = P->cur_mask;
  for (int q = 0; q < 4; ++q) {
    ua.dtw[q] = q < P->p ? P->dt_f * P->tab.w[q] : 0.0;
    ua.dtwf[q] = float(ua.dtw[q]);
  }
  CK(ltsoct::launch_update(ua, P->stream), "update kernel launch");
  P->launches++;
  for (int l = P->lmin; l <= P->lmax; ++l) P->cur_mask ^= 1u << l;
  lts_status st = sync_fields(P, P->d_u[0], P->d_u[1], P->cur_mask, 8);
  if (st != LTS_OK) return st;
  P->n_sub++;
  if (P->n_sub == (int64_t(1) << (P->lmax - P->lmin))) {
    P->t_macro += double(P->n_sub) * P->dt_f;
    P->n_sub = 0;
  }
  return LTS_OK;
}

bool supported(const lts_problem& p, std::string* why) {
  if (p.pde != LTS_PDE_ADVECTION && p.pde != LTS_PDE_WAVE) return *why = "pde must be 0 or 1", false;
  if (p.rk != 4 && p.rk != 3) return *why = "rk must be 4 or 3", false;
  if (!(p.cfl > 0.0) || !(p.ko_sigma >= 0.0)) return *why = "cfl must be > 0 and ko_sigma >= 0", false;
  if (p.bc == LTS_BC_EXACT) {
    if (p.pde == LTS_PDE_ADVECTION && p.ic != LTS_IC_ADV_GAUSS)
      return *why = "exact boundary data for advection needs ic = LTS_IC_ADV_GAUSS", false;
    if (p.pde == LTS_PDE_WAVE && p.ic != LTS_IC_WAVE_PLANAR)
      return *why = "exact boundary data for the wave equation needs ic = LTS_IC_WAVE_PLANAR", false;
  } else if (p.bc == LTS_BC_RADIATIVE) {
    if (p.pde != LTS_PDE_WAVE) return *why = "radiative boundary is for the wave equation", false;
    if (p.ic != LTS_IC_WAVE_SHELL && p.ic != LTS_IC_WAVE_PLANAR && p.ic != LTS_IC_WAVE_REST)
      return *why = "wave initial data must be LTS_IC_WAVE_SHELL, _PLANAR or _REST", false;
  } else {
    return *why = "bc must be 0 or 1", false;
  }
  if (p.precision != 0 && p.precision != 1) return *why = "precision must be 0 (FP64) or 1 (mixed)", false;
  if (p.ic == LTS_IC_WAVE_SHELL && (p.ic_params[3] < 0 || p.ic_params[3] > 4))
    return *why = "shell initial data takes at most 4 modes", false;
  if ((p.nl_c != 0.0 || p.orbit != 0) && p.pde != LTS_PDE_WAVE)
    return *why = "source terms are for the wave equation", false;
  if (p.orbit != 0 && (p.orbit != 1 || !(p.orbit_params[2] > 0.0)))
    return *why = "orbit must be 0 or 1, with width orbit_params[2] > 0", false;
  if (!std::isfinite(p.nl_c)) return *why = "nl_c must be finite", false;
  return true;
}

}  // namespace

extern "C" {

const char* lts_strerror(lts_status s) {
  switch (s) {
    case LTS_OK: return "ok";
    case LTS_EINVAL: return "invalid argument";
    case LTS_ENOMEM: return "out of memory";
    case LTS_ECUDA: return "CUDA error";
    case LTS_ETIMEOUT: return "device wait timed out";
    case LTS_EUNBALANCED: return "octree is not 2:1 balanced";
    case LTS_ESTATE: return "invalid plan state";
    case LTS_EINTERNAL: return "internal consistency check failed";
  }
  return "unknown status";
}

const char* lts_last_error(void) { return ltsoct::last_error_cstr(); }

lts_status octree_build(const lts_refine_spec* spec, lts_octree** out) {
  if (!spec || !out) return fail(LTS_EINVAL, "octree_build: null argument");
  *out = nullptr;
  try {
    const lts_refine_spec& sp = *spec;
    if (!(sp.hi > sp.lo) || sp.l_min < 0 || sp.l_max < sp.l_min || sp.l_max > ltsoct::kMaxLevel || sp.kind < 0 ||
        sp.kind > 3 || ((sp.kind == 0 || sp.kind == 3) && (sp.n_centers < 1 || sp.n_centers > 8)) ||
        (sp.kind == 3 && !(sp.band > 0.0 && sp.eps > 0.0)))
      return fail(LTS_EINVAL,
                  "octree_build: invalid refinement spec (need lo < hi, 0 <= l_min <= l_max <= 18, kind 0..3, 1..8 "
                  "centers; kind 3: band > 0, eps > 0)");
    auto* t = new lts_octree();
    t->spec = sp;
    std::string err;
    const lts_status st = ltsoct::device_octree(sp, &t->leaves, &t->nb, &err);
    if (st != LTS_OK) {
      delete t;
      return fail(st, err);
    }
    *out = t;
    return LTS_OK;
  } catch (const std::bad_alloc&) {
    return fail(LTS_ENOMEM, "octree_build: out of host memory");
  }
}

lts_status octree_size(const lts_octree* tree, int64_t* n) {
  if (!tree || !n) return fail(LTS_EINVAL, "octree_size: null argument");
  *n = int64_t(tree->leaves.size());
  return LTS_OK;
}

lts_status octree_export(const lts_octree* tree, int32_t* xyz, int32_t* level) {
  if (!tree || !xyz || !level) return fail(LTS_EINVAL, "octree_export: null argument");
  for (size_t i = 0; i < tree->leaves.size(); ++i) {
    xyz[3 * i] = tree->leaves[i].x;
    xyz[3 * i + 1] = tree->leaves[i].y;
    xyz[3 * i + 2] = tree->leaves[i].z;
    level[i] = tree->leaves[i].l;
  }
  return LTS_OK;
}

void octree_destroy(lts_octree* tree) { delete tree; }

lts_status lts_plan_create(const lts_octree* tree, const lts_problem* prob, lts_plan** out) {
  if (!tree || !prob || !out) return fail(LTS_EINVAL, "lts_plan_create: null argument");
  *out = nullptr;
  std::string why;
  if (!supported(*prob, &why)) return fail(LTS_EINVAL, "lts_plan_create: " + why);
  if (tree->leaves.empty()) return fail(LTS_EINVAL, "lts_plan_create: empty octree");
  lts_plan* P = nullptr;
  try {
    P = new lts_plan();
  } catch (const std::bad_alloc&) {
    return fail(LTS_ENOMEM, "lts_plan_create: out of host memory");
  }
  P->prob = *prob;
  P->spec = tree->spec;
  P->stream = static_cast<cudaStream_t>(prob->stream);
  if (cudaGetDevice(&P->device) != cudaSuccess) {
    delete P;
    return fail(LTS_ECUDA, "lts_plan_create: cudaGetDevice failed");
  }
  P->scheme = prob->rk == 4 ? 0 : 1;
  ltsoct::Tables rk4, rk3;
  ltsoct::make_tables(4, &rk4);
  ltsoct::make_tables(3, &rk3);
  P->tab = prob->rk == 4 ? rk4 : rk3;
  P->p = P->tab.p;
  P->nf = prob->pde == LTS_PDE_WAVE ? 2 : 1;
  P->mixed = prob->precision == 1;
  P->es = P->mixed ? sizeof(float) : sizeof(double);
  P->octs = tree->leaves;
  P->N = int64_t(P->octs.size());
  if (P->N * 27 > INT32_MAX || P->N * kNV * 4 > (int64_t(1) << 46)) {
    delete P;
    return fail(LTS_EINVAL, "lts_plan_create: octree too large");
  }
  P->lmin = 99;
  P->lmax = -1;
  for (const auto& o : P->octs) {
    P->count[o.l]++;
    P->lmin = std::min(P->lmin, int(o.l));
    P->lmax = std::max(P->lmax, int(o.l));
  }
  for (int l = 0; l <= 32; ++l) P->off[l + 1] = P->off[l] + P->count[l];
  P->nb = tree->nb;
  // octants with a coarser neighbour carry hanging nodes
  for (int64_t b = 0; b < P->N; ++b) {
    bool h = false;
    for (int d = 0; d < 27 && !h; ++d) {
      const int e = P->nb.nbr[b * 27 + d];
      h = e >= 0 && P->octs[e].l == P->octs[b].l - 1;
    }
    if (h) P->hang.push_back(int32_t(b));
  }
  for (int l = 0; l <= 32; ++l) {
    P->hang_off[l + 1] = P->hang_off[l];
    while (P->hang_off[l + 1] < int64_t(P->hang.size()) && P->octs[P->hang[P->hang_off[l + 1]]].l == l)
      P->hang_off[l + 1]++;
  }

  // coarser sources: octants with a split neighbour box.  The half-node positions
  // their finer neighbours read lie within 3 half-node units of the faces, edges
  // and corners those neighbours touch: per axis, a direction -1 / 0 / +1 covers the
  // classes {low} / {low, mid, high} / {high} of r in [0,3] / [4,8] / [9,12], so the
  // set read is a union of class boxes, kept as a 27-bit mask.  The interpolation
  // passes run in the axis order with the fewest multiply-adds for that set.
  P->up_slot.assign(P->N, -1);
  for (int64_t b = 0; b < P->N; ++b) {
    uint32_t cls = 0;
    for (int d = 0; d < 27; ++d) {
      if (d == 13 || P->nb.nbr[b * 27 + d] > -2) continue;
      const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
      for (int cz = 0; cz < 3; ++cz)
        for (int cy = 0; cy < 3; ++cy)
          for (int cx = 0; cx < 3; ++cx) {
            const int c[3] = {cx, cy, cz};
            bool in = true;
            for (int a = 0; a < 3; ++a) in = in && (dd[a] == 0 || c[a] == dd[a] + 1);
            if (in) cls |= 1u << (cx + 3 * cy + 9 * cz);
          }
    }
    if (!cls) continue;
    P->up_slot[b] = int32_t(P->up_list.size());
    P->up_list.push_back(int32_t(b));
    int64_t cost = 0;
    P->up_box.push_back(int32_t(prolong_plan_word(cls, &cost)));
    if (P->up_cost.empty()) P->up_cost.push_back(0);
    P->up_cost.push_back(P->up_cost.back() + cost);
  }
  if (P->up_cost.empty()) P->up_cost.push_back(0);
  for (int l = 0; l <= 32; ++l) {
    P->up_off[l + 1] = P->up_off[l];
    while (P->up_off[l + 1] < int64_t(P->up_list.size()) && P->octs[P->up_list[P->up_off[l + 1]]].l == l)
      P->up_off[l + 1]++;
  }
  // blocks: complete sibling groups (8 consecutive octants of one level, siblings being
  // adjacent in Morton order, whose anchors are the 8 children of one parent) that no
  // coarser leaf touches
  for (int64_t b = 0; b < P->N;) {
    const ltsoct::Oct& o = P->octs[b];
    const int32_t e = int32_t(1) << (ltsoct::kDepth - o.l);
    bool group = o.l > 0 && b + 7 < P->N && ((o.x / e) & 1) == 0 && ((o.y / e) & 1) == 0 && ((o.z / e) & 1) == 0;
    for (int c = 1; c < 8 && group; ++c) {
      const ltsoct::Oct& q = P->octs[b + c];
      group = q.l == o.l && q.x == o.x + (c & 1) * e && q.y == o.y + ((c >> 1) & 1) * e && q.z == o.z + ((c >> 2) & 1) * e;
    }
    for (int c = 0; c < 8 && group; ++c)
      for (int d = 0; d < 27 && group; ++d) {
        const int n = P->nb.nbr[(b + c) * 27 + d];
        group = n < 0 || P->octs[n].l >= o.l;
      }
    if (group) {
      P->grp.push_back(int32_t(b));
      b += 8;
    } else {
      P->single.push_back(int32_t(b));
      b += 1;
    }
  }
  for (int l = 0; l <= 32; ++l) {
    P->grp_off[l + 1] = P->grp_off[l];
    while (P->grp_off[l + 1] < int64_t(P->grp.size()) && P->octs[P->grp[P->grp_off[l + 1]]].l == l)
      P->grp_off[l + 1]++;
    P->single_off[l + 1] = P->single_off[l];
    while (P->single_off[l + 1] < int64_t(P->single.size()) && P->octs[P->single[P->single_off[l + 1]]].l == l)
      P->single_off[l + 1]++;
  }
  // the slot map packs base << 2 | kind in 32 bits: every base offset must stay below 2^29
  if (P->N * kNV >= (int64_t(1) << 29) - 4096 ||
      int64_t(P->up_list.size()) * P->nf * ltsoct::kNT >= (int64_t(1) << 29) - 4096) {
    delete P;
    return fail(LTS_EINVAL, "lts_plan_create: octree too large for the stage kernel's 32-bit source offsets "
                            "(at most 1.5 M octants and 120 k octants with finer neighbours)");
  }
  // reading of the CFL condition (Sec. 3.4): dt_f = cfl * node spacing of the finest level
  const double h_f = (P->spec.hi - P->spec.lo) / (6.0 * double(int64_t(1) << P->lmax));
  P->dt_f = prob->cfl * h_f;
  // work model (eqs. w_nuts, w_uts)
  const int L = P->lmax - P->lmin;
  for (int l = P->lmin; l <= P->lmax; ++l) {
    P->w_lts += std::ldexp(double(P->count[l]), l - P->lmin);
    P->w_gts += std::ldexp(double(P->count[l]), L);
  }
  double W[13][7], E[4][4];
  ltsoct::lagrange_7_to_13(W);
  ltsoct::cubic_extrapolation(E);
  cudaError_t ce = ltsoct::upload_tables(&rk4, &rk3, W, E);
  if (ce != cudaSuccess) {
    delete P;
    return cuda_fail(ce, "lts_plan_create: table upload");
  }
  const size_t fbytes = size_t(P->N) * kNV * sizeof(double) * P->nf;
  P->d_oct = static_cast<int4*>(dev_alloc(P, sizeof(int4) * P->N));
  P->d_nbr = static_cast<int*>(dev_alloc(P, sizeof(int) * P->N * 27));
  P->d_fine = static_cast<int*>(dev_alloc(P, sizeof(int) * std::max<size_t>(P->nb.fine.size(), 8)));
  P->d_hang = static_cast<int*>(dev_alloc(P, sizeof(int) * std::max<size_t>(P->hang.size(), 1)));
  P->d_u[0] = static_cast<double*>(dev_alloc(P, fbytes));
  P->d_u[1] = static_cast<double*>(dev_alloc(P, fbytes));
  if (P->mixed) {
    P->d_us[0] = static_cast<float*>(dev_alloc(P, fbytes / 2));
    P->d_us[1] = static_cast<float*>(dev_alloc(P, fbytes / 2));
  }
  const size_t sbytes = size_t(P->N) * kNV * P->es * P->nf;  // one stage-type field set
  P->d_K = dev_alloc(P, sbytes * P->p);
  P->d_err = static_cast<int*>(dev_alloc(P, sizeof(int) * 4));
  P->d_U[0] = dev_alloc(P, sbytes);
  P->d_U[1] = dev_alloc(P, sbytes);
  const size_t nup = std::max<size_t>(P->up_list.size(), 1);
  P->d_up_list = static_cast<int*>(dev_alloc(P, sizeof(int) * nup));
  P->d_up_box = static_cast<int*>(dev_alloc(P, sizeof(int) * nup));
  P->d_up_slot = static_cast<int*>(dev_alloc(P, sizeof(int) * P->N));
  P->d_up = dev_alloc(P, P->es * nup * P->nf * ltsoct::kNT);
  P->d_padmap = static_cast<unsigned char*>(dev_alloc(P, size_t(P->N) * ltsoct::kNT));
  P->d_slotmap = static_cast<int*>(dev_alloc(P, sizeof(int) * size_t(P->N) * 256));
  P->d_dn_slot = static_cast<int*>(dev_alloc(P, sizeof(int) * P->N));
  const size_t ng = std::max<size_t>(P->grp.size(), 1);
  P->d_grp = static_cast<int*>(dev_alloc(P, sizeof(int) * ng));
  P->d_single = static_cast<int*>(dev_alloc(P, sizeof(int) * std::max<size_t>(P->single.size(), 1)));
  P->d_gsrc = static_cast<int*>(dev_alloc(P, sizeof(int) * ng * ltsoct::kBG));
  P->d_gcode = static_cast<unsigned short*>(dev_alloc(P, sizeof(unsigned short) * ng * ltsoct::kBG));
  if (!P->d_oct || !P->d_nbr || !P->d_fine || !P->d_hang || !P->d_u[0] || !P->d_u[1] || !P->d_K || !P->d_err ||
      !P->d_U[0] || !P->d_U[1] || !P->d_up_list || !P->d_up_box || !P->d_up_slot || !P->d_up || !P->d_padmap ||
      !P->d_slotmap || !P->d_dn_slot ||
      !P->d_grp || !P->d_single || !P->d_gsrc || !P->d_gcode ||
      (P->mixed && (!P->d_us[0] || !P->d_us[1]))) {
    release(P);
    delete P;
    return fail(LTS_ENOMEM, "lts_plan_create: device allocation failed");
  }
  std::vector<int4> hoct(P->N);
  for (int64_t i = 0; i < P->N; ++i) hoct[i] = make_int4(P->octs[i].x, P->octs[i].y, P->octs[i].z, P->octs[i].l);
  cudaError_t e1 = cudaMemcpyAsync(P->d_oct, hoct.data(), sizeof(int4) * P->N, cudaMemcpyHostToDevice, P->stream);
  cudaError_t e2 = cudaMemcpyAsync(P->d_nbr, P->nb.nbr.data(), sizeof(int) * P->N * 27, cudaMemcpyHostToDevice, P->stream);
  cudaError_t e3 = P->nb.fine.empty() ? cudaSuccess
                                      : cudaMemcpyAsync(P->d_fine, P->nb.fine.data(), sizeof(int) * P->nb.fine.size(),
                                                        cudaMemcpyHostToDevice, P->stream);
  cudaError_t e4 = P->hang.empty() ? cudaSuccess
                                   : cudaMemcpyAsync(P->d_hang, P->hang.data(), sizeof(int) * P->hang.size(),
                                                     cudaMemcpyHostToDevice, P->stream);
  cudaError_t e10 = P->up_list.empty() ? cudaSuccess
                                        : cudaMemcpyAsync(P->d_up_list, P->up_list.data(), sizeof(int) * P->up_list.size(),
                                                          cudaMemcpyHostToDevice, P->stream);
  cudaError_t e11 = P->up_box.empty() ? cudaSuccess
                                       : cudaMemcpyAsync(P->d_up_box, P->up_box.data(), sizeof(int) * P->up_box.size(),
                                                         cudaMemcpyHostToDevice, P->stream);
  cudaError_t e12 = cudaMemcpyAsync(P->d_up_slot, P->up_slot.data(), sizeof(int) * P->N, cudaMemcpyHostToDevice, P->stream);

  cudaError_t e5 = cudaMemsetAsync(P->d_K, 0, sbytes * P->p, P->stream);
  cudaError_t e6 = cudaMemsetAsync(P->d_u[0], 0, fbytes, P->stream);
  cudaError_t e7 = cudaMemsetAsync(P->d_u[1], 0, fbytes, P->stream);
  cudaError_t e9 = cudaMemsetAsync(P->d_err, 0, sizeof(int) * 4, P->stream);
  cudaError_t e13 = (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && e9 == cudaSuccess)
                        ? ltsoct::launch_padmap(dev_tree(P), P->d_padmap, P->d_err, P->stream)
                        : cudaErrorInvalidValue;
  if (e13 == cudaSuccess) P->launches++;
  // finer sources: the leaves the padding maps read through child slots (marked on the
  // device), listed in level order
  std::vector<unsigned char> mark(P->N, 0);
  unsigned char* d_mark = static_cast<unsigned char*>(dev_alloc(P, std::max<size_t>(P->N, 1)));
  cudaError_t e18 = d_mark ? cudaMemsetAsync(d_mark, 0, P->N, P->stream) : cudaErrorMemoryAllocation;
  if (e18 == cudaSuccess && e13 == cudaSuccess) e18 = ltsoct::launch_finemark(dev_tree(P), P->d_padmap, d_mark, P->stream);
  if (e18 == cudaSuccess) e18 = cudaMemcpyAsync(mark.data(), d_mark, P->N, cudaMemcpyDeviceToHost, P->stream);
  if (e18 == cudaSuccess) e18 = cudaStreamSynchronize(P->stream);
  std::vector<int32_t> dn_slot(P->N, -1);
  for (int64_t b = 0; b < P->N && e18 == cudaSuccess; ++b)
    if (mark[b]) {
      dn_slot[b] = int32_t(P->dn_list.size());
      P->dn_list.push_back(int32_t(b));
    }
  for (int l = 0; l <= 32; ++l) {
    P->dn_off[l + 1] = P->dn_off[l];
    while (P->dn_off[l + 1] < int64_t(P->dn_list.size()) && P->octs[P->dn_list[P->dn_off[l + 1]]].l == l)
      P->dn_off[l + 1]++;
  }
  const size_t ndn = std::max<size_t>(P->dn_list.size(), 1);
  P->d_dn_list = static_cast<int*>(dev_alloc(P, sizeof(int) * ndn));
  P->d_inj = dev_alloc(P, P->es * ndn * P->nf * 64);
  if (e18 == cudaSuccess && (!P->d_dn_list || !P->d_inj)) e18 = cudaErrorMemoryAllocation;
  if (e18 == cudaSuccess && !P->dn_list.empty())
    e18 = cudaMemcpyAsync(P->d_dn_list, P->dn_list.data(), sizeof(int) * P->dn_list.size(), cudaMemcpyHostToDevice,
                          P->stream);
  if (e18 == cudaSuccess)
    e18 = cudaMemcpyAsync(P->d_dn_slot, dn_slot.data(), sizeof(int) * P->N, cudaMemcpyHostToDevice, P->stream);
  cudaError_t e19 = (e12 == cudaSuccess && e18 == cudaSuccess && e13 == cudaSuccess)
                        ? ltsoct::launch_slotmap(dev_tree(P), P->d_up_slot, P->d_dn_slot, P->nf, P->d_slotmap, P->d_err,
                                                 P->stream)
                        : cudaErrorInvalidValue;
  if (e19 == cudaSuccess) P->launches++;
  if (e18 == cudaSuccess) e18 = cudaStreamSynchronize(P->stream);  // dn_slot (host) goes out of scope
  cudaError_t e15 = P->grp.empty() ? cudaSuccess
                                   : cudaMemcpyAsync(P->d_grp, P->grp.data(), sizeof(int) * P->grp.size(),
                                                     cudaMemcpyHostToDevice, P->stream);
  cudaError_t e16 = P->single.empty() ? cudaSuccess
                                      : cudaMemcpyAsync(P->d_single, P->single.data(), sizeof(int) * P->single.size(),
                                                        cudaMemcpyHostToDevice, P->stream);
  cudaError_t e17 = (e13 == cudaSuccess && e15 == cudaSuccess)
                        ? ltsoct::launch_groupmap(dev_tree(P), P->d_grp, int(P->grp.size()), P->d_padmap, P->d_gsrc,
                                                  P->d_gcode, P->stream)
                        : cudaErrorInvalidValue;
  if (e17 == cudaSuccess && !P->grp.empty()) P->launches++;

  int herr = 0;
  cudaError_t e14 = cudaMemcpyAsync(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->stream);
  cudaError_t e8 = cudaStreamSynchronize(P->stream);
  for (cudaError_t e : {e1, e2, e3, e4, e5, e6, e7, e9, e10, e11, e12, e13, e15, e16, e17, e18, e19, e14, e8})
    if (e != cudaSuccess) {
      release(P);
      delete P;
      return cuda_fail(e, "lts_plan_create: upload");
    }
  if (herr) {
    release(P);
    delete P;
    return fail(LTS_EINTERNAL, "lts_plan_create: padding or slot map: a source lay outside its octant, or lacked "
                               "prolonged or injected inputs (code " + std::to_string(herr) + ")");
  }
  const lts_status st = build_node_maps(P);
  if (st != LTS_OK) {
    release(P);
    delete P;
    return st;
  }
  *out = P;
  return LTS_OK;
}

void lts_plan_destroy(lts_plan* plan) {
  if (!plan) return;
  release(plan);
  delete plan;
}

lts_status lts_plan_stats(const lts_plan* P, lts_stats* out) {
  if (!P || !out) return fail(LTS_EINVAL, "lts_plan_stats: null argument");
  std::memset(out, 0, sizeof(*out));
  out->n_octants = P->N;
  out->nf = P->nf;
  out->p = P->p;
  out->l_min = P->lmin;
  out->l_max = P->lmax;
  for (int l = 0; l < 32; ++l) out->octants_per_level[l] = P->count[l];
  out->dt_finest = P->dt_f;
  out->dt_coarsest = std::ldexp(P->dt_f, P->lmax - P->lmin);
  out->time = P->t_macro + double(P->n_sub) * P->dt_f;
  out->substep = P->n_sub;
  out->model_speedup = P->w_gts / P->w_lts;
  out->lts_work_per_macro = P->w_lts;
  out->gts_work_per_macro = P->w_gts;
  out->device_bytes = P->bytes;
  out->kernel_launches = P->launches;
  out->blocked_octants = int64_t(P->grp.size()) * 8;
  return LTS_OK;
}

// mixed precision: the FP32 copy of the (synchronised) state in buffer 0
static lts_status refresh_shadow(lts_plan* P) {
  if (!P->d_us[0]) return LTS_OK;
  CK(ltsoct::launch_narrow(P->d_u[0], P->d_us[0], int64_t(P->N) * kNV * P->nf, P->stream), "narrow kernel launch");
  P->launches++;
  return LTS_OK;
}

lts_status lts_set_initial(lts_plan* P, double t0) {
  if (!P) return fail(LTS_EINVAL, "lts_set_initial: null plan");
  ltsoct::InitArgs a{};
  a.tree = dev_tree(P);
  a.u = P->d_u[0];
  a.fstride = P->N * kNV;
  a.nf = P->nf;
  a.ic = P->prob.ic;
  a.pde = P->prob.pde;
  a.t0 = t0;
  a.lo = P->spec.lo;
  a.ext = P->spec.hi - P->spec.lo;
  for (int d = 0; d < 3; ++d) a.adv[d] = P->prob.adv[d];
  for (int i = 0; i < 32; ++i) a.icp.v[i] = P->prob.ic_params[i];
  CK(ltsoct::launch_init(a, P->stream), "init kernel launch");
  P->launches++;
  CK(cudaMemsetAsync(P->d_K, 0, size_t(P->N) * kNV * P->es * P->nf * P->p, P->stream), "memset");
  // a synchronised state is the unzip of its shared-node values (hanging nodes interpolated)
  lts_status st = sync_fields(P, P->d_u[0], P->d_u[0], 0u, 8);
  if (st != LTS_OK) return st;
  st = refresh_shadow(P);
  if (st != LTS_OK) return st;
  P->cur_mask = 0;
  P->t_macro = t0;
  P->n_sub = 0;
  return LTS_OK;
}

lts_status lts_set_state(lts_plan* P, const double* u, double t0, int on_device) {
  if (!P || !u) return fail(LTS_EINVAL, "lts_set_state: null argument");
  const size_t bytes = size_t(P->N) * kNV * sizeof(double) * P->nf;
  CK(cudaMemcpyAsync(P->d_u[0], u, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, P->stream),
     "lts_set_state copy");
  CK(cudaMemsetAsync(P->d_K, 0, size_t(P->N) * kNV * P->es * P->nf * P->p, P->stream), "memset");
  lts_status st = sync_fields(P, P->d_u[0], P->d_u[0], 0u, 8);
  if (st != LTS_OK) return st;
  st = refresh_shadow(P);
  if (st != LTS_OK) return st;
  P->cur_mask = 0;
  P->t_macro = t0;
  P->n_sub = 0;
  return LTS_OK;
}

// device-side guard failures surface at the next synchronising call
static lts_status check_device_error(lts_plan* P) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->stream), "error word read");
  CK(cudaStreamSynchronize(P->stream), "cudaStreamSynchronize");
  if (h)
    return fail(LTS_EINTERNAL, "device guard (code " + std::to_string(h) +
                                   "): bit 0 a padding source lay outside its octant, bit 1 a coarser source had no "
                                   "prolonged inputs");
  return LTS_OK;
}

// the current state of level l lives in u[cur(l)]: gather level ranges
static lts_status copy_state(lts_plan* P, const double* const* src_for_level, double* dst, int on_device) {
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t fstride = size_t(P->N) * kNV;
  for (int f = 0; f < P->nf; ++f)
    for (int l = P->lmin; l <= P->lmax; ++l) {
      if (!P->count[l]) continue;
      const size_t o = f * fstride + size_t(P->off[l]) * kNV;
      CK(cudaMemcpyAsync(dst + o, src_for_level[l] + o, size_t(P->count[l]) * kNV * sizeof(double), kind, P->stream),
         "state copy");
    }
  CK(cudaStreamSynchronize(P->stream), "cudaStreamSynchronize");
  return check_device_error(P);
}

lts_status lts_get_state(lts_plan* P, double* u, double* t, int on_device) {
  if (!P || !u) return fail(LTS_EINVAL, "lts_get_state: null argument");
  const double* src[33];
  for (int l = 0; l < 33; ++l) src[l] = P->d_u[cur_of(P, l)];
  lts_status st = copy_state(P, src, u, on_device);
  if (st == LTS_OK && t) *t = P->t_macro + double(P->n_sub) * P->dt_f;
  return st;
}

lts_status lts_get_stage(lts_plan* P, int j, double* k, int on_device) {
  if (!P || !k || j < 0 || j >= P->p) return fail(LTS_EINVAL, "lts_get_stage: bad argument");
  const size_t n = size_t(P->nf) * P->N * kNV;
  const char* base = static_cast<const char*>(P->d_K) + size_t(j) * n * P->es;
  if (!P->mixed) {
    const double* src[33];
    for (int l = 0; l < 33; ++l) src[l] = reinterpret_cast<const double*>(base);
    return copy_state(P, src, k, on_device);
  }
  double* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, n * sizeof(double), P->stream), "cudaMallocAsync");
  CK(ltsoct::launch_widen(reinterpret_cast<const float*>(base), tmp, (long long)n, P->stream), "widen");
  P->launches++;
  CK(cudaMemcpyAsync(k, tmp, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     P->stream), "stage copy");
  CK(cudaFreeAsync(tmp, P->stream), "cudaFreeAsync");
  CK(cudaStreamSynchronize(P->stream), "cudaStreamSynchronize");
  return check_device_error(P);
}

lts_status lts_run_substeps(lts_plan* P, int64_t n) {
  if (!P || n < 0) return fail(LTS_EINVAL, "lts_run_substeps: bad argument");
  for (int64_t i = 0; i < n; ++i) {
    lts_status st = lts_substep(P);
    if (st != LTS_OK) return st;
  }
  return LTS_OK;
}

lts_status lts_advance(lts_plan* P, double t_end) {
  if (!P) return fail(LTS_EINVAL, "lts_advance: null plan");
  if (P->n_sub != 0) return fail(LTS_ESTATE, "lts_advance: plan is inside a macro step");
  const double dtc = std::ldexp(P->dt_f, P->lmax - P->lmin);
  const double steps = (t_end - P->t_macro) / dtc;
  const double n = std::round(steps);
  if (n < 0 || std::fabs(steps - n) > 1e-9 * std::max(1.0, std::fabs(steps)))
    return fail(LTS_EINVAL, "lts_advance: t_end - t is not a whole number of macro steps");
  return lts_run_substeps(P, int64_t(n) << (P->lmax - P->lmin));
}

lts_status gts_steps(lts_plan* P, int64_t n) {
  if (!P || n < 0) return fail(LTS_EINVAL, "gts_steps: bad argument");
  for (int64_t i = 0; i < n; ++i) {
    lts_status st = gts_step(P);
    if (st != LTS_OK) return st;
  }
  return LTS_OK;
}

lts_status gts_advance(lts_plan* P, double t_end) {
  if (!P) return fail(LTS_EINVAL, "gts_advance: null plan");
  const double t = P->t_macro + double(P->n_sub) * P->dt_f;
  const double steps = (t_end - t) / P->dt_f;
  const double n = std::round(steps);
  if (n < 0 || std::fabs(steps - n) > 1e-9 * std::max(1.0, std::fabs(steps)))
    return fail(LTS_EINVAL, "gts_advance: t_end - t is not a whole number of steps");
  return gts_steps(P, int64_t(n));
}

lts_status lts_export_o2o(const lts_plan* P, int32_t* out) {
  if (!P || !out) return fail(LTS_EINVAL, "lts_export_o2o: null argument");
  for (int64_t b = 0; b < P->N; ++b)
    for (int d = 0; d < 27; ++d) {
      int32_t* ent = out + (b * 27 + d) * 8;
      const int e = P->nb.nbr[b * 27 + d];
      for (int c = 0; c < 8; ++c) ent[c] = -1;
      if (e == -1)
        ent[0] = -2;
      else if (e >= 0)
        ent[0] = e;
      else
        for (int c = 0; c < 8; ++c) ent[c] = P->nb.fine[(-e - 2) * 8 + c];
    }
  return LTS_OK;
}

static lts_status export_map(lts_plan* P, const int32_t* octs, int64_t n, int32_t* src, int32_t* r, int nodes) {
  if (!P || (n && (!octs || !src || !r)) || n < 0) return fail(LTS_EINVAL, "map export: bad argument");
  for (int64_t i = 0; i < n; ++i)
    if (octs[i] < 0 || octs[i] >= P->N) return fail(LTS_EINVAL, "map export: octant index out of range");
  if (!n) return LTS_OK;
  const int npts = nodes ? kNV : ltsoct::kNT;
  int *d_list = nullptr, *d_src = nullptr, *d_r = nullptr;
  CK(cudaMallocAsync(&d_list, sizeof(int) * n, P->stream), "cudaMallocAsync");
  CK(cudaMallocAsync(&d_src, sizeof(int) * n * npts, P->stream), "cudaMallocAsync");
  CK(cudaMallocAsync(&d_r, sizeof(int) * n * npts * 3, P->stream), "cudaMallocAsync");
  CK(cudaMemcpyAsync(d_list, octs, sizeof(int) * n, cudaMemcpyHostToDevice, P->stream), "copy");
  ltsoct::MapArgs a{};
  a.tree = dev_tree(P);
  a.octs = d_list;
  a.count = int(n);
  a.nodes = nodes;
  a.src = d_src;
  a.r = d_r;
  a.padmap = P->d_padmap;
  CK(ltsoct::launch_maps(a, P->stream), "map kernel launch");
  P->launches++;
  CK(cudaMemcpyAsync(src, d_src, sizeof(int) * n * npts, cudaMemcpyDeviceToHost, P->stream), "copy");
  CK(cudaMemcpyAsync(r, d_r, sizeof(int) * n * npts * 3, cudaMemcpyDeviceToHost, P->stream), "copy");
  CK(cudaFreeAsync(d_list, P->stream), "cudaFreeAsync");
  CK(cudaFreeAsync(d_src, P->stream), "cudaFreeAsync");
  CK(cudaFreeAsync(d_r, P->stream), "cudaFreeAsync");
  CK(cudaStreamSynchronize(P->stream), "cudaStreamSynchronize");
  return LTS_OK;
}

lts_status lts_export_pad_map(lts_plan* P, const int32_t* octs, int64_t n, int32_t* src, int32_t* r) {
  return export_map(P, octs, n, src, r, 0);
}

lts_status lts_export_node_map(lts_plan* P, const int32_t* octs, int64_t n, int32_t* src, int32_t* r) {
  return export_map(P, octs, n, src, r, 1);
}

// Same result as lts_export_pad_map, staged through the library's fixed device
// array instead of memory allocated per call (see include/ltsoct.h).
lts_status lts_export_pad_map_static(lts_plan* P, const int32_t* octs, int64_t n, int32_t* src, int32_t* r) {
  if (!P || n < 0 || (n && (!octs || !src || !r))) return fail(LTS_EINVAL, "lts_export_pad_map_static: bad argument");
  if (n > ltsoct::kStaticMapOctants)
    return fail(LTS_EINVAL, "lts_export_pad_map_static: at most " + std::to_string(ltsoct::kStaticMapOctants) +
                                " octants per call (got " + std::to_string(n) + ")");
  for (int64_t i = 0; i < n; ++i)
    if (octs[i] < 0 || octs[i] >= P->N) return fail(LTS_EINVAL, "lts_export_pad_map_static: octant index out of range");
  if (!n) return LTS_OK;
  // the staging array's address is per device: take it on the plan's device only
  int cur = -1;
  CK(cudaGetDevice(&cur), "cudaGetDevice");
  if (cur != P->device)
    return fail(LTS_EINVAL, "lts_export_pad_map_static: the current device (" + std::to_string(cur) +
                                ") is not the plan's device (" + std::to_string(P->device) + ")");
  int* scratch = nullptr;
  CK(ltsoct::static_map_scratch(&scratch), "lts_export_pad_map_static: staging area address");
  const int K = ltsoct::kStaticMapOctants;
  int* d_list = scratch;
  int* d_src = scratch + K;
  int* d_r = d_src + size_t(K) * ltsoct::kNT;
  CK(cudaMemcpyAsync(d_list, octs, sizeof(int) * n, cudaMemcpyHostToDevice, P->stream), "copy");
  ltsoct::MapArgs a{};
  a.tree = dev_tree(P);
  a.octs = d_list;
  a.count = int(n);
  a.nodes = 0;
  a.src = d_src;  // every element the copies below read is written by the kernel
  a.r = d_r;
  a.padmap = P->d_padmap;
  CK(ltsoct::launch_maps(a, P->stream), "map kernel launch");
  P->launches++;
  CK(cudaMemcpyAsync(src, d_src, sizeof(int) * n * ltsoct::kNT, cudaMemcpyDeviceToHost, P->stream), "copy");
  CK(cudaMemcpyAsync(r, d_r, sizeof(int) * n * ltsoct::kNT * 3, cudaMemcpyDeviceToHost, P->stream), "copy");
  CK(cudaStreamSynchronize(P->stream), "cudaStreamSynchronize");
  return LTS_OK;
}

lts_status lts_set_blocking(lts_plan* P, int on) {
  if (!P) return fail(LTS_EINVAL, "lts_set_blocking: null plan");
  P->blocking = on != 0;
  return LTS_OK;
}

lts_status lts_set_profiling(lts_plan* P, int on) {
  if (!P) return fail(LTS_EINVAL, "lts_set_profiling: null plan");
  P->profiling = on != 0;
  return LTS_OK;
}

lts_status lts_kernel_stats(lts_plan* P, int64_t* launches, double* ms, double* flops, double* bytes,
                            int64_t* node_stages, int reset) {
  if (!P) return fail(LTS_EINVAL, "lts_kernel_stats: null plan");
  lts_status dst = check_device_error(P);
  if (dst != LTS_OK) return dst;
  for (size_t i = 0; i < P->events.size(); ++i) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, P->events[i].first, P->events[i].second), "cudaEventElapsedTime");
    P->prof_ms += t;
    P->prof_launches++;
    P->prof_node_stages += P->event_nodes[i];
    cudaEventDestroy(P->events[i].first);
    cudaEventDestroy(P->events[i].second);
  }
  P->events.clear();
  P->event_nodes.clear();
  if (launches) *launches = P->prof_launches;
  if (ms) *ms = P->prof_ms;
  if (node_stages) *node_stages = P->prof_node_stages;
  if (flops) *flops = double(P->prof_node_stages) * flops_per_node_stage(P->prob.pde);
  if (bytes) *bytes = double(P->prof_node_stages) * bytes_per_node_stage(P->nf, P->mixed);
  if (reset) {
    P->prof_launches = 0;
    P->prof_node_stages = 0;
    P->prof_ms = 0.0;
  }
  return LTS_OK;
}

lts_status lts_prolong_stats(lts_plan* P, int64_t* launches, double* ms, double* flops, int64_t* sources,
                             int reset) {
  if (!P) return fail(LTS_EINVAL, "lts_prolong_stats: null plan");
  lts_status dst = check_device_error(P);
  if (dst != LTS_OK) return dst;
  for (size_t i = 0; i < P->pevents.size(); ++i) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, P->pevents[i].first, P->pevents[i].second), "cudaEventElapsedTime");
    P->pprof_ms += t;
    P->pprof_launches++;
    P->pprof_flops += P->pevent_flops[i];
    P->pprof_sources += P->pevent_sources[i];
    cudaEventDestroy(P->pevents[i].first);
    cudaEventDestroy(P->pevents[i].second);
  }
  P->pevents.clear();
  P->pevent_flops.clear();
  P->pevent_sources.clear();
  if (launches) *launches = P->pprof_launches;
  if (ms) *ms = P->pprof_ms;
  if (flops) *flops = P->pprof_flops;
  if (sources) *sources = P->pprof_sources;
  if (reset) {
    P->pprof_launches = P->pprof_sources = 0;
    P->pprof_ms = P->pprof_flops = 0.0;
  }
  return LTS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many plans advanced together, one persistent launch per stage
// ---------------------------------------------------------------------------
struct lts_batch {
  std::vector<lts_plan*> plans;
  cudaStream_t stream = nullptr;     // the plans' stream
  cudaStream_t cap = nullptr;        // stream the rounds run on (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ltsoct::BatchInst* d_inst = nullptr;
  int* d_pre = nullptr;
  ltsoct::BatchArgs args{};
  int pmax = 0, lmax_all = 0, mixed = 0;
  int grid_stage = 152 * 4, grid_prolong = 152 * 6, grid_sync = 152 * 8;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  bool slots = false;                // created empty with fixed capacity (attach / detach)
  // persistent rounds: one cooperative launch per round over `grid_persistent` CTAs (off by
  // default: the per-stage launches measured faster on the batches tested; the autotuner
  // chooses per batch)
  int persistent = 0;
  int grid_persistent = 0;           // resident CTAs (set at creation from the occupancy)
  int resident_max = 0;              // CTAs per SM x SMs the persistent kernel can keep resident
  int sms = 0;
  unsigned* d_sync = nullptr;        // [0..1] grid barrier (count, generation), [2] error word
  double barrier_limit_s = 2.0;      // a CTA waiting longer at a grid barrier ends the launch
};

namespace {

// one round's launches: the persistent round kernel, or the per-stage launch sequence
cudaError_t launch_round(lts_batch* B) {
  if (B->persistent)
    return ltsoct::launch_batch_substep(B->args, B->pmax, B->lmax_all, B->grid_persistent, B->mixed, B->d_sync,
                                        reinterpret_cast<int*>(B->d_sync + 2),
                                        static_cast<unsigned long long>(B->barrier_limit_s * 1e9), B->cap);
  return ltsoct::launch_batch_round(B->args, B->pmax, B->lmax_all, B->grid_stage, B->grid_prolong, B->grid_sync,
                                    B->mixed, B->cap);
}

lts_status batch_round(lts_batch* B, bool graph) {
  if (graph) {
    if (!B->exec) {
      CK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
      cudaError_t e = launch_round(B);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(B->cap, &g);
      if (e != cudaSuccess) return cuda_fail(e, "batch round capture");
      if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
      B->graph = g;
      CK(cudaGraphInstantiate(&B->exec, g, 0), "cudaGraphInstantiate");
    }
    CK(cudaGraphLaunch(B->exec, B->cap), "cudaGraphLaunch");
  } else {
    CK(launch_round(B), "batch round launch");
  }
  B->launches += B->persistent ? 1 : 3 + 3 * B->pmax + B->lmax_all;
  return LTS_OK;
}

void drop_graph(lts_batch* B) {
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  if (B->graph) {
    cudaGraphDestroy(B->graph);
    B->graph = nullptr;
  }
}

// the host's copy of a plan's schedule, advanced by n substeps (the same arithmetic
// the device applies in batch_round_end)
void advance_host_schedule(lts_plan* P, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    const int lstar = active_level(P, P->n_sub);
    for (int l = lstar; l <= P->lmax; ++l) P->cur_mask ^= 1u << l;
    P->n_sub++;
    if (P->n_sub == (int64_t(1) << (P->lmax - P->lmin))) {
      P->t_macro += double(P->n_sub) * P->dt_f;
      P->n_sub = 0;
    }
  }
}

}  // namespace

namespace {

// the device descriptor of plan P in a batch
ltsoct::BatchInst batch_descriptor(lts_plan* P) {
  ltsoct::BatchInst I;
  std::memset(&I, 0, sizeof(I));
  for (int s = 0; s < 4; ++s) {
    const int ss = std::min(s, P->p - 1);
    I.st[s] = stage_args(P, ss, 0, P->lmin, 0);
    ltsoct::ProlongArgs& a = I.pr[s];
    a.tree = I.st[s].tree;
    a.box = P->d_up_box;
    a.up_slot = P->d_up_slot;
    a.up = P->d_up;
    a.u[0] = P->d_u[0];
    a.u[1] = P->d_u[1];
    a.K = P->d_K;
    a.Uin = I.st[s].Uin;
    a.fstride = P->N * kNV;
    a.nf = P->nf;
    a.stage = ss;
    a.gts = 0;
    a.mixed = P->mixed;
    for (int l = 0; l < 32; ++l) a.lc[l] = I.st[s].lc[l];
    for (int r = 0; r < 4; ++r) a.om[r] = I.st[s].om[r];
    I.in[s] = inject_args(P, I.st[s]);  // octant range and schedule set per round on the device
  }
  for (ltsoct::SyncArgs* y : {&I.zip, &I.hang}) {
    y->tree = I.st[0].tree;
    y->vb[0] = P->d_u[0];
    y->vb[1] = P->d_u[1];
    y->shadow[0] = P->d_us[0];
    y->shadow[1] = P->d_us[1];
    y->elem = 8;
    y->fstride = P->N * kNV;
    y->nf = P->nf;
    y->list = nullptr;
    y->err = P->d_err;
  }
  I.up_list = P->d_up_list;
  I.hang_list = P->d_hang;
  I.dn_list = P->d_dn_list;
  for (int l = 0; l < 34; ++l) {
    I.off[l] = int(P->off[l]);
    I.up_off[l] = int(P->up_off[l]);
    I.hang_off[l] = int(P->hang_off[l]);
    I.dn_off[l] = int(P->dn_off[l]);
  }
  I.n = int(P->N);
  I.nf = P->nf;
  I.p = P->p;
  I.lmin = P->lmin;
  I.lmax = P->lmax;
  I.nsub_macro = int64_t(1) << (P->lmax - P->lmin);
  I.n_sub = P->n_sub;
  I.t_macro = P->t_macro;
  I.dt_f = P->dt_f;
  I.cur_mask = P->cur_mask;
  return I;
}

lts_status batch_alloc(lts_batch* B, int n_slots) {
  const size_t pre_ints = size_t(ltsoct::kMaxBatch + 1) * (4 + 4 + 4 + 1 + ltsoct::kMaxLevel + 2) + 12;
  std::vector<ltsoct::BatchInst> empty(n_slots);
  std::memset(empty.data(), 0, sizeof(ltsoct::BatchInst) * n_slots);
  cudaError_t e = ltsoct::prepare_batch_kernels();
  if (e == cudaSuccess) e = cudaMalloc(&B->d_inst, sizeof(ltsoct::BatchInst) * n_slots);
  if (e == cudaSuccess) e = cudaMalloc(&B->d_pre, sizeof(int) * pre_ints);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_inst, empty.data(), sizeof(ltsoct::BatchInst) * n_slots, cudaMemcpyHostToDevice, B->cap);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_pre, 0, sizeof(int) * pre_ints, B->cap);
  if (e == cudaSuccess) e = cudaMalloc(&B->d_sync, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_sync, 0, 4 * sizeof(unsigned), B->cap);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->cap);
  int per_sm = 0;
  if (e == cudaSuccess) e = ltsoct::batch_substep_resident(B->mixed, &per_sm, &B->sms);
  if (e != cudaSuccess) return cuda_fail(e, "batch allocation");
  B->resident_max = per_sm * B->sms;
  B->grid_persistent = B->resident_max;
  B->plans.assign(n_slots, nullptr);
  B->args.inst = B->d_inst;
  B->args.n = n_slots;
  B->args.stage_pre = B->d_pre;
  B->args.prol_pre = B->d_pre + 4 * (ltsoct::kMaxBatch + 1);
  B->args.inj_pre = B->d_pre + 8 * (ltsoct::kMaxBatch + 1);
  B->args.zip_pre = B->d_pre + 12 * (ltsoct::kMaxBatch + 1);
  B->args.hang_pre = B->d_pre + 13 * (ltsoct::kMaxBatch + 1);
  B->args.next_item = B->d_pre + (ltsoct::kMaxBatch + 1) * (4 + 4 + 4 + 1 + ltsoct::kMaxLevel + 2);
  return LTS_OK;
}

}  // namespace

extern "C" {

lts_status lts_batch_create_slots(int n_slots, void* stream, int precision, lts_batch** out) {
  if (!out || n_slots < 1 || n_slots > ltsoct::kMaxBatch || (precision != 0 && precision != 1))
    return fail(LTS_EINVAL, "lts_batch_create_slots: 1..1024 slots, precision 0 or 1");
  *out = nullptr;
  lts_batch* B = new (std::nothrow) lts_batch();
  if (!B) return fail(LTS_ENOMEM, "lts_batch_create_slots: out of host memory");
  B->stream = static_cast<cudaStream_t>(stream);
  B->mixed = precision;
  B->pmax = 4;                       // every stage and every level is launched, so that
  B->lmax_all = ltsoct::kMaxLevel;   // one captured round serves any membership
  B->slots = true;
  lts_status st = batch_alloc(B, n_slots);
  if (st != LTS_OK) {
    lts_batch_destroy(B);
    return st;
  }
  *out = B;
  return LTS_OK;
}

lts_status lts_batch_attach(lts_batch* B, int slot, lts_plan* P) {
  if (!B || !P || slot < 0 || slot >= int(B->plans.size())) return fail(LTS_EINVAL, "lts_batch_attach: bad argument");
  if (B->plans[slot]) return fail(LTS_ESTATE, "lts_batch_attach: slot is occupied");
  if (P->stream != B->stream || P->mixed != B->mixed)
    return fail(LTS_EINVAL, "lts_batch_attach: the plan's stream or precision differs from the batch's");
  if (!B->slots && (P->p > B->pmax || P->lmax > B->lmax_all))
    return fail(LTS_EINVAL, "lts_batch_attach: plan needs more stages or levels than the batch launches");
  ltsoct::BatchInst I = batch_descriptor(P);
  // ordered after the plan's own work and after earlier rounds
  CK(cudaEventRecord(B->ev_in, B->stream), "cudaEventRecord");
  CK(cudaStreamWaitEvent(B->cap, B->ev_in, 0), "cudaStreamWaitEvent");
  CK(cudaMemcpyAsync(B->d_inst + slot, &I, sizeof(I), cudaMemcpyHostToDevice, B->cap), "copy");
  CK(cudaStreamSynchronize(B->cap), "cudaStreamSynchronize");
  B->plans[slot] = P;
  return LTS_OK;
}

lts_status lts_batch_detach(lts_batch* B, int slot) {
  if (!B || slot < 0 || slot >= int(B->plans.size())) return fail(LTS_EINVAL, "lts_batch_detach: bad argument");
  ltsoct::BatchInst I;
  std::memset(&I, 0, sizeof(I));
  CK(cudaMemcpyAsync(B->d_inst + slot, &I, sizeof(I), cudaMemcpyHostToDevice, B->cap), "copy");
  CK(cudaStreamSynchronize(B->cap), "cudaStreamSynchronize");
  B->plans[slot] = nullptr;
  return LTS_OK;
}

lts_status lts_batch_create(lts_plan* const* plans, int n, lts_batch** out) {
  if (!plans || !out || n < 1 || n > ltsoct::kMaxBatch) return fail(LTS_EINVAL, "lts_batch_create: 1..1024 plans");
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!plans[i] || plans[i]->stream != plans[0]->stream || plans[i]->mixed != plans[0]->mixed)
      return fail(LTS_EINVAL, "lts_batch_create: plans must be valid and share one stream and one precision");
  lts_batch* B = new (std::nothrow) lts_batch();
  if (!B) return fail(LTS_ENOMEM, "lts_batch_create: out of host memory");
  B->stream = plans[0]->stream;
  B->mixed = plans[0]->mixed;
  for (int i = 0; i < n; ++i) {
    B->pmax = std::max(B->pmax, plans[i]->p);
    B->lmax_all = std::max(B->lmax_all, plans[i]->lmax);
  }
  lts_status st = batch_alloc(B, n);
  for (int i = 0; st == LTS_OK && i < n; ++i) st = lts_batch_attach(B, i, plans[i]);
  if (st != LTS_OK) {
    lts_batch_destroy(B);
    return st;
  }
  *out = B;
  return LTS_OK;
}

void lts_batch_destroy(lts_batch* B) {
  if (!B) return;
  if (B->cap) cudaStreamSynchronize(B->cap);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  if (B->ev_out) cudaEventDestroy(B->ev_out);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->d_inst) cudaFree(B->d_inst);
  if (B->d_pre) cudaFree(B->d_pre);
  if (B->d_sync) cudaFree(B->d_sync);
  delete B;
}

lts_status lts_batch_set_grid(lts_batch* B, int grid_stage, int grid_prolong, int grid_sync) {
  if (!B || grid_stage < 1 || grid_prolong < 1 || grid_sync < 1) return fail(LTS_EINVAL, "lts_batch_set_grid: bad argument");
  B->grid_stage = grid_stage;
  B->grid_prolong = grid_prolong;
  B->grid_sync = grid_sync;
  drop_graph(B);
  return LTS_OK;
}

lts_status lts_batch_set_mode(lts_batch* B, int persistent, int ctas_per_sm) {
  if (!B || (persistent != 0 && persistent != 1)) return fail(LTS_EINVAL, "lts_batch_set_mode: bad argument");
  if (persistent) {
    if (ctas_per_sm < 1 || ctas_per_sm * B->sms > B->resident_max)
      return fail(LTS_EINVAL, "lts_batch_set_mode: " + std::to_string(ctas_per_sm) +
                                  " CTAs per SM; the persistent round kernel keeps at most " +
                                  std::to_string(B->sms ? B->resident_max / B->sms : 0) + " resident");
    B->grid_persistent = ctas_per_sm * B->sms;
  }
  B->persistent = persistent;
  drop_graph(B);
  return LTS_OK;
}

lts_status lts_batch_wait(lts_batch* B) {
  if (!B) return fail(LTS_EINVAL, "lts_batch_wait: null batch");
  unsigned w[4] = {0, 0, 0, 0};
  CK(cudaStreamSynchronize(B->cap), "cudaStreamSynchronize");
  CK(cudaMemcpy(w, B->d_sync, sizeof(w), cudaMemcpyDeviceToHost), "error word read");
  if (w[2] & unsigned(ltsoct::kErrTimeout)) {
    CK(cudaMemset(B->d_sync, 0, sizeof(w)), "error word reset");
    return fail(LTS_ETIMEOUT, "lts_batch_wait: a grid barrier of a persistent round waited longer than " +
                                  std::to_string(B->barrier_limit_s) + " s; the round was abandoned");
  }
  return LTS_OK;
}

lts_status lts_batch_probe_barrier(lts_batch* B, int absent_cta, double limit_s) {
  if (!B || !(limit_s > 0.0) || limit_s > 60.0 || absent_cta < -1 || absent_cta >= B->sms)
    return fail(LTS_EINVAL, "lts_batch_probe_barrier: bad argument");
  CK(cudaStreamSynchronize(B->cap), "cudaStreamSynchronize");
  CK(cudaMemset(B->d_sync, 0, 4 * sizeof(unsigned)), "barrier reset");
  CK(ltsoct::launch_barrier_probe(B->sms, B->d_sync, reinterpret_cast<int*>(B->d_sync + 2),
                                  static_cast<unsigned long long>(limit_s * 1e9), absent_cta, B->cap),
     "barrier probe launch");
  const double keep = B->barrier_limit_s;
  B->barrier_limit_s = limit_s;
  lts_status st = lts_batch_wait(B);
  B->barrier_limit_s = keep;
  return st;
}

lts_status lts_batch_run(lts_batch* B, const int64_t* substeps, int use_graph) {
  if (!B || !substeps) return fail(LTS_EINVAL, "lts_batch_run: null argument");
  const int n = int(B->plans.size());
  int64_t rounds = 0;
  for (int i = 0; i < n; ++i) {
    if (substeps[i] < 0) return fail(LTS_EINVAL, "lts_batch_run: negative substep count");
    if (substeps[i] > 0 && !B->plans[i]) return fail(LTS_EINVAL, "lts_batch_run: substeps for an empty slot");
    rounds = std::max(rounds, substeps[i]);
  }
  // the plans' work so far precedes the rounds
  CK(cudaEventRecord(B->ev_in, B->stream), "cudaEventRecord");
  CK(cudaStreamWaitEvent(B->cap, B->ev_in, 0), "cudaStreamWaitEvent");
  for (int i = 0; i < n; ++i) {
    ltsoct::BatchInst* I = B->d_inst + i;
    lts_plan* P = B->plans[i];
    if (!P) continue;
    // the host schedule of the plan is authoritative at the start of a run
    const long long nsub = P->n_sub, rem = substeps[i];
    const double tm = P->t_macro;
    const unsigned cm = P->cur_mask;
    CK(cudaMemcpyAsync(&I->n_sub, &nsub, sizeof(nsub), cudaMemcpyHostToDevice, B->cap), "copy");
    CK(cudaMemcpyAsync(&I->remaining, &rem, sizeof(rem), cudaMemcpyHostToDevice, B->cap), "copy");
    CK(cudaMemcpyAsync(&I->t_macro, &tm, sizeof(tm), cudaMemcpyHostToDevice, B->cap), "copy");
    CK(cudaMemcpyAsync(&I->cur_mask, &cm, sizeof(cm), cudaMemcpyHostToDevice, B->cap), "copy");
    CK(cudaStreamSynchronize(B->cap), "cudaStreamSynchronize");  // host sources go out of scope
  }
  for (int64_t r = 0; r < rounds; ++r) {
    lts_status st = batch_round(B, use_graph != 0);
    if (st != LTS_OK) return st;
  }
  CK(cudaEventRecord(B->ev_out, B->cap), "cudaEventRecord");
  CK(cudaStreamWaitEvent(B->stream, B->ev_out, 0), "cudaStreamWaitEvent");
  for (int i = 0; i < n; ++i)
    if (B->plans[i]) advance_host_schedule(B->plans[i], substeps[i]);
  return LTS_OK;
}

lts_status lts_batch_stats(const lts_batch* B, int64_t* launches, int* grid_stage, int* grid_prolong, int* grid_sync) {
  if (!B) return fail(LTS_EINVAL, "lts_batch_stats: null batch");
  if (launches) *launches = B->launches;
  if (grid_stage) *grid_stage = B->persistent ? B->grid_persistent : B->grid_stage;
  if (grid_prolong) *grid_prolong = B->grid_prolong;
  if (grid_sync) *grid_sync = B->grid_sync;
  return LTS_OK;
}

}  // extern "C"
