// Device-side argument blocks and launchers of libltsoct (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ltsoct_internal.h"

namespace ltsoct {

struct DevTree {
  const int4* oct;   // (x, y, z, level), level order
  const int* nbr;    // [N][27]
  const int* fine;   // [F][8]
  int n;
};

struct IcParams {
  double v[32];
};

// One RK stage over the active octants [first, n) (Alg. 2 compute_stage, or
// Alg. 1 when gts != 0).
// constants of one refinement level, computed on the host
struct LevelConst {
  double dt;       // step of the level (dt_f for every level under GTS)
  double inv12h;   // 1 / (12 h), h the node spacing
  double inv12h2;  // 1 / (12 h^2)
  double kos;      // Kreiss-Oliger factor sigma / (64 h)
};

// a weighted sum of RK stages: sum_t w[t] K_j[t]
struct StageTerms {
  int n;
  int j[4];
  double w[4];
};

// FP32 copies of the per-stage constants, used by the mixed-precision kernels so that
// no node converts an FP64 constant (conversions share GB300's small FP64 pipe)
struct StageConstF {
  float lc[32][3];       // per level: kos, inv12h, inv12h2
  float dt[32];          // per level: dt
  float dtw_next[32][4]; // per level: dt * the weights of the next stage input (StageArgs::next)
  float dtw_upd[32][4];  // per level: dt * the RK weights
  float w[4];            // RK weights
  float adv[3];
  float nl_c;
  float orb[4];          // orbit radius, angular speed, width, amplitude
  float lo, xscale;      // x = lo + xscale * (lattice6 coordinate)
  int sources;           // 1: the wave equation has source terms
};

// per level l: dt_l times the weights of the next stage input (next[l][q] for the
// terms of StageArgs::next) and of the RK update (upd[l][j])
struct StageWeights {
  double next[32][4];
  double upd[32][4];
};

struct StageArgs {
  DevTree tree;
  double* u[2];          // double-buffered state [nf][N][343]; level l uses u[(cur_mask >> l) & 1]
  void* K;               // RK stages [p][nf][N][343] (stage type: double, or float when mixed)
  const void* Uin;       // stage inputs of this stage (stage >= 1), [nf][N][343], stage type
  void* Uout;            // stage inputs of the next stage, written by the epilogue, stage type
  long long fstride;     // N * 343
  int nf, p, stage;
  int first;             // first active octant (level order)
  int lstar, lmax;       // coarsest active level, finest level
  unsigned cur_mask;
  int gts;               // 1: every octant steps with dt_f and the same-level tableau
  int write_update;      // 1: the last stage also writes u_new into the other buffer
  double t_b;            // start time of the steps in this substep
  double lo, ext;        // domain [lo, lo + ext]^3
  int pde, bc, ic;
  double adv[3];
  LevelConst lc[32];
  StageTerms om[4];      // this stage's correction terms per relation (eqs. fc_1, fc_2)
  StageTerms next;       // a[stage+1][.] terms of the next stage input
  StageWeights dtw;      // the same and the RK weights, times dt of each level
  double w[4];           // RK weights
  double gamma[4];       // gamma[stage][.] for exact boundary data
  IcParams icp;
  int* err;              // device error word: bit 0 source coordinate out of range, bit 1 a coarser
                         // source without prolonged inputs
  const void* up;        // prolonged stage inputs of coarser sources, [slot][nf][2197], stage type
  int mixed;             // 1: FP32 stages, tile and right-hand side; FP64 state and corrections
  float* us[2];          // mixed: FP32 copies of u[2], kept equal to float(u) (stage inputs read them)
  const int* up_slot;    // slot of an octant in `up` (-1: not a coarser source)
  const unsigned char* padmap;  // [N][2197]: slot of the source of every padded point in the neighbour view
  const int* slotmap;    // [N][256]: per octant and slot, base << 2 | kind (built once per plan)
  const void* inj;       // finer sources' stage inputs at their even nodes, [slot][nf][64], stage type
  const int* list;         // stage_kernel: work item x is octant list[first + x] (nullptr: first + x)
  // block kernel (Sec. 3.2.5 octree-to-block decomposition): CTA x steps the complete
  // sibling group grp[first + x] (8 consecutive octants) as one 13^3-node block
  const int* grp;
  const int* gsrc;               // [G][kBG] source octant of every ghost point of a block tile (-1: exterior)
  const unsigned short* gcode;   // [G][kBG] rx | ry << 4 | rz << 8 | (level diff + 1) << 12 | exterior << 15
  // wave source terms (eq. phi and the orbiting Gaussians); c_s is this stage's node
  double nl_c;
  int orbit;
  double orb[4];         // radius, angular speed, width, amplitude
  double c_s;
  StageConstF cf;
};

// Prolongation of the stage inputs of coarser sources (Fig. unzip, coarse -> fine)
// for one stage: every listed octant has finer neighbours; its time-corrected
// stage inputs (eqs. fc_1 / fc_2) are interpolated to the half-node positions of
// the box its finer neighbours read.
struct ProlongArgs {
  DevTree tree;
  const int* list;       // octants to process (level order)
  int count;
  const int* box;        // per slot: class mask of the half-node positions read (27 bits, in the
                         // frame of the pass order) | pass order << 27 (kProlongOrders)
  const int* up_slot;
  void* up;
  const double* u[2];
  const void* K;
  const void* Uin;
  long long fstride;
  int nf, stage, lstar;
  int mixed;
  unsigned cur_mask;
  int gts;
  LevelConst lc[32];
  StageTerms om[4];
};

// Stage inputs of finer sources (Fig. unzip, fine -> coarse injection) for one stage:
// every listed octant is a finer leaf some coarser octant's padding map reads; its stage
// inputs at its 64 even nodes (the points a coarser octant's padded block can hold) are
// formed once, with the coarse <- fine time correction of eq. fc_1 under LTS (FP64), or
// copied from the stage inputs under GTS, into inj[first + item][nf][64].
struct InjectArgs {
  DevTree tree;
  const int* list;       // octants to process (level order): finer-source list entries [first, first + count)
  int first, count;
  void* inj;
  const double* u[2];
  const float* us[2];
  const void* K;
  const void* Uin;
  long long fstride;
  int nf, stage, gts, mixed;
  unsigned cur_mask;
  LevelConst lc[32];
  StageTerms om1;        // this stage's correction terms for a finer source (relation 1)
};

// axis orders of the three interpolation passes of the prolongation
constexpr int kProlongOrders[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct SyncArgs {
  DevTree tree;
  void* vb[2];           // level l's array is vb[(sel_mask >> l) & 1]
  int elem;              // element size of the arrays: 8 (double) or 4 (float)
  unsigned sel_mask;
  long long fstride;
  int nf;
  const int* list;       // octants to process (hanging pass), or nullptr = [0, n)
  int count;
  int* err;
  float* shadow[2];      // FP64 state in mixed precision: its FP32 copies, written with it (or nullptr)
  // the plan's compact node maps (map_dst nullptr: sources resolved per node); a launch
  // handles entries [map_first, map_first + map_count)
  const int* map_dst;              // destination element (octant * 343 + node)
  const int* map_src;              // zip: source element; hanging: source octant
  const unsigned short* map_code;  // hanging: half-node code rx | ry << 4 | rz << 8
  long long map_first, map_count;
};

constexpr int kBN = 343 - 125;     // boundary nodes of an octant (on its faces)

struct UpdateArgs {
  double* u[2];
  float* us[2];          // mixed: FP32 copies of u
  const void* K;         // stage type
  int mixed;
  long long fstride;
  int nf, p, scheme;
  int n;
  const int4* oct;
  unsigned cur_mask;
  double dtw[4];         // dt_f times the RK weights
  float dtwf[4];         // the same in FP32 (mixed precision)
};

struct InitArgs {
  DevTree tree;
  double* u;             // [nf][N][343]
  long long fstride;
  int nf, ic, pde;
  double t0, lo, ext;
  double adv[3];
  IcParams icp;
};

struct MapArgs {
  DevTree tree;
  const int* octs;
  int count;
  int nodes;             // 0: 2197 padded points, 1: 343 nodes
  int* src;
  int* r;
  const unsigned char* padmap;  // padding maps: decode this plan's padding map (nullptr: resolve)
};

// ---- batches: many instances advanced together ------------------------------
// Device-resident descriptor of one instance of a batch.  The static parts are
// written by the host at batch creation; the schedule fields are advanced on the
// device by batch_round_begin / batch_round_end, so that a round is a fixed
// sequence of launches (capturable in a CUDA graph).
struct BatchInst {
  StageArgs st[4];       // per stage
  ProlongArgs pr[4];     // per stage
  InjectArgs in[4];      // per stage
  SyncArgs zip, hang;    // reconcile of the state at the end of a macro step
  const int* up_list;
  const int* hang_list;
  const int* dn_list;    // finer sources of the padding maps (level order)
  int off[34];           // level offsets (level order)
  int up_off[34];        // per-level ranges of up_list
  int hang_off[34];      // per-level ranges of hang_list
  int dn_off[34];        // per-level ranges of dn_list
  int n, nf, p, lmin, lmax;
  long long nsub_macro;  // substeps per macro step, 2^(lmax - lmin)
  // schedule state
  long long n_sub;       // substep index within the macro step
  long long remaining;   // substeps still to run
  double t_macro, dt_f;
  unsigned cur_mask;
  int lstar, active, reconcile;
};

constexpr int kMaxBatch = 1024;

struct BatchArgs {
  BatchInst* inst;
  int n;
  int* stage_pre;        // [4][kMaxBatch + 1]: prefix sums of the active octants of each stage
  int* prol_pre;         // [4][kMaxBatch + 1]: prefix sums of the octants to prolong
  int* inj_pre;          // [4][kMaxBatch + 1]: prefix sums of the finer sources to inject
  int* zip_pre;          // [kMaxBatch + 1]: octants of instances that reconcile this round
  int* hang_pre;         // [kMaxLevel + 2][kMaxBatch + 1]: their hanging-node octants per level
  int* next_item;        // [3][4]: next unclaimed work item of the prolong / stage / injection work of
                         // each stage, zeroed by batch_round_begin
};

cudaError_t prepare_batch_kernels();  // outside any stream capture
cudaError_t launch_batch_round(const BatchArgs& a, int pmax, int lmax_all, int grid_stage, int grid_prolong,
                               int grid_sync, int mixed, cudaStream_t s);
// persistent rounds: one cooperative launch per round, phases separated by a grid barrier
// with a time limit (kErrTimeout in *err when a CTA waited longer than limit_ns)
constexpr int kErrTimeout = 1 << 4;
cudaError_t batch_substep_resident(int mixed, int* per_sm, int* sms);  // CTAs per SM and SMs
cudaError_t launch_batch_substep(const BatchArgs& a, int pmax, int lmax_all, int grid, int mixed, unsigned* bar,
                                 int* err, unsigned long long limit_ns, cudaStream_t s);
cudaError_t launch_barrier_probe(int grid, unsigned* bar, int* err, unsigned long long limit_ns, int absent,
                                 cudaStream_t s);

cudaError_t upload_tables(const Tables* rk4, const Tables* rk3, const double W[13][7], const double E[4][4]);
cudaError_t launch_stage(const StageArgs& a, int count, cudaStream_t s);
cudaError_t launch_block(const StageArgs& a, int count, cudaStream_t s);
cudaError_t launch_groupmap(const DevTree& t, const int* grp, int count, const unsigned char* padmap, int* gsrc,
                            unsigned short* gcode, cudaStream_t s);
constexpr int kBW = 19;               // padded block width of a sibling group: 13 nodes + 2 x 3
constexpr int kBT = kBW * kBW * kBW;  // 6859 padded points
constexpr int kBG = kBT - 13 * 13 * 13;  // 4662 of them outside the block's 13^3 nodes
cudaError_t launch_prolong(const ProlongArgs& a, cudaStream_t s);
cudaError_t launch_sync_zip(const SyncArgs& a, cudaStream_t s);
cudaError_t launch_sync_hanging(const SyncArgs& a, cudaStream_t s);
cudaError_t launch_nodemap(const DevTree& t, const int* hang_pos, int* zipmap, int* hang_src,
                           unsigned short* hang_code, int* err, cudaStream_t s);
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s);
cudaError_t launch_init(const InitArgs& a, cudaStream_t s);
cudaError_t launch_maps(const MapArgs& a, cudaStream_t s);
cudaError_t launch_padmap(const DevTree& t, unsigned char* out, int* err, cudaStream_t s);
cudaError_t launch_finemark(const DevTree& t, const unsigned char* padmap, unsigned char* mark, cudaStream_t s);
cudaError_t launch_slotmap(const DevTree& t, const int* up_slot, const int* dn_slot, int nf, int* out, int* err,
                           cudaStream_t s);
cudaError_t launch_inject(const InjectArgs& a, cudaStream_t s);
cudaError_t launch_widen(const float* in, double* out, long long n, cudaStream_t s);
cudaError_t launch_narrow(const double* in, float* out, long long n, cudaStream_t s);

// allocation-free padding-map export: largest octant list one call accepts
constexpr int kStaticMapOctants = 32;
cudaError_t static_map_scratch(int** out);

}  // namespace ltsoct
