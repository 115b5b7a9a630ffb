/*
 * ltsoct.h -- C ABI of libltsoct: local timestepping (LTS) for explicit RK solves
 * on 2:1-balanced, Morton-ordered octrees, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Fernando & Sundar, "Scalable Local Timestepping on Octree Grids"
 * (arXiv 2011.10570).  The hot path is the per-level LTS substep: unzip every
 * active octant into a padded 13^3 block (Sec. 3.3, Fig. unzip) with ghost values
 * from same-level, coarser (Lagrange interpolation) and finer (injection)
 * neighbours, corrected in time by the stage relations of eqs. rk_crrection,
 * fc_1 and fc_2; evaluate the finite-difference right-hand side; apply the RK
 * stage update (eq. rk_schemes); zip back (Sec. 3.3, Fig. dg_to_cg).
 *
 * Conventions used by every entry point
 *  - Octants are stored in "level order": ascending (level, Morton key).
 *  - Node layout: 7 nodes per axis (element order 6); node (i,j,k) has index
 *    i + 7 j + 49 k.  A state array is [nf][N][343] FP64, nf = 1 (advection: u)
 *    or 2 (wave: chi, phi), in level order ("DG" layout: every octant keeps
 *    its own copy of shared face nodes, Fig. dg_to_cg).
 *  - Lattice: anchors are integers in [0, 2^20)^3; an octant of level l has edge
 *    2^(20-l).  Physical x = lo + (hi - lo) * X / 2^20 on every axis.
 *  - Every call returns an lts_status.  No call aborts or throws across the ABI.
 *    On failure, lts_last_error() returns a thread-local message.
 *  - Work is enqueued on the plan's CUDA stream (lts_problem.stream, NULL = the
 *    legacy default stream).  Calls that return host data synchronise it.
 *  - Device memory is allocated through lts_problem.dev_alloc/dev_free when given
 *    (e.g. PyTorch's caching allocator), else with cudaMalloc/cudaFree.  The
 *    library owns all device state; the caller owns every buffer it passes in.
 *  - A plan is not thread-safe: one host thread drives it at a time.
 */
#ifndef LTSOCT_H
#define LTSOCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LTS_OK = 0,
  LTS_EINVAL = 1,      /* invalid argument (size, level range, time not on the step grid, ...) */
  LTS_ENOMEM = 2,      /* host or device allocation failed */
  LTS_ECUDA = 3,       /* a CUDA runtime call failed (message in lts_last_error) */
  LTS_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
  LTS_EUNBALANCED = 5, /* octree violates the 2:1 balance the method needs */
  LTS_ESTATE = 6,      /* call not valid in the plan's current state */
  LTS_EINTERNAL = 7    /* a device-side consistency check failed */
} lts_status;

typedef struct lts_octree lts_octree;
typedef struct lts_plan lts_plan;

/* Refinement (Sec. 3.2.2).  The paper refines by a wavelet criterion; this
 * library uses an integer geometric predicate so that trees are reproducible
 * bit for bit: an octant of level l < l_max is split if
 *   kind 0: its closed box comes within `radius` of any of the n_centers points;
 *   kind 1: its closed box meets the shell radius-band <= |x - centers[0]| <= radius+band;
 *   kind 2: its closed box comes within `band` of the circle of `radius` around
 *           centers[0] in the plane z = centers[0].z (distance evaluated in IEEE
 *           doubles from the box's exact lattice extents, no contraction);
 *   kind 3: the wavelet criterion the paper uses: the largest wavelet coefficient of the
 *           field f(x) = sum_c exp(-(|x - centers[c]| - radius)^2 / band) on the box exceeds
 *           eps, the coefficient being the largest |f - I f| over the 13^3 half-node points
 *           of the box that are not its nodes, I the degree-6 tensor Lagrange interpolant
 *           from its 7^3 nodes (exact rational weights rounded once, fixed summation order).
 * Octants of level < l_min are always split.  Centers and radii are mapped to
 * lattice units as llround((c - lo)/(hi - lo) * 2^20) and floor/ceil of
 * (r/(hi - lo) * 2^20)^2; the tests are exact int64 comparisons. */
typedef struct {
  double lo, hi;
  int l_min, l_max; /* 0 <= l_min <= l_max <= 18 */
  int kind;
  int n_centers;    /* 1..8 */
  double centers[8][3];
  double radius, band;
  double eps;       /* kind 3 only */
} lts_refine_spec;

enum { LTS_PDE_ADVECTION = 0, LTS_PDE_WAVE = 1 };
enum { LTS_BC_EXACT = 0, LTS_BC_RADIATIVE = 1 };
enum {
  LTS_IC_ADV_GAUSS = 0,   /* ic_params[0..2] x0, [3] w: u = exp(-|x - x0 - a t|^2 / w) */
  LTS_IC_WAVE_SHELL = 2,  /* [0] R, [1] w, [2] amp, [3] nmodes (<= 4), [4] kscale, [5+5m..] eps, kx, ky, kz, theta:
                             chi = exp(-(r-R)^2/w) (1 + amp sum eps sin(kscale k.x + theta)), phi = 0 */
  LTS_IC_WAVE_PLANAR = 3, /* [0] s0, [1] w: chi = (f(x-t) + f(x+t))/2, f(s) = exp(-(s-s0)^2/w), phi = chi_t */
  LTS_IC_WAVE_REST = 5    /* chi = phi = 0 (a field at rest, driven by source terms) */
};

/* The problem (Sec. 4.2).  pde 0: u_t + adv . grad u = 0.  pde 1: chi_t = phi,
 * phi_t = lap chi + sources (eqs. chi, phi; sources below).  Both add Kreiss-Oliger dissipation
 * (ko_sigma / (64 h)) sum_d delta_d^6.  bc 0 (exact): exterior ghosts are the
 * RK stage values of the closed-form solution named by `ic`; bc 1 (radiative,
 * wave only): exterior ghosts by cubic extrapolation and, at nodes on the domain
 * boundary, df/dt = -(x/r) . grad f - k f / r with k = 1 for chi, 2 for phi. */
typedef struct {
  int pde;
  double adv[3];
  double cfl;          /* dt_finest = cfl * h_finest, h = node spacing (Sec. 3.4 CFL) */
  double ko_sigma;
  int rk;              /* 4: classical RK4; 3: SSPRK3 */
  int bc;
  int ic;
  double ic_params[32];
  int precision;       /* 0: FP64 throughout; where the coefficients are integers (the wave
                          equation's Laplacian and dissipation of chi, the coarse -> fine
                          interpolation lines) the sums are exact in 64-bit integers and each
                          result is rounded once to FP64, within the error bound of the FP64
                          evaluation.  1: mixed -- RK stages, stage inputs, the padded block and
                          the right-hand side in FP32; the state, the RK update and the time
                          corrections (eqs. fc_1, fc_2) in FP64 */
  void* stream;        /* cudaStream_t; NULL = default stream */
  void* (*dev_alloc)(size_t bytes, void* ctx);  /* optional device allocator */
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  /* source terms of the wave equation (pde 1 only; zero-initialised = none), added to
   * phi_t at every node except boundary nodes under bc 1:
   *   nl_c:  -nl_c sin(2 chi) / r^2 (eq. phi; the paper's non-linear runs use c = 1),
   *          taken as 0 at r = 0;
   *   orbit: 1 adds A sum_{i=1,2} exp(-|x - x_i(t)|^2 / w) with x_1 = R (cos W t, sin W t, 0),
   *          x_2 = -x_1, orbit_params = {R, W, w > 0, A}, evaluated at the stage time
   *          t_b + c_s dt of each RK stage.  Not in the paper: a driven workload. */
  double nl_c;
  int orbit;
  double orbit_params[4];
} lts_problem;

typedef struct {
  int64_t n_octants;
  int nf, p;                    /* fields, RK stages */
  int l_min, l_max;             /* levels present in the tree */
  int64_t octants_per_level[32];
  double dt_finest;             /* dt of the finest level */
  double dt_coarsest;           /* one LTS macro step = 2^(l_max - l_min) * dt_finest */
  double time;                  /* current time of the plan (synchronised time + substeps) */
  int64_t substep;              /* substep index within the current macro step */
  double model_speedup;         /* eqs. w_nuts, w_uts, invS: W_gts / W_lts */
  double lts_work_per_macro;    /* octant-steps of one macro step (eq. w_nuts) */
  double gts_work_per_macro;    /* octant-steps of 2^(l_max-l_min) global steps (eq. w_uts) */
  size_t device_bytes;          /* device memory held by the plan */
  int64_t kernel_launches;      /* kernels the plan has launched so far */
  int64_t blocked_octants;      /* octants stepped in sibling-group blocks (lts_set_blocking) */
} lts_stats;

/* ---- octree: Sec. 3.2.2 construction, Sec. 3.2.3 2:1 balance -------------- */
/* Refine from the root by the predicate, balance 2:1 across faces, edges and
 * corners (the unique coarsest balanced refinement), sort in level order.
 * Host-side; *out is owned by the caller and freed with octree_destroy. */
lts_status octree_build(const lts_refine_spec* spec, lts_octree** out);
lts_status octree_size(const lts_octree* tree, int64_t* n);
/* Copies the leaves in level order into caller host buffers xyz[3n], level[n]. */
lts_status octree_export(const lts_octree* tree, int32_t* xyz, int32_t* level);
void octree_destroy(lts_octree* tree);

/* ---- plan: Sec. 3.2.4 meshing (o2o), Sec. 3.6 per-level schedule ---------- */
/* Builds the neighbour tables, the time-correction tables of eqs. fc_1 / fc_2,
 * uploads them and allocates the state (u double-buffered per level, RK stages).
 * The tree must outlive nothing: the plan copies what it needs. */
lts_status lts_plan_create(const lts_octree* tree, const lts_problem* prob, lts_plan** out);
void lts_plan_destroy(lts_plan* plan);
lts_status lts_plan_stats(const lts_plan* plan, lts_stats* out);

/* ---- state ---------------------------------------------------------------- */
/* Initial data of prob->ic at every node at time t0 (device kernel). */
lts_status lts_set_initial(lts_plan* plan, double t0);
/* u: [nf][N][343] FP64, host memory (on_device = 0) or device memory (1). */
lts_status lts_set_state(lts_plan* plan, const double* u, double t0, int on_device);
/* Copies the current DG state; synchronises the stream.  t (optional) gets the time. */
lts_status lts_get_state(lts_plan* plan, double* u, double* t, int on_device);
/* RK stage j (0-based) of every octant's most recent step, [nf][N][343], widened to FP64
 * in the mixed-precision mode. */
lts_status lts_get_stage(lts_plan* plan, int j, double* k, int on_device);

/* ---- time stepping ------------------------------------------------------------ */
/* Alg. 2 substeps of dt_finest (Fig. blk_loop): in substep n of a macro step the
 * levels l >= l*(n) step, l* the smallest l with n % 2^(l_max - l) == 0.  After
 * the last substep of a macro step the duplicated DG nodes are reconciled
 * (shared-node sync).  Asynchronous. */
lts_status lts_run_substeps(lts_plan* plan, int64_t n);
/* LTS to t_end: (t_end - time) must be a whole number of macro steps (to 1e-9
 * relative), and the plan must be at a macro-step boundary; else LTS_EINVAL. */
lts_status lts_advance(lts_plan* plan, double t_end);
/* Alg. 1: n global steps of dt_finest with the shared-node sync of every stage. */
lts_status gts_steps(lts_plan* plan, int64_t n);
/* GTS to t_end: (t_end - time) must be a whole number of dt_finest. */
lts_status gts_advance(lts_plan* plan, double t_end);

/* ---- maps for parity checks ---------------------------------------------------- */
/* o2o (Sec. 3.2.4): out[N][27][8] int32 host buffer; direction d = (dx+1) +
 * 3(dy+1) + 9(dz+1); entry 0 = the leaf covering the same-size box in direction d
 * (same size or coarser), or -2 if the box lies outside the domain; if the box is
 * split, the 8 entries are its children in Morton child order (-1: not a leaf). */
lts_status lts_export_o2o(const lts_plan* plan, int32_t* out);
/* Padding sources computed by the device resolver the stage kernel uses, for the
 * n octants listed in octs (host int32): src[n][2197] (leaf index, -1 outside the
 * domain) and r[n][2197][3] (half-node coordinates in the source). */
lts_status lts_export_pad_map(lts_plan* plan, const int32_t* octs, int64_t n, int32_t* src, int32_t* r);
/* Same for the 343 nodes of each listed octant (the shared-node owners). */
lts_status lts_export_node_map(lts_plan* plan, const int32_t* octs, int64_t n, int32_t* src, int32_t* r);
/* Allocation-free variant of lts_export_pad_map (the paper has no counterpart:
 * this is a service of the library).  For callers that must not allocate device
 * memory while they run -- e.g. a process whose device memory is all reserved up
 * front by its own pool, or a loop that cannot afford an allocator call and the
 * synchronisation it may bring.  Results are staged in one fixed device array
 * inside the library (about 1.1 MB, held by every GPU that loads the library
 * until the process exits), so at most 32 octants per call (more: LTS_EINVAL).
 * The array's device address is looked up on the first call on each device, with
 * that device current; make that first call outside any stream capture.  Every
 * call shares the array and overwrites what the last call left there; calls whose
 * GPU work overlaps (other threads, other plans, other streams) race on it.  The
 * octant list, src[n][2197] and r[n][2197][3] are host buffers as above; the call
 * synchronises the plan's stream.  The device current at the call must be the one
 * that was current when the plan was created (else LTS_EINVAL), since the array's
 * address differs per device. */
lts_status lts_export_pad_map_static(lts_plan* plan, const int32_t* octs, int64_t n, int32_t* src, int32_t* r);

/* Octree-to-block decomposition (Sec. 3.2.5).  With blocking on (the default), every
 * complete sibling group (the 8 children of one parent, all leaves of one level) is
 * stepped by one CTA as a single block of 13^3 nodes with a 19^3 padded tile, and the
 * remaining octants one by one.  A group qualifies when no leaf coarser than its children
 * touches any child: there, every padded point of a child holds the same value in the
 * children's own tiles and in the block tile, and the copies of the nodes the siblings
 * share stay equal, so results are bit-identical either way (at a coarser neighbour the
 * padding rule takes the coarse interpolant on the block's surface, where the block tile
 * holds the siblings' own values).  Blocking cuts the gathered points per node from 6.4
 * to 2.5.  Errors: LTS_EINVAL (null plan). */
lts_status lts_set_blocking(lts_plan* plan, int on);

/* ---- measurement ------------------------------------------------------------------- */
/* When on, every stage-kernel launch is bracketed by CUDA events on the plan's
 * stream; lts_kernel_stats synchronises and reports, since the last reset, the
 * number of stage launches, their summed device time (ms), and the algorithmic
 * flops and HBM bytes of those launches.  Per node-stage: wave 59 flops (both fields,
 * FMA = 2), advection 45; per node-stage and field 38 bytes in FP64 (own stage input,
 * step-start state and stage, 8 each; the next stage input, 6 over the stages; the
 * update's share, 8) and 24 in mixed precision (the same arrays with FP32 stages).
 * Gathers of neighbours' values are not counted (they are expected to hit L2). */
lts_status lts_set_profiling(lts_plan* plan, int on);
lts_status lts_kernel_stats(lts_plan* plan, int64_t* launches, double* ms, double* flops, double* bytes,
                            int64_t* node_stages, int reset);
/* The same for the prolongation launches (coarse -> fine padding, Fig. unzip: the coarser
 * sources' stage inputs corrected in time by eqs. fc_1 / fc_2 and interpolated to the
 * half-node positions their finer neighbours read), bracketed by events while profiling is
 * on: the number of launches, their summed device time (ms), the coarser sources they
 * prolonged, and their FP64-equivalent flops as directly evaluated (FMA = 2): per source
 * and field the interpolation's multiply-adds of the plan's pass-order cost model (7 per
 * odd half-node position of each pass), and under LTS the corrected inputs at its 343
 * nodes (one multiply-add per correction term and one for the step).  The kernel itself
 * evaluates mirrored position pairs with fewer operations, so the rate is an equivalent.
 * Out-pointers may be null.  Errors: LTS_EINVAL (null plan); a device fault recorded
 * earlier is returned. */
lts_status lts_prolong_stats(lts_plan* plan, int64_t* launches, double* ms, double* flops, int64_t* sources,
                             int reset);

/* ---- batches: many independent solves advanced together (NEXT-2) ------------------ */
/* A batch advances several plans together in rounds: in each round every plan with
 * substeps left performs one LTS substep of its own schedule (Alg. 2, Fig. blk_loop),
 * and the schedule is advanced on the device, so a round is a fixed launch sequence that
 * can be captured once in a CUDA graph and replayed.  Two modes (lts_batch_set_mode):
 *   persistent: the whole round is one cooperative launch whose CTAs stay
 *     resident and claim work items (the prolongations and octant-stages of all plans,
 *     stage by stage, then the reconciles) between grid-wide barriers; every barrier
 *     wait has a time limit (2 s), past which the launch is abandoned and the next
 *     lts_batch_wait returns LTS_ETIMEOUT;
 *   per-stage (the default): each RK stage is a launch of the prolongation and one of
 *     the stage kernel over all plans, with round start / end and reconcile launches
 *     around them.
 * Results equal those of running each plan alone, in either mode.  The plans must share
 * one stream and one precision; the batch keeps pointers to them (they must outlive
 * it).  Up to 1024 plans. */
typedef struct lts_batch lts_batch;
lts_status lts_batch_create(lts_plan* const* plans, int n, lts_batch** out);
/* An empty batch of n_slots slots on `stream` (cudaStream_t) for plans of one precision
 * (0 FP64, 1 mixed).  Plans join and leave between runs with attach / detach (continuous
 * batching); every run launches all 4 stages and all levels, so one captured round
 * serves any membership.  A detached plan keeps its state and can run alone again. */
lts_status lts_batch_create_slots(int n_slots, void* stream, int precision, lts_batch** out);
lts_status lts_batch_attach(lts_batch* batch, int slot, lts_plan* plan);
lts_status lts_batch_detach(lts_batch* batch, int slot);
void lts_batch_destroy(lts_batch* batch);
/* Advance the plan in slot i by substeps[i] substeps (host array, one count per slot;
 * 0 for empty slots), in max(substeps) rounds.  use_graph: replay one captured round.
 * Asynchronous on the plans' stream. */
lts_status lts_batch_run(lts_batch* batch, const int64_t* substeps, int use_graph);
/* Grid sizes (CTAs) of the per-stage launches; set by an autotuner or by hand. */
lts_status lts_batch_set_grid(lts_batch* batch, int grid_stage, int grid_prolong, int grid_sync);
/* persistent = 1: one cooperative launch per round with ctas_per_sm CTAs on every SM (at
 * most what the round kernel keeps resident; more: LTS_EINVAL); persistent = 0: the
 * per-stage launches.  Drops the captured round. */
lts_status lts_batch_set_mode(lts_batch* batch, int persistent, int ctas_per_sm);
/* Waits for the batch's rounds and reports a device-side failure: LTS_ETIMEOUT if a grid
 * barrier of a persistent round waited past its limit (the round was abandoned part way:
 * the plans' states are then undefined; the error word is cleared). */
lts_status lts_batch_wait(lts_batch* batch);
/* Test of the barrier's time limit: one launch of the grid barrier alone over one CTA
 * per SM, limit_s seconds per wait (0 < limit_s <= 60).  absent_cta in [0, SMs) makes
 * that CTA leave without arriving, so the others' waits run out: LTS_ETIMEOUT; -1: every
 * CTA arrives, LTS_OK.  Synchronises the batch's stream. */
lts_status lts_batch_probe_barrier(lts_batch* batch, int absent_cta, double limit_s);
/* launches: kernels launched by the batch's rounds so far; grid_stage: the grid of the
 * current mode's stage work (the persistent launch's, in persistent mode). */
lts_status lts_batch_stats(const lts_batch* batch, int64_t* launches, int* grid_stage, int* grid_prolong,
                           int* grid_sync);

const char* lts_strerror(lts_status s);
const char* lts_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
