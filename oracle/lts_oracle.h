/*
 * lts_oracle.h -- CPU oracle for local timestepping (LTS) on 2:1-balanced
 * Morton-ordered octrees (Fernando & Sundar, "Scalable Local Timestepping on
 * Octree Grids", arXiv 2011.10570).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct FP64
 * restatement of the method, used to check the CUDA library.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (shared meaning, separate code):
 *   lattice: integer anchors in [0, 2^ORC_D)^3; an octant of level l has edge
 *            e = 2^(ORC_D - l) lattice units.
 *   nodes:   7 per axis (element order 6), node (i,j,k) of an octant sits at
 *            lattice6 coordinate 6*A + (i,j,k)*e  (lattice6 = 6 x lattice).
 *   padded block: 13^3 points, i,j,k in [-3, 9] (ghost width 3).
 *   octant order: ascending (level, Morton key)  ("level order").
 *   DG arrays: [field][octant][343], node index i + 7 j + 49 k.
 */
#ifndef LTS_ORACLE_H
#define LTS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_D 20

typedef struct {
  double lo, hi;          /* cube domain [lo,hi]^3 */
  int l_min, l_max;       /* refinement levels */
  int kind;               /* 0: balls of `radius` around centers; 1: shell |x-c0| in [radius-band, radius+band];
                             2: within `band` of the circle of `radius` around c0 in the plane z = c0.z;
                             3: wavelet criterion (Sec. 3.2.2) on the field
                                f(x) = sum_c exp(-(|x - c| - radius)^2 / band), tolerance eps */
  int n_centers;
  double centers[8][3];
  double radius, band;
  double eps;
} orc_refine;

enum { ORC_PDE_ADVECTION = 0, ORC_PDE_WAVE = 1 };
enum { ORC_BC_EXACT = 0, ORC_BC_RADIATIVE = 1 };
enum {
  ORC_IC_ADV_GAUSS = 0,   /* p[0..2] x0, p[3] w : u = exp(-|x - x0 - a t|^2 / w) */
  ORC_IC_ADV_POLY = 1,    /* p[0..63] c[i + 4 j + 16 k] : u = sum c x^i y^j z^k at x - a t */
  ORC_IC_WAVE_SHELL = 2,  /* p[0] R, p[1] w, p[2] amp, p[3] nmodes, p[4] kscale, p[5+5m..] eps, kx, ky, kz, theta */
  ORC_IC_WAVE_PLANAR = 3, /* p[0] s0, p[1] w : chi = (f(x-t) + f(x+t))/2, f = exp(-(s-s0)^2/w) */
  ORC_IC_WAVE_POLY = 4,   /* p[0..63] cubic P, p[64..127] cubic Q : chi = P + tQ + t^2/2 lap P + t^3/6 lap Q */
  ORC_IC_WAVE_REST = 5    /* chi = phi = 0 */
};

typedef struct {
  int pde;
  double adv[3];
  double cfl;
  double ko_sigma;
  int rk;                  /* 4: classical RK4, 3: SSPRK3 */
  int bc;
  int ic;
  double ic_params[160];
  double nl_c;             /* wave: phi_t += -nl_c sin(2 chi) / r^2 (eq. phi), 0 at r = 0 */
  int orbit;               /* wave: 1 adds two Gaussian sources on a circular orbit (a reading of the paper) */
  double orbit_params[4];  /* orbit radius, angular speed, width w, amplitude A:
                              phi_t += A sum_{i=1,2} exp(-|x - x_i(t)|^2 / w),
                              x_1 = radius (cos wt, sin wt, 0), x_2 = -x_1 */
} orc_problem;

typedef struct orc_tree orc_tree;
typedef struct orc_solver orc_solver;

/* ---- octree (Sec. 3.2.2 construction, Sec. 3.2.3 2:1 balance) ---- */
uint64_t orc_morton(uint32_t x, uint32_t y, uint32_t z);
orc_tree* orc_tree_build(const orc_refine* spec);          /* refine + balance + level order */
orc_tree* orc_tree_refine_only(const orc_refine* spec);    /* refinement without balancing */
orc_tree* orc_tree_from_leaves(double lo, double hi, int64_t n, const int32_t* xyz, const int32_t* level);
void orc_tree_free(orc_tree* t);
int64_t orc_tree_size(const orc_tree* t);
void orc_tree_export(const orc_tree* t, int32_t* xyz, int32_t* level);     /* level order */
int orc_refine_pred(const orc_refine* spec, int32_t x, int32_t y, int32_t z, int level);
/* kind 3: the largest wavelet coefficient of the box (max over its 13^3 half-node points
 * with an odd coordinate of |f - I f|, I the degree-6 Lagrange interpolant from its 7^3 nodes) */
double orc_wavelet_coeff(const orc_refine* spec, int32_t x, int32_t y, int32_t z, int level);

/* ---- maps (Sec. 3.2.4 meshing, Sec. 3.3 unzip) ---- */
/* leaf index (level order) containing lattice cell (x,y,z), -1 if outside */
int64_t orc_find_leaf(const orc_tree* t, int64_t x, int64_t y, int64_t z);
/* o2o: out[b][27][8], dir = (dx+1) + 3(dy+1) + 9(dz+1) */
void orc_o2o(const orc_tree* t, int32_t* out);
/* source of lattice6 point P: leaf index or -1 (outside domain); r = half-node coords in the source */
int64_t orc_point_source(const orc_tree* t, int64_t px, int64_t py, int64_t pz, int32_t r[3]);
/* padding map of octant b: src[2197], r[2197][3]; interior points get src = b */
void orc_pad_map(const orc_tree* t, int64_t b, int32_t* src, int32_t* r);
/* node (sync) map of octant b: src[343], r[343][3] */
void orc_node_map(const orc_tree* t, int64_t b, int32_t* src, int32_t* r);

/* ---- operators (Sec. 3.3 FD, Fig. unzip interpolation) ---- */
void orc_interp_weights(double W[13][7]);
double orc_interp_point(const double* v343, int rx, int ry, int rz);
/* derivatives of a padded 13^3 tile at its 343 interior nodes: d1,d2,ko are [3][343] */
void orc_tile_ops(const double* tile, double h, double* d1, double* d2, double* ko6);

/* ---- RK and LTS corrections (eq. rk_schemes, eqs. rk_crrection, fc_1, fc_2) ---- */
int orc_tableau(int rk, double a[4][4], double w[4], double c[4]);
/* omega[s][j] for a source step (t_N, dt_N) serving a requester step starting at
 * t_N + theta dt_N with dt_b = rho dt_N */
int orc_omega(int rk, double theta, double rho, double* omega /* [p][p] */);
int orc_stage_taylor(int rk, double* gamma /* [p][p] */);
/* exact solution and its time derivatives d[f][m] = d^m/dt^m, m = 0..5 */
void orc_exact_derivs(const orc_problem* pr, const double x[3], double t, double d[2][6]);

/* ---- solver ---- */
orc_solver* orc_solver_create(const orc_tree* t, const orc_refine* spec, const orc_problem* pr);
void orc_solver_free(orc_solver* s);
int orc_solver_nf(const orc_solver* s);
double orc_solver_dt_f(const orc_solver* s);
double orc_solver_time(const orc_solver* s);
int orc_solver_substep_index(const orc_solver* s);
void orc_set_initial(orc_solver* s, double t0);
void orc_set_state(orc_solver* s, const double* u, double t0);
void orc_get_state(const orc_solver* s, double* u);
void orc_get_stage(const orc_solver* s, int stage, double* k);
/* padded 13^3 block [nf][2197] of octant b from the current state (first-stage input) */
void orc_solver_tile(orc_solver* s, int64_t b, double* T);
void orc_exact_state(const orc_solver* s, double t, double* u);
/* Alg. 2 with the substep schedule of Fig. blk_loop: n substeps of dt_f */
void orc_lts_substeps(orc_solver* s, int64_t n);
/* one substep computing stage j only on octants with mask[j*N + b] != 0, and
 * the step update only where fmask[b] != 0 (dependency-cone checks) */
void orc_lts_substep_masked(orc_solver* s, const uint8_t* mask, const uint8_t* fmask);
/* Alg. 1: n global steps of dt_f */
void orc_gts_steps(orc_solver* s, int64_t n);
/* DG -> shared-node -> DG synchronisation of one field array [nf][N][343] in place */
void orc_sync(orc_solver* s, double* v);
/* active level of substep n (Fig. blk_loop) */
int orc_active_level(int l_min, int l_max, int64_t n);
/* eqs. w_nuts, w_uts, invS: returns S = W_gts / W_lts */
double orc_work_model(const orc_tree* t, double* w_lts, double* w_gts);
void orc_set_threads(int n);
/* negative controls for the tests (0 = the method as stated): 1 no time correction,
 * 2 nearest node instead of interpolation, 3 wrong advection sign, 4 step-end
 * state for inactive coarser sources, 5 radiative k of chi and phi swapped,
 * 6 sign of the radiative x^i/r term flipped, 7 wrong cubic-extrapolation row */
void orc_set_mutation(int m);

#ifdef __cplusplus
}
#endif
#endif
