/*
 * lts_oracle.c -- CPU oracle for local timestepping on 2:1-balanced octrees
 * (Fernando & Sundar, "Scalable Local Timestepping on Octree Grids").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the library.  Plain loops in FP64,
 * compiled with -ffp-contract=off.  Every function names the passage of the
 * paper it restates; where the paper is silent or garbled the reading taken
 * is stated beside the code as a reading.
 *
 * Parity status: every function here is pinned by a CPU test against
 * brute force, closed forms, exact polynomial reproduction or values the
 * paper prints (see tests/test_oracle_*.py).
 */
#include "lts_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NP 7
#define NV 343
#define PW 13
#define NT 2197
#define ROOT_EDGE ((int64_t)1 << ORC_D)
#define L6 (6 * ROOT_EDGE)

/* Negative controls for the tests: a deliberately wrong variant of one step, so
 * that the tests can show their pins catch it.  0 = the method as stated. */
static int g_mutation = 0;
void orc_set_mutation(int m) { g_mutation = m; }

static void die(const char* msg) {
  fprintf(stderr, "lts_oracle: %s\n", msg);
  abort();
}

/* ------------------------------------------------------------------------ */
/* Octree (Sec. 3.2: linear octree on [0,2^L]^3, SFC ordering)               */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t x, y, z, l;
} oct_t;

struct orc_tree {
  double lo, hi;
  int64_t n;
  oct_t* oct;          /* level order */
  uint64_t* key;       /* Morton key of each octant (level order) */
  int64_t* by_morton;  /* level-order indices sorted by Morton key */
  uint64_t* mkeys;     /* keys in Morton order */
  int64_t level_count[ORC_D + 1];
};

/* Morton key: bits interleaved x lowest, ...z1 y1 x1 z0 y0 x0 (SFC order, Sec. 3.2.4). */
uint64_t orc_morton(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t k = 0;
  for (int b = 0; b < 21; ++b) {
    k |= (uint64_t)((x >> b) & 1u) << (3 * b);
    k |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
    k |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
  }
  return k;
}

static int64_t edge_of(int l) { return ROOT_EDGE >> l; }

/* Refinement predicates.  Kinds 0-2 are integer geometric predicates (a reading: they
 * reproduce the configurations' trees exactly; centers and radii are mapped to lattice
 * units and squared distances compared in int64); kind 3 is the paper's wavelet
 * criterion of Sec. 3.2.2. */
static int64_t to_lattice(double v, double lo, double hi) {
  return llround((v - lo) / (hi - lo) * (double)ROOT_EDGE);
}

static int64_t radius_sq_floor(double r, double lo, double hi) {
  double rl = r / (hi - lo) * (double)ROOT_EDGE;
  return (int64_t)floor(rl * rl);
}

static int64_t radius_sq_ceil(double r, double lo, double hi) {
  double rl = r / (hi - lo) * (double)ROOT_EDGE;
  return (int64_t)ceil(rl * rl);
}

/* kind 2: distance from the box to the circle of radius R around c in the plane
 * z = c_z: with rho the distance from the axis, d^2 = drho^2 + dz^2 where drho is the
 * distance from R to the box's range of rho and dz the box's distance to the plane */
static int circle_pred(const orc_refine* s, const int64_t a[3], int64_t e) {
  int64_t cc[3];
  for (int d = 0; d < 3; ++d) cc[d] = to_lattice(s->centers[0][d], s->lo, s->hi);
  int64_t rmin2 = 0, rmax2 = 0;
  for (int d = 0; d < 2; ++d) {
    int64_t lo = a[d], hi = a[d] + e, dn = 0;
    if (cc[d] < lo) dn = lo - cc[d];
    if (cc[d] > hi) dn = cc[d] - hi;
    rmin2 += dn * dn;
    int64_t f1 = cc[d] - lo, f2 = hi - cc[d];
    if (f1 < 0) f1 = -f1;
    if (f2 < 0) f2 = -f2;
    int64_t df = f1 > f2 ? f1 : f2;
    rmax2 += df * df;
  }
  int64_t dz = 0;
  if (cc[2] < a[2]) dz = a[2] - cc[2];
  if (cc[2] > a[2] + e) dz = cc[2] - a[2] - e;
  double R = s->radius / (s->hi - s->lo) * (double)ROOT_EDGE;
  double b = s->band / (s->hi - s->lo) * (double)ROOT_EDGE;
  double rmin = sqrt((double)rmin2), rmax = sqrt((double)rmax2);
  double dr = 0.0;
  if (rmin - R > dr) dr = rmin - R;
  if (R - rmax > dr) dr = R - rmax;
  double dzd = (double)dz;
  return dr * dr + dzd * dzd <= b * b;
}

/* kind 3, the wavelet criterion of Sec. 3.2.2: a box is split while its field fails to be
 * interpolated from its own nodes at the nodes of its children by more than eps.  The
 * field is a sum of Gaussian shells f(x) = sum_c exp(-(|x - c| - R)^2 / w) (R = radius,
 * w = band; R = 0 gives Gaussian bumps).  The degree-6 Lagrange weights at the half-node
 * positions k/2 are the exact rationals prod_{m != j} (k - 2m) / prod_{m != j} (2j - 2m),
 * each rounded once, and every sum runs in a fixed order, so the decision is reproducible. */
static double wavelet_field(const orc_refine* s, const double x[3]) {
  double f = 0.0;
  for (int c = 0; c < s->n_centers; ++c) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double t = x[a] - s->centers[c][a];
      d2 += t * t;
    }
    double r = sqrt(d2) - s->radius;
    f += exp(-(r * r) / s->band);
  }
  return f;
}

static void half_weights(double w[13][7]) {
  for (int k = 0; k < 13; ++k)
    for (int j = 0; j < 7; ++j) {
      int64_t num = 1, den = 1;
      for (int m = 0; m < 7; ++m) {
        if (m == j) continue;
        num *= (int64_t)(k - 2 * m);
        den *= (int64_t)(2 * j - 2 * m);
      }
      w[k][j] = (double)num / (double)den;
    }
}

double orc_wavelet_coeff(const orc_refine* s, int32_t x, int32_t y, int32_t z, int level) {
  int64_t e = edge_of(level);
  int64_t a[3] = {x, y, z};
  double w[13][7];
  half_weights(w);
  /* the field at the 13^3 half-node points: lattice6 coordinate 6 a + k e / 2 */
  double* F = (double*)malloc(13 * 13 * 13 * sizeof(double));
  for (int kz = 0; kz < 13; ++kz)
    for (int ky = 0; ky < 13; ++ky)
      for (int kx = 0; kx < 13; ++kx) {
        int64_t k3[3] = {kx, ky, kz};
        double p[3];
        for (int d = 0; d < 3; ++d) {
          int64_t P = 6 * a[d] + k3[d] * (e / 2);
          p[d] = s->lo + (s->hi - s->lo) * ((double)P / (6.0 * (double)ROOT_EDGE));
        }
        F[kx + 13 * ky + 169 * kz] = wavelet_field(s, p);
      }
  double cmax = 0.0;
  for (int kz = 0; kz < 13; ++kz)
    for (int ky = 0; ky < 13; ++ky)
      for (int kx = 0; kx < 13; ++kx) {
        if (!((kx | ky | kz) & 1)) continue;
        /* interpolate from the nodes (even half-node indices): x, then y, then z */
        double sz = 0.0;
        for (int c = 0; c < 7; ++c) {
          double sy = 0.0;
          for (int b = 0; b < 7; ++b) {
            double sx = 0.0;
            for (int q = 0; q < 7; ++q) sx = sx + w[kx][q] * F[2 * q + 13 * 2 * b + 169 * 2 * c];
            sy = sy + w[ky][b] * sx;
          }
          sz = sz + w[kz][c] * sy;
        }
        double d = fabs(F[kx + 13 * ky + 169 * kz] - sz);
        if (d > cmax) cmax = d;
      }
  free(F);
  return cmax;
}

int orc_refine_pred(const orc_refine* s, int32_t x, int32_t y, int32_t z, int level) {
  int64_t e = edge_of(level);
  int64_t a[3] = {x, y, z};
  if (s->kind == 2) return circle_pred(s, a, e);
  if (s->kind == 3) return orc_wavelet_coeff(s, x, y, z, level) > s->eps;
  int ncent = s->kind == 1 ? 1 : s->n_centers;
  for (int c = 0; c < ncent; ++c) {
    int64_t cc[3];
    for (int d = 0; d < 3; ++d) cc[d] = to_lattice(s->centers[c][d], s->lo, s->hi);
    int64_t dmin = 0, dmax = 0;
    for (int d = 0; d < 3; ++d) {
      int64_t lo = a[d], hi = a[d] + e;
      int64_t dn = 0;
      if (cc[d] < lo) dn = lo - cc[d];
      if (cc[d] > hi) dn = cc[d] - hi;
      dmin += dn * dn;
      int64_t f1 = cc[d] - lo, f2 = hi - cc[d];
      if (f1 < 0) f1 = -f1;
      if (f2 < 0) f2 = -f2;
      int64_t df = f1 > f2 ? f1 : f2;
      dmax += df * df;
    }
    if (s->kind == 0) {
      if (dmin <= radius_sq_floor(s->radius, s->lo, s->hi)) return 1;
    } else {
      int64_t outer = radius_sq_floor(s->radius + s->band, s->lo, s->hi);
      double rin = s->radius - s->band;
      int64_t inner = rin > 0 ? radius_sq_ceil(rin, s->lo, s->hi) : 0;
      if (dmin <= outer && dmax >= inner) return 1;
    }
  }
  return 0;
}

typedef struct {
  oct_t* v;
  int64_t n, cap;
} octvec;

static void push(octvec* q, oct_t o) {
  if (q->n == q->cap) {
    q->cap = q->cap ? 2 * q->cap : 1024;
    q->v = (oct_t*)realloc(q->v, (size_t)q->cap * sizeof(oct_t));
    if (!q->v) die("out of memory");
  }
  q->v[q->n++] = o;
}

/* Sec. 3.2.2: split from the root while l < l_min, or l < l_max and the predicate holds. */
static void refine_rec(const orc_refine* s, oct_t o, octvec* out) {
  int split = o.l < s->l_min || (o.l < s->l_max && orc_refine_pred(s, o.x, o.y, o.z, o.l));
  if (!split) {
    push(out, o);
    return;
  }
  int32_t h = (int32_t)edge_of(o.l + 1);
  for (int c = 0; c < 8; ++c) {
    oct_t ch = {o.x + (c & 1) * h, o.y + ((c >> 1) & 1) * h, o.z + ((c >> 2) & 1) * h, o.l + 1};
    refine_rec(s, ch, out);
  }
}

static uint64_t okey(const oct_t* o) { return orc_morton((uint32_t)o->x, (uint32_t)o->y, (uint32_t)o->z); }

static int cmp_morton(const void* a, const void* b) {
  uint64_t ka = okey((const oct_t*)a), kb = okey((const oct_t*)b);
  return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

static int cmp_level_morton(const void* a, const void* b) {
  const oct_t* oa = (const oct_t*)a;
  const oct_t* ob = (const oct_t*)b;
  if (oa->l != ob->l) return oa->l < ob->l ? -1 : 1;
  return cmp_morton(a, b);
}

/* binary search in a Morton-sorted leaf array: the leaf containing cell c is the
 * one with the largest anchor key <= key(c) (leaves tile the domain) */
static int64_t search_sorted(const oct_t* v, const uint64_t* keys, int64_t n, int64_t x, int64_t y, int64_t z) {
  if (x < 0 || y < 0 || z < 0 || x >= ROOT_EDGE || y >= ROOT_EDGE || z >= ROOT_EDGE) return -1;
  uint64_t k = orc_morton((uint32_t)x, (uint32_t)y, (uint32_t)z);
  int64_t lo = 0, hi = n - 1, ans = -1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (keys[mid] <= k) {
      ans = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  if (ans < 0) die("cell below first leaf");
  const oct_t* o = &v[ans];
  int64_t e = edge_of(o->l);
  if (x < o->x || x >= o->x + e || y < o->y || y >= o->y + e || z < o->z || z >= o->z + e)
    die("leaf search: cell not covered (tree does not tile the domain)");
  return ans;
}

/* compares (key, index) pairs by key */
static int cmpkp(const void* a, const void* b) {
  uint64_t ka = *(const uint64_t*)a, kb = *(const uint64_t*)b;
  return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

static void build_index(orc_tree* t) {
  /* level order, then Morton index */
  qsort(t->oct, (size_t)t->n, sizeof(oct_t), cmp_level_morton);
  t->key = (uint64_t*)malloc((size_t)t->n * sizeof(uint64_t));
  t->by_morton = (int64_t*)malloc((size_t)t->n * sizeof(int64_t));
  t->mkeys = (uint64_t*)malloc((size_t)t->n * sizeof(uint64_t));
  for (int64_t i = 0; i < t->n; ++i) t->key[i] = okey(&t->oct[i]);
  /* sort indices by key (insertion via qsort on pairs) */
  typedef struct {
    uint64_t k;
    int64_t i;
  } kp;
  kp* tmp = (kp*)malloc((size_t)t->n * sizeof(kp));
  for (int64_t i = 0; i < t->n; ++i) {
    tmp[i].k = t->key[i];
    tmp[i].i = i;
  }
  qsort(tmp, (size_t)t->n, sizeof(kp), cmpkp);
  for (int64_t i = 0; i < t->n; ++i) {
    t->by_morton[i] = tmp[i].i;
    t->mkeys[i] = tmp[i].k;
  }
  free(tmp);
  memset(t->level_count, 0, sizeof(t->level_count));
  for (int64_t i = 0; i < t->n; ++i) t->level_count[t->oct[i].l]++;
}

/* Sec. 3.2.3, 2:1 balance across faces, edges and corners: repeat until no
 * change -- for every leaf and each of its 26 same-size neighbour boxes, split
 * the leaf covering that box if it is more than one level coarser. */
static void balance(octvec* q) {
  for (;;) {
    qsort(q->v, (size_t)q->n, sizeof(oct_t), cmp_morton);
    uint64_t* keys = (uint64_t*)malloc((size_t)q->n * sizeof(uint64_t));
    for (int64_t i = 0; i < q->n; ++i) keys[i] = okey(&q->v[i]);
    uint8_t* mark = (uint8_t*)calloc((size_t)q->n, 1);
    int64_t nmark = 0;
    for (int64_t i = 0; i < q->n; ++i) {
      oct_t o = q->v[i];
      int64_t e = edge_of(o.l);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (!dx && !dy && !dz) continue;
            int64_t j = search_sorted(q->v, keys, q->n, o.x + dx * e, o.y + dy * e, o.z + dz * e);
            if (j < 0) continue;
            if (q->v[j].l < o.l - 1 && !mark[j]) {
              mark[j] = 1;
              ++nmark;
            }
          }
    }
    free(keys);
    if (!nmark) {
      free(mark);
      return;
    }
    octvec nq = {0, 0, 0};
    for (int64_t i = 0; i < q->n; ++i) {
      oct_t o = q->v[i];
      if (!mark[i]) {
        push(&nq, o);
        continue;
      }
      int32_t h = (int32_t)edge_of(o.l + 1);
      for (int c = 0; c < 8; ++c) {
        oct_t ch = {o.x + (c & 1) * h, o.y + ((c >> 1) & 1) * h, o.z + ((c >> 2) & 1) * h, o.l + 1};
        push(&nq, ch);
      }
    }
    free(mark);
    free(q->v);
    *q = nq;
  }
}

static orc_tree* tree_from_vec(double lo, double hi, octvec* q) {
  orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
  t->lo = lo;
  t->hi = hi;
  t->n = q->n;
  t->oct = q->v;
  build_index(t);
  return t;
}

orc_tree* orc_tree_refine_only(const orc_refine* spec) {
  if (spec->l_min < 0 || spec->l_max < spec->l_min || spec->l_max > ORC_D - 2) return NULL;
  octvec q = {0, 0, 0};
  oct_t root = {0, 0, 0, 0};
  refine_rec(spec, root, &q);
  return tree_from_vec(spec->lo, spec->hi, &q);
}

orc_tree* orc_tree_build(const orc_refine* spec) {
  if (spec->l_min < 0 || spec->l_max < spec->l_min || spec->l_max > ORC_D - 2) return NULL;
  octvec q = {0, 0, 0};
  oct_t root = {0, 0, 0, 0};
  refine_rec(spec, root, &q);
  balance(&q);
  return tree_from_vec(spec->lo, spec->hi, &q);
}

orc_tree* orc_tree_from_leaves(double lo, double hi, int64_t n, const int32_t* xyz, const int32_t* level) {
  octvec q = {0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    oct_t o = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], level[i]};
    push(&q, o);
  }
  return tree_from_vec(lo, hi, &q);
}

void orc_tree_free(orc_tree* t) {
  if (!t) return;
  free(t->oct);
  free(t->key);
  free(t->by_morton);
  free(t->mkeys);
  free(t);
}

int64_t orc_tree_size(const orc_tree* t) { return t->n; }

void orc_tree_export(const orc_tree* t, int32_t* xyz, int32_t* level) {
  for (int64_t i = 0; i < t->n; ++i) {
    xyz[3 * i] = t->oct[i].x;
    xyz[3 * i + 1] = t->oct[i].y;
    xyz[3 * i + 2] = t->oct[i].z;
    level[i] = t->oct[i].l;
  }
}

/* ------------------------------------------------------------------------ */
/* Maps (Sec. 3.2.4 o2o / o2n, Sec. 3.3 padding sources)                     */
/* ------------------------------------------------------------------------ */

int64_t orc_find_leaf(const orc_tree* t, int64_t x, int64_t y, int64_t z) {
  if (x < 0 || y < 0 || z < 0 || x >= ROOT_EDGE || y >= ROOT_EDGE || z >= ROOT_EDGE) return -1;
  uint64_t k = orc_morton((uint32_t)x, (uint32_t)y, (uint32_t)z);
  int64_t lo = 0, hi = t->n - 1, ans = -1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (t->mkeys[mid] <= k) {
      ans = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  if (ans < 0) die("find_leaf: below first leaf");
  int64_t idx = t->by_morton[ans];
  const oct_t* o = &t->oct[idx];
  int64_t e = edge_of(o->l);
  if (x < o->x || x >= o->x + e || y < o->y || y >= o->y + e || z < o->z || z >= o->z + e)
    die("find_leaf: cell not covered");
  return idx;
}

/* o2o (Sec. 3.2.4): for each octant and each of the 27 same-size boxes around
 * it, the leaves covering that box: one leaf (same size or coarser), or the
 * children of the box that are leaves (finer).  Exterior boxes give -2. */
void orc_o2o(const orc_tree* t, int32_t* out) {
  for (int64_t b = 0; b < t->n; ++b) {
    const oct_t* o = &t->oct[b];
    int64_t e = edge_of(o->l);
    for (int d = 0; d < 27; ++d) {
      int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      int32_t* ent = out + (b * 27 + d) * 8;
      for (int c = 0; c < 8; ++c) ent[c] = -1;
      int64_t ax = o->x + dx * e, ay = o->y + dy * e, az = o->z + dz * e;
      int64_t j = orc_find_leaf(t, ax, ay, az);
      if (j < 0) {
        ent[0] = -2;
        continue;
      }
      if (t->oct[j].l <= o->l) {
        ent[0] = (int32_t)j;
        continue;
      }
      int64_t h = e / 2;
      for (int c = 0; c < 8; ++c) {
        int64_t k = orc_find_leaf(t, ax + (c & 1) * h, ay + ((c >> 1) & 1) * h, az + ((c >> 2) & 1) * h);
        ent[c] = t->oct[k].l == o->l + 1 ? (int32_t)k : -1;
      }
    }
  }
}

static int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

/* Reading of Sec. 3.3 / Fig. dg_to_cg: the value at a lattice point P comes from the coarsest leaf
 * whose closed box contains P, ties to the smallest Morton key; with octants in
 * (level, Morton) order this is the smallest level-order index.  The leaves
 * containing P are the leaves covering the (up to 8) unit cells touching P. */
int64_t orc_point_source(const orc_tree* t, int64_t px, int64_t py, int64_t pz, int32_t r[3]) {
  int64_t P[3] = {px, py, pz};
  int64_t hi_cell[3], lo_cell[3];
  for (int a = 0; a < 3; ++a) {
    hi_cell[a] = floor_div(P[a], 6);
    lo_cell[a] = -floor_div(-P[a], 6) - 1; /* ceil(P/6) - 1 */
  }
  int64_t best = -1;
  for (int c = 0; c < 8; ++c) {
    int64_t cx = (c & 1) ? hi_cell[0] : lo_cell[0];
    int64_t cy = (c & 2) ? hi_cell[1] : lo_cell[1];
    int64_t cz = (c & 4) ? hi_cell[2] : lo_cell[2];
    int64_t j = orc_find_leaf(t, cx, cy, cz);
    if (j < 0) continue;
    if (best < 0 || j < best) best = j;
  }
  if (best >= 0 && r) {
    const oct_t* o = &t->oct[best];
    int64_t e = edge_of(o->l);
    int64_t A[3] = {o->x, o->y, o->z};
    for (int a = 0; a < 3; ++a) {
      int64_t num = 2 * (P[a] - 6 * A[a]);
      if (num % e != 0) die("point_source: point not on the source's half-node lattice");
      int64_t rr = num / e;
      if (rr < 0 || rr > 12) die("point_source: point outside source box");
      r[a] = (int32_t)rr;
    }
  }
  return best;
}

void orc_pad_map(const orc_tree* t, int64_t b, int32_t* src, int32_t* r) {
  const oct_t* o = &t->oct[b];
  int64_t e = edge_of(o->l);
  for (int k = -3; k <= 9; ++k)
    for (int j = -3; j <= 9; ++j)
      for (int i = -3; i <= 9; ++i) {
        int q = (i + 3) + PW * (j + 3) + PW * PW * (k + 3);
        int32_t rr[3] = {-1, -1, -1};
        int64_t s = orc_point_source(t, 6 * (int64_t)o->x + i * e, 6 * (int64_t)o->y + j * e,
                                     6 * (int64_t)o->z + k * e, rr);
        if (i >= 0 && i <= 6 && j >= 0 && j <= 6 && k >= 0 && k <= 6) {
          s = b;
          rr[0] = 2 * i;
          rr[1] = 2 * j;
          rr[2] = 2 * k;
        }
        src[q] = (int32_t)s;
        r[3 * q] = rr[0];
        r[3 * q + 1] = rr[1];
        r[3 * q + 2] = rr[2];
      }
}

void orc_node_map(const orc_tree* t, int64_t b, int32_t* src, int32_t* r) {
  const oct_t* o = &t->oct[b];
  int64_t e = edge_of(o->l);
  for (int k = 0; k < NP; ++k)
    for (int j = 0; j < NP; ++j)
      for (int i = 0; i < NP; ++i) {
        int q = i + NP * j + NP * NP * k;
        int32_t rr[3] = {-1, -1, -1};
        int64_t s = orc_point_source(t, 6 * (int64_t)o->x + i * e, 6 * (int64_t)o->y + j * e,
                                     6 * (int64_t)o->z + k * e, rr);
        src[q] = (int32_t)s;
        r[3 * q] = rr[0];
        r[3 * q + 1] = rr[1];
        r[3 * q + 2] = rr[2];
      }
}

/* ------------------------------------------------------------------------ */
/* Operators: Lagrange interpolation (coarse -> fine padding, Sec. 3.3) and   */
/* centred finite differences with Kreiss-Oliger dissipation (a reading of the paper).     */
/* ------------------------------------------------------------------------ */

/* 1-D Lagrange basis of degree 6 on nodes 0..6 evaluated at r/2, r = 0..12 */
void orc_interp_weights(double W[13][7]) {
  for (int r = 0; r < 13; ++r) {
    double x = 0.5 * r;
    for (int m = 0; m < 7; ++m) {
      double v = 1.0;
      for (int q = 0; q < 7; ++q)
        if (q != m) v *= (x - q) / (double)(m - q);
      W[r][m] = v;
    }
    if (r % 2 == 0) /* exact nodes: unit vectors */
      for (int m = 0; m < 7; ++m) W[r][m] = (m == r / 2) ? 1.0 : 0.0;
  }
}

static double g_W[13][7];
static int g_W_ready = 0;

static void ensure_W(void) {
  if (!g_W_ready) {
    orc_interp_weights(g_W);
    g_W_ready = 1;
  }
}

/* tensor-product interpolation, x then y then z, skipping zero weights */
double orc_interp_point(const double* v, int rx, int ry, int rz) {
  ensure_W();
  double sz = 0.0;
  for (int c = 0; c < 7; ++c) {
    double wz = g_W[rz][c];
    if (wz == 0.0) continue;
    double sy = 0.0;
    for (int b = 0; b < 7; ++b) {
      double wy = g_W[ry][b];
      if (wy == 0.0) continue;
      double sx = 0.0;
      for (int a = 0; a < 7; ++a) {
        double wx = g_W[rx][a];
        if (wx == 0.0) continue;
        sx += wx * v[a + 7 * b + 49 * c];
      }
      sy += wy * sx;
    }
    sz += wz * sy;
  }
  return sz;
}

static inline int tix(int i, int j, int k) { return (i + 3) + PW * (j + 3) + PW * PW * (k + 3); }

/* 4th-order centred first and second derivatives and the 6th difference used by
 * Kreiss-Oliger dissipation, at interior node (i,j,k) along axis a. */
static void stencil_line(const double* T, int i, int j, int k, int a, double v[7]) {
  for (int m = -3; m <= 3; ++m) {
    int ii = i + (a == 0 ? m : 0), jj = j + (a == 1 ? m : 0), kk = k + (a == 2 ? m : 0);
    v[m + 3] = T[tix(ii, jj, kk)];
  }
}

static double d1_of(const double v[7], double h) { return (v[1] - 8.0 * v[2] + 8.0 * v[4] - v[5]) / (12.0 * h); }
static double d2_of(const double v[7], double h) {
  return (-v[1] + 16.0 * v[2] - 30.0 * v[3] + 16.0 * v[4] - v[5]) / (12.0 * h * h);
}
static double ko6_of(const double v[7]) {
  return v[0] - 6.0 * v[1] + 15.0 * v[2] - 20.0 * v[3] + 15.0 * v[4] - 6.0 * v[5] + v[6];
}

void orc_tile_ops(const double* T, double h, double* d1, double* d2, double* ko6) {
  for (int k = 0; k < NP; ++k)
    for (int j = 0; j < NP; ++j)
      for (int i = 0; i < NP; ++i) {
        int n = i + NP * j + NP * NP * k;
        for (int a = 0; a < 3; ++a) {
          double v[7];
          stencil_line(T, i, j, k, a, v);
          if (d1) d1[a * NV + n] = d1_of(v, h);
          if (d2) d2[a * NV + n] = d2_of(v, h);
          if (ko6) ko6[a * NV + n] = ko6_of(v);
        }
      }
}

/* ------------------------------------------------------------------------ */
/* Runge-Kutta tableaus (eq. rk_schemes) and the LTS stage corrections       */
/* (eqs. rk_crrection, fc_1, fc_2; a reading of the paper)                                */
/* ------------------------------------------------------------------------ */

int orc_tableau(int rk, double a[4][4], double w[4], double c[4]) {
  memset(a, 0, 16 * sizeof(double));
  memset(w, 0, 4 * sizeof(double));
  memset(c, 0, 4 * sizeof(double));
  if (rk == 4) { /* classical RK4 */
    a[1][0] = 0.5;
    a[2][1] = 0.5;
    a[3][2] = 1.0;
    w[0] = 1.0 / 6.0;
    w[1] = 1.0 / 3.0;
    w[2] = 1.0 / 3.0;
    w[3] = 1.0 / 6.0;
    c[1] = 0.5;
    c[2] = 0.5;
    c[3] = 1.0;
    return 4;
  }
  if (rk == 3) { /* SSPRK3 (Gottlieb-Shu, ref. of Sec. 1) */
    a[1][0] = 1.0;
    a[2][0] = 0.25;
    a[2][1] = 0.25;
    w[0] = 1.0 / 6.0;
    w[1] = 1.0 / 6.0;
    w[2] = 2.0 / 3.0;
    c[1] = 1.0;
    c[2] = 0.5;
    return 3;
  }
  return 0;
}

/* C of eq. rk_crrection, from the tableau for a linear autonomous F:
 * k_i = sum_m C[i][m] dt^m Y_m with Y_m the (m+1)-th time derivative,
 * so column 0 is 1 and column m+1 = A * column m. */
static void c_matrix(int p, double a[4][4], double C[4][4]) {
  memset(C, 0, 16 * sizeof(double));
  for (int i = 0; i < p; ++i) C[i][0] = 1.0;
  for (int m = 0; m + 1 < p; ++m)
    for (int i = 0; i < p; ++i) {
      double s = 0.0;
      for (int j = 0; j < p; ++j) s += a[i][j] * C[j][m];
      C[i][m + 1] = s;
    }
}

/* inverse of a lower-triangular matrix by forward substitution */
static void lower_inverse(int p, double L[4][4], double Li[4][4]) {
  memset(Li, 0, 16 * sizeof(double));
  for (int col = 0; col < p; ++col)
    for (int i = 0; i < p; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i][k] * Li[k][col];
      Li[i][col] = s / L[i][i];
    }
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

/* Stage correction in units dt_N = 1 (a reading of the paper):
 *   Y = P_N^-1 C^-1 K_N                       (eq. rk_crrection inverted)
 *   u_N(t_N + theta) = u_N + sum_m theta^(m+1)/(m+1)! Y_m
 *   K~ = C P_rho B_theta Y                    (eqs. fc_1 / fc_2)
 *   u~_s = u_N(t_N + theta) + rho sum_j a_sj K~_j
 * so u~_s = u_N + dt_N sum_j omega[s][j] k^N_j with
 *   omega_s = (e_theta + rho a_s C P_rho B_theta) C^-1. */
int orc_omega(int rk, double theta, double rho, double* omega) {
  double a[4][4], w[4], c[4], C[4][4], Ci[4][4];
  int p = orc_tableau(rk, a, w, c);
  if (!p) return 0;
  c_matrix(p, a, C);
  lower_inverse(p, C, Ci);
  double B[4][4] = {{0}};
  for (int m = 0; m < p; ++m)
    for (int j = m; j < p; ++j) B[m][j] = pow(theta, j - m) / factorial(j - m);
  for (int s = 0; s < p; ++s) {
    double row[4];
    for (int m = 0; m < p; ++m) row[m] = pow(theta, m + 1) / factorial(m + 1);
    double aC[4] = {0, 0, 0, 0};
    for (int m = 0; m < p; ++m)
      for (int j = 0; j < p; ++j) aC[m] += a[s][j] * C[j][m];
    double aCP[4];
    for (int m = 0; m < p; ++m) aCP[m] = aC[m] * pow(rho, m);
    for (int jj = 0; jj < p; ++jj) {
      double v = 0.0;
      for (int m = 0; m < p; ++m) v += aCP[m] * B[m][jj];
      row[jj] += rho * v;
    }
    for (int j = 0; j < p; ++j) {
      double v = 0.0;
      for (int m = 0; m < p; ++m) v += row[m] * Ci[m][j];
      omega[s * p + j] = v;
    }
  }
  return p;
}

/* gamma = A C: stage input s of a linear problem is
 * u + sum_m gamma[s][m] dt^(m+1) Y_m (used for exact boundary data) */
int orc_stage_taylor(int rk, double* gamma) {
  double a[4][4], w[4], c[4], C[4][4];
  int p = orc_tableau(rk, a, w, c);
  if (!p) return 0;
  c_matrix(p, a, C);
  for (int s = 0; s < p; ++s)
    for (int m = 0; m < p; ++m) {
      double v = 0.0;
      for (int j = 0; j < p; ++j) v += a[s][j] * C[j][m];
      gamma[s * p + m] = v;
    }
  return p;
}

/* ------------------------------------------------------------------------ */
/* Closed-form solutions (Sec. 4.2, eq. lsm with c = 0; configs' advection)  */
/* ------------------------------------------------------------------------ */

/* derivatives g^(m)(0), m = 0..5, of g(s) = exp(q0 + q1 s + q2 s^2) */
static void expquad_derivs(double q0, double q1, double q2, double g[6]) {
  double G = exp(q0), Q1 = q1, Q2 = 2.0 * q2;
  g[0] = G;
  g[1] = Q1 * G;
  g[2] = (Q2 + Q1 * Q1) * G;
  g[3] = (3.0 * Q1 * Q2 + Q1 * Q1 * Q1) * G;
  g[4] = (3.0 * Q2 * Q2 + 6.0 * Q1 * Q1 * Q2 + Q1 * Q1 * Q1 * Q1) * G;
  g[5] = (15.0 * Q1 * Q2 * Q2 + 10.0 * Q1 * Q1 * Q1 * Q2 + Q1 * Q1 * Q1 * Q1 * Q1) * G;
}

static double poly_eval(const double* c, double x, double y, double z) {
  double s = 0.0;
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 4; ++j)
      for (int i = 0; i < 4; ++i) {
        double v = c[i + 4 * j + 16 * k];
        if (v == 0.0) continue;
        s += v * pow(x, i) * pow(y, j) * pow(z, k);
      }
  return s;
}

static void poly_laplacian(const double* c, double* out) {
  for (int q = 0; q < 64; ++q) out[q] = 0.0;
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 4; ++j)
      for (int i = 0; i < 4; ++i) {
        double v = c[i + 4 * j + 16 * k];
        if (v == 0.0) continue;
        if (i >= 2) out[(i - 2) + 4 * j + 16 * k] += i * (i - 1) * v;
        if (j >= 2) out[i + 4 * (j - 2) + 16 * k] += j * (j - 1) * v;
        if (k >= 2) out[i + 4 * j + 16 * (k - 2)] += k * (k - 1) * v;
      }
}

static double binom(int n, int k) { return factorial(n) / (factorial(k) * factorial(n - k)); }

/* m-th time derivative of p(x - a t) at (x,t): Taylor coefficients in tau of p(y - a tau) */
static void adv_poly_derivs(const double* c, const double* adv, const double y[3], double d[6]) {
  for (int m = 0; m < 6; ++m) d[m] = 0.0;
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 4; ++j)
      for (int i = 0; i < 4; ++i) {
        double v = c[i + 4 * j + 16 * k];
        if (v == 0.0) continue;
        for (int al = 0; al <= i; ++al)
          for (int be = 0; be <= j; ++be)
            for (int ga = 0; ga <= k; ++ga) {
              int m = al + be + ga;
              if (m > 5) continue;
              double term = v * binom(i, al) * binom(j, be) * binom(k, ga) * pow(y[0], i - al) *
                            pow(y[1], j - be) * pow(y[2], k - ga) * pow(-adv[0], al) * pow(-adv[1], be) *
                            pow(-adv[2], ga);
              d[m] += term * factorial(m);
            }
      }
}

void orc_exact_derivs(const orc_problem* pr, const double x[3], double t, double d[2][6]) {
  const double* p = pr->ic_params;
  for (int f = 0; f < 2; ++f)
    for (int m = 0; m < 6; ++m) d[f][m] = 0.0;
  if (pr->ic == ORC_IC_ADV_GAUSS) {
    /* u = exp(-|x - x0 - a t|^2 / w); along tau: g(tau) = exp(Q(tau)) */
    double dd[3], adotd = 0.0, aa = 0.0, dsq = 0.0;
    for (int a = 0; a < 3; ++a) {
      dd[a] = x[a] - p[a] - pr->adv[a] * t;
      adotd += pr->adv[a] * dd[a];
      aa += pr->adv[a] * pr->adv[a];
      dsq += dd[a] * dd[a];
    }
    double w = p[3];
    expquad_derivs(-dsq / w, 2.0 * adotd / w, -aa / w, d[0]);
  } else if (pr->ic == ORC_IC_ADV_POLY) {
    double y[3];
    for (int a = 0; a < 3; ++a) y[a] = x[a] - pr->adv[a] * t;
    adv_poly_derivs(p, pr->adv, y, d[0]);
  } else if (pr->ic == ORC_IC_WAVE_PLANAR) {
    /* chi = (f(x - t) + f(x + t)) / 2, phi = chi_t */
    double s0 = p[0], w = p[1];
    double gm[6], gp[6];
    double sm = x[0] - t - s0, sp = x[0] + t - s0;
    expquad_derivs(-sm * sm / w, -2.0 * sm / w, -1.0 / w, gm);
    expquad_derivs(-sp * sp / w, -2.0 * sp / w, -1.0 / w, gp);
    double chi[7];
    for (int m = 0; m < 6; ++m) chi[m] = 0.5 * ((m % 2 ? -1.0 : 1.0) * gm[m] + gp[m]);
    for (int m = 0; m < 6; ++m) d[0][m] = chi[m];
    for (int m = 0; m < 5; ++m) d[1][m] = chi[m + 1];
    d[1][5] = 0.0; /* not needed by RK of order <= 4 */
  } else if (pr->ic == ORC_IC_WAVE_POLY) {
    const double* P = p;
    const double* Q = p + 64;
    double lP[64], lQ[64];
    poly_laplacian(P, lP);
    poly_laplacian(Q, lQ);
    double vP = poly_eval(P, x[0], x[1], x[2]), vQ = poly_eval(Q, x[0], x[1], x[2]);
    double vlP = poly_eval(lP, x[0], x[1], x[2]), vlQ = poly_eval(lQ, x[0], x[1], x[2]);
    double chi[6];
    chi[0] = vP + t * vQ + 0.5 * t * t * vlP + t * t * t / 6.0 * vlQ;
    chi[1] = vQ + t * vlP + 0.5 * t * t * vlQ;
    chi[2] = vlP + t * vlQ;
    chi[3] = vlQ;
    chi[4] = 0.0;
    chi[5] = 0.0;
    for (int m = 0; m < 6; ++m) d[0][m] = chi[m];
    for (int m = 0; m < 5; ++m) d[1][m] = chi[m + 1];
  } else if (pr->ic == ORC_IC_WAVE_SHELL) {
    /* r chi = (G(r - t) + G(r + t)) / 2, G(s) = s F(|s|) (odd), F = exp(-(s - R)^2 / w).
     * Time derivatives: d^m chi = ((-1)^m G^(m)(r - t) + G^(m)(r + t)) / (2 r). */
    double R = p[0], w = p[1];
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double Gm[7], Gp[7];
    double args[2] = {r - t, r + t};
    for (int q = 0; q < 2; ++q) {
      double s = args[q];
      double sa = fabs(s);
      double F[6];
      double z = sa - R;
      expquad_derivs(-z * z / w, -2.0 * z / w, -1.0 / w, F); /* derivatives of F at |s| */
      /* G(s) = s F(|s|) is odd: for s >= 0, G^(m)(s) = s F^(m)(s) + m F^(m-1)(s);
       * for s < 0, G^(m)(s) = (-1)^(m+1) G^(m)(|s|). */
      double* G = q ? Gp : Gm;
      for (int m = 0; m < 6; ++m) {
        double gpos = sa * F[m] + (m ? m * F[m - 1] : 0.0);
        G[m] = (s >= 0 || m % 2 == 1) ? gpos : -gpos;
      }
    }
    double chi[6];
    if (r > 1e-12) {
      for (int m = 0; m < 6; ++m) chi[m] = ((m % 2 ? -1.0 : 1.0) * Gm[m] + Gp[m]) / (2.0 * r);
    } else {
      /* r -> 0 limit: d/dr of the numerator / 2 = G^(m+1)(t) (even function of t for odd G) */
      for (int m = 0; m < 5; ++m) chi[m] = Gp[m + 1];
      chi[5] = 0.0;
    }
    for (int m = 0; m < 6; ++m) d[0][m] = chi[m];
    for (int m = 0; m < 5; ++m) d[1][m] = chi[m + 1];
  }
}

/* ------------------------------------------------------------------------ */
/* Solver state and the stage computation (Sec. 3.3-3.6)                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t src;   /* source octant, -1 = outside the domain */
  uint8_t r[3];  /* half-node coordinates in the source */
  uint8_t ext;   /* bit a set: coordinate a outside the closed domain */
} padent;

struct orc_solver {
  const orc_tree* t;
  orc_refine spec;
  orc_problem pr;
  int nf, p, l_min, l_max, L;
  double a[4][4], w[4], c[4];
  double omega[4][16]; /* 0 same level, 1 finer source, 2 coarser active, 3 coarser inactive (Fig. oct_2_1_nuts) */
  double gamma[16];
  double dt_f, t_macro;
  int64_t n_sub;
  int64_t N;
  size_t fsz; /* N * 343 */
  double *u, *u_start, *K, *tmp;
  padent** pad;
  padent** nodes;
};

int orc_solver_nf(const orc_solver* s) { return s->nf; }
double orc_solver_dt_f(const orc_solver* s) { return s->dt_f; }
double orc_solver_time(const orc_solver* s) { return s->t_macro + (double)s->n_sub * s->dt_f; }
int orc_solver_substep_index(const orc_solver* s) { return (int)s->n_sub; }

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

orc_solver* orc_solver_create(const orc_tree* t, const orc_refine* spec, const orc_problem* pr) {
  orc_solver* s = (orc_solver*)calloc(1, sizeof(orc_solver));
  s->t = t;
  s->spec = *spec;
  s->pr = *pr;
  s->nf = pr->pde == ORC_PDE_WAVE ? 2 : 1;
  s->p = orc_tableau(pr->rk, s->a, s->w, s->c);
  if (!s->p) {
    free(s);
    return NULL;
  }
  /* actual level range of the tree */
  int lmin = 99, lmax = -1;
  for (int l = 0; l <= ORC_D; ++l)
    if (t->level_count[l]) {
      if (l < lmin) lmin = l;
      if (l > lmax) lmax = l;
    }
  s->l_min = lmin;
  s->l_max = lmax;
  s->L = lmax - lmin;
  orc_omega(pr->rk, 0.0, 1.0, s->omega[0]);
  orc_omega(pr->rk, 0.0, 2.0, s->omega[1]);
  orc_omega(pr->rk, 0.0, 0.5, s->omega[2]);
  orc_omega(pr->rk, 0.5, 0.5, s->omega[3]);
  orc_stage_taylor(pr->rk, s->gamma);
  /* reading: dt_f = CFL * h at the finest level, h = node spacing */
  double h_f = (spec->hi - spec->lo) / (6.0 * (double)((int64_t)1 << lmax));
  s->dt_f = pr->cfl * h_f;
  s->N = t->n;
  s->fsz = (size_t)t->n * NV;
  size_t tot = s->fsz * (size_t)s->nf;
  s->u = (double*)calloc(tot, sizeof(double));
  s->u_start = (double*)calloc(tot, sizeof(double));
  s->tmp = (double*)calloc(tot, sizeof(double));
  s->K = (double*)calloc(tot * (size_t)s->p, sizeof(double));
  s->pad = (padent**)calloc((size_t)t->n, sizeof(padent*));
  s->nodes = (padent**)calloc((size_t)t->n, sizeof(padent*));
  if (!s->u || !s->u_start || !s->tmp || !s->K || !s->pad || !s->nodes) die("out of memory");
  ensure_W();
  return s;
}

void orc_solver_free(orc_solver* s) {
  if (!s) return;
  for (int64_t b = 0; b < s->N; ++b) {
    free(s->pad[b]);
    free(s->nodes[b]);
  }
  free(s->pad);
  free(s->nodes);
  free(s->u);
  free(s->u_start);
  free(s->tmp);
  free(s->K);
  free(s);
}

static int level_of(const orc_solver* s, int64_t b) { return s->t->oct[b].l; }
static double dt_level(const orc_solver* s, int l) { return s->dt_f * (double)((int64_t)1 << (s->l_max - l)); }

static double* fld(double* base, const orc_solver* s, int f, int64_t b) { return base + (size_t)f * s->fsz + (size_t)b * NV; }
static double* kfld(const orc_solver* s, int j, int f, int64_t b) {
  return s->K + ((size_t)j * s->nf + f) * s->fsz + (size_t)b * NV;
}

static void pos6_to_x(const orc_solver* s, const int64_t P[3], double x[3]) {
  double L = s->spec.hi - s->spec.lo;
  for (int a = 0; a < 3; ++a) x[a] = s->spec.lo + L * ((double)P[a] / (6.0 * (double)ROOT_EDGE));
}

static padent* get_pad(orc_solver* s, int64_t b) {
  if (s->pad[b]) return s->pad[b];
  padent* pe = (padent*)malloc(NT * sizeof(padent));
  const oct_t* o = &s->t->oct[b];
  int64_t e = edge_of(o->l);
  for (int k = -3; k <= 9; ++k)
    for (int j = -3; j <= 9; ++j)
      for (int i = -3; i <= 9; ++i) {
        int q = tix(i, j, k);
        int64_t P[3] = {6 * (int64_t)o->x + i * e, 6 * (int64_t)o->y + j * e, 6 * (int64_t)o->z + k * e};
        padent ent;
        ent.ext = 0;
        for (int a = 0; a < 3; ++a)
          if (P[a] < 0 || P[a] > L6) ent.ext |= (uint8_t)(1 << a);
        if (i >= 0 && i <= 6 && j >= 0 && j <= 6 && k >= 0 && k <= 6) {
          ent.src = (int32_t)b;
          ent.r[0] = (uint8_t)(2 * i);
          ent.r[1] = (uint8_t)(2 * j);
          ent.r[2] = (uint8_t)(2 * k);
        } else {
          int32_t rr[3] = {0, 0, 0};
          int64_t src = orc_point_source(s->t, P[0], P[1], P[2], rr);
          ent.src = (int32_t)src;
          for (int a = 0; a < 3; ++a) ent.r[a] = (uint8_t)(src >= 0 ? rr[a] : 0);
        }
        pe[q] = ent;
      }
  s->pad[b] = pe;
  return pe;
}

static padent* get_nodes(orc_solver* s, int64_t b) {
  if (s->nodes[b]) return s->nodes[b];
  padent* pe = (padent*)malloc(NV * sizeof(padent));
  const oct_t* o = &s->t->oct[b];
  int64_t e = edge_of(o->l);
  for (int k = 0; k < NP; ++k)
    for (int j = 0; j < NP; ++j)
      for (int i = 0; i < NP; ++i) {
        int32_t rr[3];
        int64_t src = orc_point_source(s->t, 6 * (int64_t)o->x + i * e, 6 * (int64_t)o->y + j * e,
                                       6 * (int64_t)o->z + k * e, rr);
        padent ent;
        ent.src = (int32_t)src;
        ent.ext = 0;
        for (int a = 0; a < 3; ++a) ent.r[a] = (uint8_t)rr[a];
        pe[i + NP * j + NP * NP * k] = ent;
      }
  s->nodes[b] = pe;
  return pe;
}

/* stage input of octant N at one node: u_N + dt_N sum_j om[j] k^N_j (zero weights
 * skipped), with u_N the state at the start of N's current step */
static double stage_value(const orc_solver* s, int f, int64_t N, int node, double dtN, const double* om) {
  double acc = 0.0;
  for (int j = 0; j < s->p; ++j) {
    if (om[j] == 0.0) continue;
    acc += om[j] * kfld(s, j, f, N)[node];
  }
  return fld(s->u_start, s, f, N)[node] + dtN * acc;
}

/* mutation 4: the end-of-step state instead of the step-start state */
static double stage_value_end(const orc_solver* s, int f, int64_t N, int node, double dtN, const double* om) {
  double acc = 0.0;
  for (int j = 0; j < s->p; ++j) {
    if (om[j] == 0.0) continue;
    acc += om[j] * kfld(s, j, f, N)[node];
  }
  return fld(s->u, s, f, N)[node] + dtN * acc;
}

/* cubic extrapolation weights from nodes 0..3 to position -m */
static void extrap_weights(int m, double E[4]) {
  for (int q = 0; q < 4; ++q) {
    double v = 1.0;
    for (int r = 0; r < 4; ++r)
      if (r != q) v *= (double)(-m - r) / (double)(q - r);
    E[q] = v;
  }
}

/* Radiative boundary (a reading of the paper): exterior ghosts by cubic extrapolation
 * along the outward normal, axis by axis (x, then y, then z). */
static void fill_extrapolated(const orc_solver* s, const oct_t* o, double* T) {
  int64_t e = edge_of(o->l);
  int64_t A[3] = {o->x, o->y, o->z};
  double E[4][4];
  for (int m = 1; m <= 3; ++m) extrap_weights(g_mutation == 7 ? m % 3 + 1 : m, E[m]); /* mutation 7: wrong row */
  for (int a = 0; a < 3; ++a) {
    int lo_bnd = (6 * A[a] == 0);
    int hi_bnd = (6 * (A[a] + e) == L6);
    if (!lo_bnd && !hi_bnd) continue;
    int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    for (int v2 = -3; v2 <= 9; ++v2)
      for (int v1 = -3; v1 <= 9; ++v1) {
        /* axes after a (in x,y,z order) must not be exterior; axes before a may be (already filled) */
        int idx[3];
        idx[b1] = v1;
        idx[b2] = v2;
        int skip = 0;
        int64_t Pb1 = 6 * A[b1] + v1 * e, Pb2 = 6 * A[b2] + v2 * e;
        if (b1 > a && (Pb1 < 0 || Pb1 > L6)) skip = 1;
        if (b2 > a && (Pb2 < 0 || Pb2 > L6)) skip = 1;
        if (skip) continue;
        (void)s;
        for (int m = 1; m <= 3; ++m) {
          if (lo_bnd) {
            double v = 0.0;
            for (int q = 0; q < 4; ++q) {
              idx[a] = q;
              v += E[m][q] * T[tix(idx[0], idx[1], idx[2])];
            }
            idx[a] = -m;
            T[tix(idx[0], idx[1], idx[2])] = v;
          }
          if (hi_bnd) {
            double v = 0.0;
            for (int q = 0; q < 4; ++q) {
              idx[a] = 6 - q;
              v += E[m][q] * T[tix(idx[0], idx[1], idx[2])];
            }
            idx[a] = 6 + m;
            T[tix(idx[0], idx[1], idx[2])] = v;
          }
        }
      }
  }
}

/* Unzip of one octant at one RK stage (Sec. 3.3, Fig. unzip): the padded 13^3
 * tile T[nf][2197] of stage inputs, with time-corrected neighbour stages
 * (eqs. fc_1, fc_2) and the physical boundary fill. */
static void unzip_tile(orc_solver* s, int64_t b, int st, int gts, int lstar, double* T /* [nf][2197] */) {
  const oct_t* o = &s->t->oct[b];
  int lb = o->l;
  double dtb = gts ? s->dt_f : dt_level(s, lb);
  double tb = orc_solver_time(s);
  int nf = s->nf;
  padent* pe = get_pad(s, b);
  int64_t e = edge_of(lb);

  /* stage inputs of every source that needs interpolation, computed once per octant-stage */
  int64_t isrc[27];
  int nisrc = 0;
  double* ival = (double*)malloc((size_t)27 * nf * NV * sizeof(double));
  for (int f = 0; f < nf; ++f) {
    double* Tf = T + (size_t)f * NT;
    for (int q = 0; q < NT; ++q) {
      padent ent = pe[q];
      if (ent.src < 0) {
        Tf[q] = 0.0;
        continue;
      }
      int64_t N = ent.src;
      int lN = level_of(s, N);
      int rel;
      double dtN;
      if (gts) {
        rel = 0;
        dtN = s->dt_f;
      } else {
        if (lN == lb)
          rel = 0;
        else if (lN == lb + 1)
          rel = 1;
        else if (lN == lb - 1)
          rel = (lN >= lstar) ? 2 : 3;
        else
          die("compute_stage: source violates 2:1 balance");
        dtN = dt_level(s, lN);
      }
      /* same level: the RK stage input itself (omega of the same-level relation is A) */
      const double* om = rel == 0 ? s->a[st] : s->omega[rel] + st * s->p;
      if (g_mutation == 1) om = s->a[st]; /* no time correction */
      if (N == b) dtN = dtb;
      int even = !(ent.r[0] & 1) && !(ent.r[1] & 1) && !(ent.r[2] & 1);
      if (g_mutation == 2 && !even) {  /* nearest coarse node instead of interpolation */
        ent.r[0] &= (uint8_t)~1u;
        ent.r[1] &= (uint8_t)~1u;
        ent.r[2] &= (uint8_t)~1u;
        even = 1;
      }
      if (even) {
        int node = ent.r[0] / 2 + NP * (ent.r[1] / 2) + NP * NP * (ent.r[2] / 2);
        Tf[q] = (g_mutation == 4 && rel == 3) ? stage_value_end(s, f, N, node, dtN, om)
                                              : stage_value(s, f, N, node, dtN, om);
      } else {
        int slot = -1;
        for (int c = 0; c < nisrc; ++c)
          if (isrc[c] == N) slot = c;
        if (slot < 0) {
          if (nisrc == 27) die("compute_stage: too many interpolation sources");
          slot = nisrc++;
          isrc[slot] = N;
          for (int ff = 0; ff < nf; ++ff)
            for (int n = 0; n < NV; ++n)
              ival[((size_t)slot * nf + ff) * NV + n] = (g_mutation == 4 && rel == 3)
                                                            ? stage_value_end(s, ff, N, n, dtN, om)
                                                            : stage_value(s, ff, N, n, dtN, om);
        }
        Tf[q] = orc_interp_point(ival + ((size_t)slot * nf + f) * NV, ent.r[0], ent.r[1], ent.r[2]);
      }
    }
  }
  free(ival);

  /* physical boundary */
  if (s->pr.bc == ORC_BC_EXACT) {
    for (int k = -3; k <= 9; ++k)
      for (int j = -3; j <= 9; ++j)
        for (int i = -3; i <= 9; ++i) {
          int q = tix(i, j, k);
          if (pe[q].src >= 0) continue;
          int64_t P[3] = {6 * (int64_t)o->x + i * e, 6 * (int64_t)o->y + j * e, 6 * (int64_t)o->z + k * e};
          double x[3], d[2][6];
          pos6_to_x(s, P, x);
          orc_exact_derivs(&s->pr, x, tb, d);
          for (int f = 0; f < nf; ++f) {
            double v = d[f][0], dtp = 1.0;
            for (int m = 0; m < s->p; ++m) {
              dtp *= dtb;
              v += s->gamma[st * s->p + m] * dtp * d[f][m + 1];
            }
            T[(size_t)f * NT + q] = v;
          }
        }
  } else {
    for (int f = 0; f < nf; ++f) fill_extrapolated(s, o, T + (size_t)f * NT);
  }
}

/* One RK stage of one octant (Alg. 2 compute_stage; Alg. 1 when gts != 0):
 * unzip into a padded 13^3 tile, then the FD right-hand side. */
static void compute_stage(orc_solver* s, int64_t b, int st, int gts, int lstar, double* kout /* [nf][343] */) {
  const oct_t* o = &s->t->oct[b];
  int lb = o->l;
  double dtb = gts ? s->dt_f : dt_level(s, lb);
  double tb = orc_solver_time(s);
  double* T = (double*)malloc((size_t)s->nf * NT * sizeof(double));
  int64_t e = edge_of(lb);
  unzip_tile(s, b, st, gts, lstar, T);

  /* right-hand side on the 7^3 interior */
  double h = (s->spec.hi - s->spec.lo) * (double)e / (6.0 * (double)ROOT_EDGE);
  double kos = s->pr.ko_sigma / (64.0 * h);
  for (int kk = 0; kk < NP; ++kk)
    for (int jj = 0; jj < NP; ++jj)
      for (int ii = 0; ii < NP; ++ii) {
        int n = ii + NP * jj + NP * NP * kk;
        if (s->pr.pde == ORC_PDE_ADVECTION) {
          double adv = 0.0, ko = 0.0;
          for (int a = 0; a < 3; ++a) {
            double v[7];
            stencil_line(T, ii, jj, kk, a, v);
            adv += s->pr.adv[a] * d1_of(v, h);
            ko += ko6_of(v);
          }
          kout[n] = (g_mutation == 3 ? adv : -adv) + kos * ko; /* mutation 3: wrong sign */
        } else {
          const double* Tc = T;
          const double* Tp = T + NT;
          double lap = 0.0, koc = 0.0, kop = 0.0;
          for (int a = 0; a < 3; ++a) {
            double v[7];
            stencil_line(Tc, ii, jj, kk, a, v);
            lap += d2_of(v, h);
            koc += ko6_of(v);
            stencil_line(Tp, ii, jj, kk, a, v);
            kop += ko6_of(v);
          }
          double phi = Tp[tix(ii, jj, kk)];
          kout[n] = phi + kos * koc;
          kout[NV + n] = lap + kos * kop;
          if (s->pr.nl_c != 0.0 || s->pr.orbit) {
            /* eq. phi: -c sin(2 chi)/r^2 (taken as 0 at r = 0); reading: orbiting
             * Gaussian sources at the stage time t_b + c_s dt_b */
            int64_t P[3] = {6 * (int64_t)o->x + ii * e, 6 * (int64_t)o->y + jj * e, 6 * (int64_t)o->z + kk * e};
            double x[3];
            pos6_to_x(s, P, x);
            double src = 0.0;
            if (s->pr.nl_c != 0.0) {
              double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
              if (r2 > 0.0) src -= s->pr.nl_c * sin(2.0 * Tc[tix(ii, jj, kk)]) / r2;
            }
            if (s->pr.orbit) {
              const double* op = s->pr.orbit_params;
              double ts = tb + s->c[st] * dtb;
              double c1 = op[0] * cos(op[1] * ts), s1 = op[0] * sin(op[1] * ts);
              double d1 = (x[0] - c1) * (x[0] - c1) + (x[1] - s1) * (x[1] - s1) + x[2] * x[2];
              double d2 = (x[0] + c1) * (x[0] + c1) + (x[1] + s1) * (x[1] + s1) + x[2] * x[2];
              src += op[3] * (exp(-d1 / op[2]) + exp(-d2 / op[2]));
            }
            kout[NV + n] += src;
          }
          if (s->pr.bc == ORC_BC_RADIATIVE) {
            int64_t P[3] = {6 * (int64_t)o->x + ii * e, 6 * (int64_t)o->y + jj * e, 6 * (int64_t)o->z + kk * e};
            int on_bnd = 0;
            for (int a = 0; a < 3; ++a)
              if (P[a] == 0 || P[a] == L6) on_bnd = 1;
            if (on_bnd) {
              /* reading: df/dt = -(x^i/r) d_i f - k_f (f - f0)/r, f0 = 0, k = 1 (chi), 2 (phi) */
              double x[3];
              pos6_to_x(s, P, x);
              double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
              for (int f = 0; f < 2; ++f) {
                const double* Tf = T + (size_t)f * NT;
                double xd = 0.0;
                for (int a = 0; a < 3; ++a) {
                  double v[7];
                  stencil_line(Tf, ii, jj, kk, a, v);
                  xd += x[a] * d1_of(v, h);
                }
                double fv = Tf[tix(ii, jj, kk)];
                double kf = f == 0 ? 1.0 : 2.0;
                if (g_mutation == 5) kf = 3.0 - kf; /* mutation 5: k of chi and phi swapped */
                if (g_mutation == 6) xd = -xd;      /* mutation 6: sign of the x^i/r term */
                kout[(size_t)f * NV + n] = -xd / r - kf * fv / r;
              }
            }
          }
        }
      }
  free(T);
}

/* ------------------------------------------------------------------------ */
/* Time stepping (Alg. 1, Alg. 2, Fig. blk_loop)                              */
/* ------------------------------------------------------------------------ */

/* Fig. blk_loop / reading: in substep n of a macro step, level l steps iff
 * n is a multiple of 2^(l_max - l); the active levels are l >= l*(n). */
int orc_active_level(int l_min, int l_max, int64_t n) {
  for (int l = l_min; l <= l_max; ++l)
    if (n % ((int64_t)1 << (l_max - l)) == 0) return l;
  return l_max;
}

void orc_set_initial(orc_solver* s, double t0) {
  const orc_tree* t = s->t;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < t->n; ++b) {
    const oct_t* o = &t->oct[b];
    int64_t e = edge_of(o->l);
    for (int n = 0; n < NV; ++n) {
      int i = n % NP, j = (n / NP) % NP, k = n / (NP * NP);
      int64_t P[3] = {6 * (int64_t)o->x + i * e, 6 * (int64_t)o->y + j * e, 6 * (int64_t)o->z + k * e};
      double x[3], d[2][6];
      pos6_to_x(s, P, x);
      orc_exact_derivs(&s->pr, x, t0, d);
      double v0 = d[0][0], v1 = d[1][0];
      if (s->pr.ic == ORC_IC_WAVE_SHELL) {
        /* reading: chi_0 = F(r) (1 + amp sum eps sin(kscale k.x + theta)), phi_0 = 0
         * (the shell data at rest, not the time derivative of the closed form) */
        const double* p = s->pr.ic_params;
        double amp = p[2], ks = p[4], pert = 0.0;
        int nm = (int)p[3];
        for (int m = 0; m < nm; ++m) {
          const double* md = p + 5 + 5 * m;
          pert += md[0] * sin(ks * (md[1] * x[0] + md[2] * x[1] + md[3] * x[2]) + md[4]);
        }
        double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]), z = r - p[0];
        v0 = exp(-z * z / p[1]) * (1.0 + amp * pert);
        v1 = 0.0;
      }
      fld(s->u, s, 0, b)[n] = v0;
      if (s->nf == 2) fld(s->u, s, 1, b)[n] = v1;
    }
  }
  /* the state at a synchronised time is the unzip of its shared-node values
   * (Sec. 3.3, Fig. dg_to_cg): hanging nodes take the coarse interpolant */
  orc_sync(s, s->u);
  memcpy(s->u_start, s->u, s->fsz * (size_t)s->nf * sizeof(double));
  memset(s->K, 0, s->fsz * (size_t)s->nf * (size_t)s->p * sizeof(double));
  s->t_macro = t0;
  s->n_sub = 0;
}

void orc_set_state(orc_solver* s, const double* u, double t0) {
  memcpy(s->u, u, s->fsz * (size_t)s->nf * sizeof(double));
  orc_sync(s, s->u);
  memcpy(s->u_start, s->u, s->fsz * (size_t)s->nf * sizeof(double));
  memset(s->K, 0, s->fsz * (size_t)s->nf * (size_t)s->p * sizeof(double));
  s->t_macro = t0;
  s->n_sub = 0;
}

/* The padded 13^3 block of octant b unzipped from the current state (Sec. 3.3,
 * Fig. unzip): the first RK stage's input with every neighbour at the same time
 * (Alg. 1 relation), physical boundary fill included.  T is [nf][2197]. */
void orc_solver_tile(orc_solver* s, int64_t b, double* T) { unzip_tile(s, b, 0, 1, s->l_min, T); }

void orc_get_state(const orc_solver* s, double* u) { memcpy(u, s->u, s->fsz * (size_t)s->nf * sizeof(double)); }

void orc_get_stage(const orc_solver* s, int stage, double* k) {
  memcpy(k, s->K + (size_t)stage * s->nf * s->fsz, s->fsz * (size_t)s->nf * sizeof(double));
}

void orc_exact_state(const orc_solver* s, double t, double* u) {
  const orc_tree* tr = s->t;
  for (int64_t b = 0; b < tr->n; ++b) {
    const oct_t* o = &tr->oct[b];
    int64_t e = edge_of(o->l);
    for (int n = 0; n < NV; ++n) {
      int i = n % NP, j = (n / NP) % NP, k = n / (NP * NP);
      int64_t P[3] = {6 * (int64_t)o->x + i * e, 6 * (int64_t)o->y + j * e, 6 * (int64_t)o->z + k * e};
      double x[3], d[2][6];
      pos6_to_x(s, P, x);
      orc_exact_derivs(&s->pr, x, t, d);
      for (int f = 0; f < s->nf; ++f) u[(size_t)f * s->fsz + (size_t)b * NV + n] = d[f][0];
    }
  }
}

/* DG -> shared nodes -> DG (zip then unzip, Sec. 3.3 / Fig. dg_to_cg; readings
 * the padding and ownership readings), in place.  Zip: every non-hanging node takes the value of its owner,
 * the coarsest leaf having it as a node (ties to the smallest Morton key).
 * Unzip: a hanging node is interpolated from the shared-node representation of
 * the coarser leaf containing it, whose own nodes are final once the coarser
 * levels are done -- so hanging nodes are filled level by level, coarse first. */
void orc_sync(orc_solver* s, double* v) {
  const orc_tree* t = s->t;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < t->n; ++b) get_nodes(s, b);
  /* zip: owners' values (owners keep theirs, so the pass is order-free) */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < t->n; ++b) {
    padent* pe = s->nodes[b];
    for (int f = 0; f < s->nf; ++f) {
      double* out = v + (size_t)f * s->fsz + (size_t)b * NV;
      for (int n = 0; n < NV; ++n) {
        padent ent = pe[n];
        if (ent.src == b) continue;
        if ((ent.r[0] & 1) || (ent.r[1] & 1) || (ent.r[2] & 1)) continue;
        out[n] = v[(size_t)f * s->fsz + (size_t)ent.src * NV + ent.r[0] / 2 + NP * (ent.r[1] / 2) +
                   NP * NP * (ent.r[2] / 2)];
      }
    }
  }
  /* unzip of hanging nodes, one level at a time */
  int64_t first = 0;
  for (int l = 0; l <= ORC_D; ++l) {
    int64_t cnt = t->level_count[l];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = first; b < first + cnt; ++b) {
      padent* pe = s->nodes[b];
      for (int f = 0; f < s->nf; ++f) {
        double* out = v + (size_t)f * s->fsz + (size_t)b * NV;
        for (int n = 0; n < NV; ++n) {
          padent ent = pe[n];
          if (!((ent.r[0] & 1) || (ent.r[1] & 1) || (ent.r[2] & 1))) continue;
          out[n] = orc_interp_point(v + (size_t)f * s->fsz + (size_t)ent.src * NV, ent.r[0], ent.r[1], ent.r[2]);
        }
      }
    }
    first += cnt;
  }
}

static void lts_substep(orc_solver* s, const uint8_t* mask, const uint8_t* fmask) {
  const orc_tree* t = s->t;
  int64_t N = t->n;
  int lstar = orc_active_level(s->l_min, s->l_max, s->n_sub);
  /* active octants: levels >= l* (a suffix of the level order) */
  int64_t first = 0;
  for (int l = 0; l < lstar; ++l) first += t->level_count[l];
  /* step start: V <- U for the active blocks (Alg. 2) */
  for (int f = 0; f < s->nf; ++f)
    memcpy(fld(s->u_start, s, f, first), fld(s->u, s, f, first), (size_t)(N - first) * NV * sizeof(double));
  for (int st = 0; st < s->p; ++st) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = first; b < N; ++b)
      if (!mask || mask[(size_t)st * N + b]) get_pad(s, b);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = first; b < N; ++b) {
      if (mask && !mask[(size_t)st * N + b]) continue;
      double kb[2 * NV];
      compute_stage(s, b, st, 0, lstar, kb);
      for (int f = 0; f < s->nf; ++f) memcpy(kfld(s, st, f, b), kb + (size_t)f * NV, NV * sizeof(double));
    }
  }
  /* compute_step_partial (Alg. 2): u = u_start + dt_l sum_i w_i k_i on the active blocks */
  for (int64_t b = first; b < N; ++b) {
    if (fmask && !fmask[b]) continue;
    double dtb = dt_level(s, level_of(s, b));
    for (int f = 0; f < s->nf; ++f) {
      double* u = fld(s->u, s, f, b);
      const double* u0 = fld(s->u_start, s, f, b);
      for (int n = 0; n < NV; ++n) {
        double acc = 0.0;
        for (int i = 0; i < s->p; ++i) acc += s->w[i] * kfld(s, i, f, b)[n];
        u[n] = u0[n] + dtb * acc;
      }
    }
  }
  s->n_sub++;
  if (s->n_sub == ((int64_t)1 << s->L)) {
    /* all blocks synchronised in time: reconcile the duplicated DG nodes */
    if (!mask && !fmask) orc_sync(s, s->u);
    s->t_macro += (double)s->n_sub * s->dt_f;
    s->n_sub = 0;
  }
}

void orc_lts_substeps(orc_solver* s, int64_t n) {
  for (int64_t i = 0; i < n; ++i) lts_substep(s, NULL, NULL);
}

void orc_lts_substep_masked(orc_solver* s, const uint8_t* mask, const uint8_t* fmask) { lts_substep(s, mask, fmask); }

/* Alg. 1: every block steps with dt_f; blk_sync of each stage and of the step */
void orc_gts_steps(orc_solver* s, int64_t nsteps) {
  const orc_tree* t = s->t;
  int64_t N = t->n;
  for (int64_t it = 0; it < nsteps; ++it) {
    memcpy(s->u_start, s->u, s->fsz * (size_t)s->nf * sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < N; ++b) get_pad(s, b);
    for (int st = 0; st < s->p; ++st) {
#pragma omp parallel for schedule(dynamic, 4)
      for (int64_t b = 0; b < N; ++b) {
        double kb[2 * NV];
        compute_stage(s, b, st, 1, s->l_min, kb);
        for (int f = 0; f < s->nf; ++f) memcpy(kfld(s, st, f, b), kb + (size_t)f * NV, NV * sizeof(double));
      }
      orc_sync(s, s->K + (size_t)st * s->nf * s->fsz);
    }
    for (int64_t b = 0; b < N; ++b)
      for (int f = 0; f < s->nf; ++f) {
        double* u = fld(s->u, s, f, b);
        const double* u0 = fld(s->u_start, s, f, b);
        for (int n = 0; n < NV; ++n) {
          double acc = 0.0;
          for (int i = 0; i < s->p; ++i) acc += s->w[i] * kfld(s, i, f, b)[n];
          u[n] = u0[n] + s->dt_f * acc;
        }
      }
    orc_sync(s, s->u);
    s->n_sub++;
    if (s->n_sub == ((int64_t)1 << s->L)) {
      s->t_macro += (double)s->n_sub * s->dt_f;
      s->n_sub = 0;
    }
  }
}

/* eqs. w_nuts, w_uts, invS (reading: alpha_l counts octants at level l_max - l) */
double orc_work_model(const orc_tree* t, double* w_lts, double* w_gts) {
  int lmin = 99, lmax = -1;
  for (int l = 0; l <= ORC_D; ++l)
    if (t->level_count[l]) {
      if (l < lmin) lmin = l;
      if (l > lmax) lmax = l;
    }
  int L = lmax - lmin;
  double wl = 0.0, total = 0.0;
  for (int l = 0; l <= L; ++l) {
    double alpha = (double)t->level_count[lmax - l];
    wl += pow(2.0, L - l) * alpha;
    total += alpha;
  }
  double wg = pow(2.0, L) * total;
  if (w_lts) *w_lts = wl;
  if (w_gts) *w_gts = wg;
  return wg / wl;
}
