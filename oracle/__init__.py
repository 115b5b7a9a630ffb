"""CPU oracle for local timestepping on 2:1-balanced octrees (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never does, and it shares no code with it.

The C source (``lts_oracle.c``) is a plain FP64 restatement of the paper's
method (Fernando & Sundar, "Scalable Local Timestepping on Octree Grids"):
octree construction and 2:1 balance (Sec. 3.2), padding sources and the
shared-node synchronisation (Sec. 3.3, Fig. dg_to_cg), finite differences with
Kreiss-Oliger dissipation, RK stages (eq. rk_schemes), the LTS stage
corrections (eqs. rk_crrection, fc_1, fc_2), GTS (Alg. 1), LTS (Alg. 2,
Fig. blk_loop) and the speedup model (eqs. w_nuts, w_uts, invS).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblts_oracle.so")
_lock = threading.Lock()
_lib = None

NV = 343
NT = 2197


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -ffp-contract=off, OpenMP)."""
    src = os.path.join(_HERE, "lts_oracle.c")
    hdr = os.path.join(_HERE, "lts_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Refine(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double), ("l_min", C.c_int), ("l_max", C.c_int),
                ("kind", C.c_int), ("n_centers", C.c_int), ("centers", (C.c_double * 3) * 8),
                ("radius", C.c_double), ("band", C.c_double), ("eps", C.c_double)]


class Problem(C.Structure):
    _fields_ = [("pde", C.c_int), ("adv", C.c_double * 3), ("cfl", C.c_double),
                ("ko_sigma", C.c_double), ("rk", C.c_int), ("bc", C.c_int), ("ic", C.c_int),
                ("ic_params", C.c_double * 160), ("nl_c", C.c_double), ("orbit", C.c_int),
                ("orbit_params", C.c_double * 4)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            vp, i64, i32p = C.c_void_p, C.c_int64, C.POINTER(C.c_int32)
            dp = C.POINTER(C.c_double)
            L.orc_morton.restype = C.c_uint64
            L.orc_morton.argtypes = [C.c_uint32] * 3
            for name in ("orc_tree_build", "orc_tree_refine_only"):
                getattr(L, name).restype = vp
                getattr(L, name).argtypes = [C.POINTER(Refine)]
            L.orc_tree_from_leaves.restype = vp
            L.orc_tree_from_leaves.argtypes = [C.c_double, C.c_double, i64, i32p, i32p]
            L.orc_tree_free.argtypes = [vp]
            L.orc_tree_size.restype = i64
            L.orc_tree_size.argtypes = [vp]
            L.orc_tree_export.argtypes = [vp, i32p, i32p]
            L.orc_refine_pred.restype = C.c_int
            L.orc_refine_pred.argtypes = [C.POINTER(Refine), C.c_int32, C.c_int32, C.c_int32, C.c_int]
            L.orc_wavelet_coeff.restype = C.c_double
            L.orc_wavelet_coeff.argtypes = [C.POINTER(Refine), C.c_int32, C.c_int32, C.c_int32, C.c_int]
            L.orc_find_leaf.restype = i64
            L.orc_find_leaf.argtypes = [vp, i64, i64, i64]
            L.orc_o2o.argtypes = [vp, i32p]
            L.orc_point_source.restype = i64
            L.orc_point_source.argtypes = [vp, i64, i64, i64, i32p]
            L.orc_pad_map.argtypes = [vp, i64, i32p, i32p]
            L.orc_node_map.argtypes = [vp, i64, i32p, i32p]
            L.orc_interp_weights.argtypes = [dp]
            L.orc_interp_point.restype = C.c_double
            L.orc_interp_point.argtypes = [dp, C.c_int, C.c_int, C.c_int]
            L.orc_tile_ops.argtypes = [dp, C.c_double, dp, dp, dp]
            L.orc_tableau.restype = C.c_int
            L.orc_tableau.argtypes = [C.c_int, dp, dp, dp]
            L.orc_omega.restype = C.c_int
            L.orc_omega.argtypes = [C.c_int, C.c_double, C.c_double, dp]
            L.orc_stage_taylor.restype = C.c_int
            L.orc_stage_taylor.argtypes = [C.c_int, dp]
            L.orc_exact_derivs.argtypes = [C.POINTER(Problem), dp, C.c_double, dp]
            L.orc_solver_create.restype = vp
            L.orc_solver_create.argtypes = [vp, C.POINTER(Refine), C.POINTER(Problem)]
            L.orc_solver_free.argtypes = [vp]
            L.orc_solver_nf.restype = C.c_int
            L.orc_solver_nf.argtypes = [vp]
            L.orc_solver_dt_f.restype = C.c_double
            L.orc_solver_dt_f.argtypes = [vp]
            L.orc_solver_time.restype = C.c_double
            L.orc_solver_time.argtypes = [vp]
            L.orc_solver_substep_index.restype = C.c_int
            L.orc_solver_substep_index.argtypes = [vp]
            L.orc_set_initial.argtypes = [vp, C.c_double]
            L.orc_set_state.argtypes = [vp, dp, C.c_double]
            L.orc_get_state.argtypes = [vp, dp]
            L.orc_get_stage.argtypes = [vp, C.c_int, dp]
            L.orc_solver_tile.argtypes = [vp, i64, dp]
            L.orc_exact_state.argtypes = [vp, C.c_double, dp]
            L.orc_lts_substeps.argtypes = [vp, i64]
            L.orc_lts_substep_masked.argtypes = [vp, C.POINTER(C.c_uint8), C.POINTER(C.c_uint8)]
            L.orc_gts_steps.argtypes = [vp, i64]
            L.orc_sync.argtypes = [vp, dp]
            L.orc_active_level.restype = C.c_int
            L.orc_active_level.argtypes = [C.c_int, C.c_int, i64]
            L.orc_work_model.restype = C.c_double
            L.orc_work_model.argtypes = [vp, dp, dp]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_mutation.argtypes = [C.c_int]
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def make_refine(spec: dict) -> Refine:
    r = Refine()
    r.lo, r.hi = spec["lo"], spec["hi"]
    r.l_min, r.l_max = spec["l_min"], spec["l_max"]
    r.kind = spec["kind"]
    cents = spec.get("centers", [])
    r.n_centers = len(cents)
    for i, c in enumerate(cents):
        for d in range(3):
            r.centers[i][d] = c[d]
    r.radius = spec.get("radius", 0.0)
    r.band = spec.get("band", 0.0)
    r.eps = spec.get("eps", 0.0)
    return r


def make_problem(prob: dict) -> Problem:
    p = Problem()
    p.pde = prob["pde"]
    for d in range(3):
        p.adv[d] = prob.get("adv", (0.0, 0.0, 0.0))[d]
    p.cfl = prob["cfl"]
    p.ko_sigma = prob["ko_sigma"]
    p.rk = prob["rk"]
    p.bc = prob["bc"]
    p.ic = prob["ic"]
    params = list(prob.get("ic_params", []))
    for i, v in enumerate(params):
        p.ic_params[i] = v
    p.nl_c = prob.get("nl_c", 0.0)
    p.orbit = int(prob.get("orbit", 0))
    for i, v in enumerate(prob.get("orbit_params", [])):
        p.orbit_params[i] = v
    return p


class Tree:
    """An octree in level order; wraps ``orc_tree``."""

    def __init__(self, handle, spec=None):
        self.h = handle
        self.spec = spec
        if not handle:
            raise ValueError("oracle: invalid refinement spec")

    @classmethod
    def build(cls, spec: dict):
        return cls(lib().orc_tree_build(C.byref(make_refine(spec))), spec)

    @classmethod
    def refine_only(cls, spec: dict):
        return cls(lib().orc_tree_refine_only(C.byref(make_refine(spec))), spec)

    @classmethod
    def from_leaves(cls, lo, hi, xyz, level):
        xyz = np.ascontiguousarray(xyz, dtype=np.int32)
        level = np.ascontiguousarray(level, dtype=np.int32)
        return cls(lib().orc_tree_from_leaves(lo, hi, len(level), _p(xyz, C.c_int32), _p(level, C.c_int32)),
                   {"lo": lo, "hi": hi})

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_tree_free(self.h)
            self.h = None

    def __len__(self):
        return lib().orc_tree_size(self.h)

    def export(self):
        n = len(self)
        xyz = np.zeros((n, 3), np.int32)
        lev = np.zeros(n, np.int32)
        lib().orc_tree_export(self.h, _p(xyz, C.c_int32), _p(lev, C.c_int32))
        return xyz, lev

    def find_leaf(self, x, y, z):
        return lib().orc_find_leaf(self.h, x, y, z)

    def o2o(self):
        out = np.zeros((len(self), 27, 8), np.int32)
        lib().orc_o2o(self.h, _p(out, C.c_int32))
        return out

    def point_source(self, px, py, pz):
        r = np.zeros(3, np.int32)
        s = lib().orc_point_source(self.h, px, py, pz, _p(r, C.c_int32))
        return s, r

    def pad_map(self, b):
        src = np.zeros(NT, np.int32)
        r = np.zeros((NT, 3), np.int32)
        lib().orc_pad_map(self.h, b, _p(src, C.c_int32), _p(r, C.c_int32))
        return src, r

    def node_map(self, b):
        src = np.zeros(NV, np.int32)
        r = np.zeros((NV, 3), np.int32)
        lib().orc_node_map(self.h, b, _p(src, C.c_int32), _p(r, C.c_int32))
        return src, r

    def work_model(self):
        wl = C.c_double()
        wg = C.c_double()
        s = lib().orc_work_model(self.h, C.byref(wl), C.byref(wg))
        return s, wl.value, wg.value


class Solver:
    """LTS / GTS state on a tree (DG layout [nf][N][343], level order)."""

    def __init__(self, tree: Tree, spec: dict, prob: dict):
        self.tree = tree
        self.spec = spec
        self.prob = prob
        self._r = make_refine(spec)
        self._pr = make_problem(prob)
        self.h = lib().orc_solver_create(tree.h, C.byref(self._r), C.byref(self._pr))
        if not self.h:
            raise ValueError("oracle: invalid problem")
        self.nf = lib().orc_solver_nf(self.h)
        self.n = len(tree)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_solver_free(self.h)
            self.h = None

    @property
    def dt_f(self):
        return lib().orc_solver_dt_f(self.h)

    @property
    def time(self):
        return lib().orc_solver_time(self.h)

    @property
    def substep_index(self):
        return lib().orc_solver_substep_index(self.h)

    def set_initial(self, t0=0.0):
        lib().orc_set_initial(self.h, t0)

    def set_state(self, u, t0=0.0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == self.nf * self.n * NV
        lib().orc_set_state(self.h, _p(u, C.c_double), t0)

    def state(self):
        u = np.zeros((self.nf, self.n, NV))
        lib().orc_get_state(self.h, _p(u, C.c_double))
        return u

    def stage(self, j):
        k = np.zeros((self.nf, self.n, NV))
        lib().orc_get_stage(self.h, j, _p(k, C.c_double))
        return k

    def tile(self, b):
        """padded 13^3 block [nf][13][13][13] (k, j, i order) of octant b from the current state"""
        T = np.zeros((self.nf, 13, 13, 13))
        lib().orc_solver_tile(self.h, int(b), _p(T, C.c_double))
        return T

    def exact(self, t):
        u = np.zeros((self.nf, self.n, NV))
        lib().orc_exact_state(self.h, t, _p(u, C.c_double))
        return u

    def lts_substeps(self, n):
        lib().orc_lts_substeps(self.h, n)

    def lts_substep_masked(self, mask, fmask):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        fmask = np.ascontiguousarray(fmask, dtype=np.uint8)
        lib().orc_lts_substep_masked(self.h, _p(mask, C.c_uint8), _p(fmask, C.c_uint8))

    def gts_steps(self, n):
        lib().orc_gts_steps(self.h, n)

    def sync(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64).copy()
        lib().orc_sync(self.h, _p(v, C.c_double))
        return v


def morton(x, y, z):
    return lib().orc_morton(x, y, z)


def interp_weights():
    W = np.zeros((13, 7))
    lib().orc_interp_weights(_p(W, C.c_double))
    return W


def interp_point(v343, rx, ry, rz):
    v = np.ascontiguousarray(v343, dtype=np.float64)
    return lib().orc_interp_point(_p(v, C.c_double), rx, ry, rz)


def tile_ops(tile, h):
    t = np.ascontiguousarray(tile, dtype=np.float64).reshape(NT)
    d1 = np.zeros((3, NV))
    d2 = np.zeros((3, NV))
    ko = np.zeros((3, NV))
    lib().orc_tile_ops(_p(t, C.c_double), h, _p(d1, C.c_double), _p(d2, C.c_double), _p(ko, C.c_double))
    return d1, d2, ko


def tableau(rk):
    a = np.zeros((4, 4))
    w = np.zeros(4)
    c = np.zeros(4)
    p = lib().orc_tableau(rk, _p(a, C.c_double), _p(w, C.c_double), _p(c, C.c_double))
    return p, a[:p, :p], w[:p], c[:p]


def omega(rk, theta, rho):
    om = np.zeros(16)
    p = lib().orc_omega(rk, theta, rho, _p(om, C.c_double))
    return om[:p * p].reshape(p, p)


def stage_taylor(rk):
    g = np.zeros(16)
    p = lib().orc_stage_taylor(rk, _p(g, C.c_double))
    return g[:p * p].reshape(p, p)


def exact_derivs(prob: dict, x, t):
    pr = make_problem(prob)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    d = np.zeros((2, 6))
    lib().orc_exact_derivs(C.byref(pr), _p(xx, C.c_double), t, _p(d, C.c_double))
    return d


def active_level(l_min, l_max, n):
    return lib().orc_active_level(l_min, l_max, n)


def set_mutation(m):
    """Negative controls for the tests only (0 = the method as stated)."""
    lib().orc_set_mutation(m)


def set_threads(n):
    lib().orc_set_threads(n)


def refine_pred(spec, x, y, z, level):
    return lib().orc_refine_pred(C.byref(make_refine(spec)), x, y, z, level)


def wavelet_coeff(spec, x, y, z, level):
    return lib().orc_wavelet_coeff(C.byref(make_refine(spec)), x, y, z, level)
