"""Thin Python binding of libltsoct (include/ltsoct.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  PyTorch supplies
device memory (its caching allocator is passed to the library as the device
allocator) and the CUDA stream.  There is no CPU fallback: importing this module
without the compiled library, or using it without a GPU, raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

# lts_status codes (include/ltsoct.h)
LTS_OK, LTS_EINVAL, LTS_ENOMEM, LTS_ECUDA, LTS_ETIMEOUT, LTS_EUNBALANCED, LTS_ESTATE, LTS_EINTERNAL = range(8)


class LtsError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.lts_last_error().decode() if _lib else ""
        super().__init__("%s: %s (%s)" % (where, _lib.lts_strerror(status).decode() if _lib else status, msg))
        self.status = status


class RefineSpec(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double), ("l_min", C.c_int), ("l_max", C.c_int),
                ("kind", C.c_int), ("n_centers", C.c_int), ("centers", (C.c_double * 3) * 8),
                ("radius", C.c_double), ("band", C.c_double), ("eps", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Problem(C.Structure):
    _fields_ = [("pde", C.c_int), ("adv", C.c_double * 3), ("cfl", C.c_double), ("ko_sigma", C.c_double),
                ("rk", C.c_int), ("bc", C.c_int), ("ic", C.c_int), ("ic_params", C.c_double * 32),
                ("precision", C.c_int), ("stream", C.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("nl_c", C.c_double), ("orbit", C.c_int), ("orbit_params", C.c_double * 4)]


class Stats(C.Structure):
    _fields_ = [("n_octants", C.c_int64), ("nf", C.c_int), ("p", C.c_int), ("l_min", C.c_int), ("l_max", C.c_int),
                ("octants_per_level", C.c_int64 * 32), ("dt_finest", C.c_double), ("dt_coarsest", C.c_double),
                ("time", C.c_double), ("substep", C.c_int64), ("model_speedup", C.c_double),
                ("lts_work_per_macro", C.c_double), ("gts_work_per_macro", C.c_double),
                ("device_bytes", C.c_size_t), ("kernel_launches", C.c_int64),
                ("blocked_octants", C.c_int64)]


EXPORTS = ["octree_build", "octree_size", "octree_export", "octree_destroy", "lts_plan_create", "lts_plan_destroy",
           "lts_plan_stats", "lts_set_initial", "lts_set_state", "lts_get_state", "lts_get_stage",
           "lts_run_substeps", "lts_advance", "gts_steps", "gts_advance", "lts_export_o2o", "lts_export_pad_map",
           "lts_export_node_map", "lts_export_pad_map_static", "lts_set_blocking", "lts_set_profiling",
           "lts_kernel_stats", "lts_prolong_stats", "lts_batch_create", "lts_batch_destroy", "lts_batch_run",
           "lts_batch_set_grid", "lts_batch_stats", "lts_batch_create_slots", "lts_batch_attach",
           "lts_batch_detach", "lts_batch_set_mode", "lts_batch_wait", "lts_batch_probe_barrier", "lts_strerror",
           "lts_last_error"]


def library_path():
    return _build.LIB


def load(path=None):
    """Load libltsoct.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError("libltsoct.so not built (%s): run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    vp, i64, st = C.c_void_p, C.c_int64, C.c_int
    i32p, dp = C.POINTER(C.c_int32), C.c_void_p
    sig = {
        "octree_build": ([C.POINTER(RefineSpec), C.POINTER(vp)], st),
        "octree_size": ([vp, C.POINTER(i64)], st),
        "octree_export": ([vp, i32p, i32p], st),
        "octree_destroy": ([vp], None),
        "lts_plan_create": ([vp, C.POINTER(Problem), C.POINTER(vp)], st),
        "lts_plan_destroy": ([vp], None),
        "lts_plan_stats": ([vp, C.POINTER(Stats)], st),
        "lts_set_initial": ([vp, C.c_double], st),
        "lts_set_state": ([vp, dp, C.c_double, C.c_int], st),
        "lts_get_state": ([vp, dp, C.POINTER(C.c_double), C.c_int], st),
        "lts_get_stage": ([vp, C.c_int, dp, C.c_int], st),
        "lts_run_substeps": ([vp, i64], st),
        "lts_advance": ([vp, C.c_double], st),
        "gts_steps": ([vp, i64], st),
        "gts_advance": ([vp, C.c_double], st),
        "lts_export_o2o": ([vp, i32p], st),
        "lts_export_pad_map": ([vp, i32p, i64, i32p, i32p], st),
        "lts_export_node_map": ([vp, i32p, i64, i32p, i32p], st),
        "lts_export_pad_map_static": ([vp, i32p, i64, i32p, i32p], st),
        "lts_set_blocking": ([vp, C.c_int], st),
        "lts_set_profiling": ([vp, C.c_int], st),
        "lts_kernel_stats": ([vp, C.POINTER(i64), C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(i64), C.c_int], st),
        "lts_prolong_stats": ([vp, C.POINTER(i64), C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(i64), C.c_int], st),
        "lts_batch_create": ([C.POINTER(vp), C.c_int, C.POINTER(vp)], st),
        "lts_batch_destroy": ([vp], None),
        "lts_batch_run": ([vp, C.POINTER(i64), C.c_int], st),
        "lts_batch_set_grid": ([vp, C.c_int, C.c_int, C.c_int], st),
        "lts_batch_stats": ([vp, C.POINTER(i64), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], st),
        "lts_batch_create_slots": ([C.c_int, vp, C.c_int, C.POINTER(vp)], st),
        "lts_batch_attach": ([vp, C.c_int, vp], st),
        "lts_batch_detach": ([vp, C.c_int], st),
        "lts_batch_set_mode": ([vp, C.c_int, C.c_int], st),
        "lts_batch_wait": ([vp], st),
        "lts_batch_probe_barrier": ([vp, C.c_int, C.c_double], st),
        "lts_strerror": ([st], C.c_char_p),
        "lts_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status, where):
    if status != 0:
        raise LtsError(status, where)


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def make_refine(spec: dict) -> RefineSpec:
    r = RefineSpec()
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


class Octree:
    """octree_build / octree_size / octree_export / octree_destroy."""

    def __init__(self, spec: dict):
        L = load()
        self.spec = spec
        self._spec = make_refine(spec)
        h = C.c_void_p()
        _check(L.octree_build(C.byref(self._spec), C.byref(h)), "octree_build")
        self.h = h

    def __len__(self):
        n = C.c_int64()
        _check(_lib.octree_size(self.h, C.byref(n)), "octree_size")
        return n.value

    def export(self):
        n = len(self)
        xyz = np.zeros((n, 3), np.int32)
        lev = np.zeros(n, np.int32)
        _check(_lib.octree_export(self.h, _i32(xyz), _i32(lev)), "octree_export")
        return xyz, lev

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.octree_destroy(self.h)
            self.h = None


class Plan:
    """lts_plan_* entry points.  State arrays are torch CUDA tensors or numpy arrays of
    shape (nf, N, 343), float64, in level order."""

    def __init__(self, tree: Octree, prob: dict, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libltsoct needs a CUDA GPU; no CPU fallback exists")
        L = load()
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
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
        if len(params) > 32:
            raise ValueError("at most 32 initial-data parameters")
        for i, v in enumerate(params):
            p.ic_params[i] = v
        p.precision = int(prob.get("precision", 0))
        p.nl_c = float(prob.get("nl_c", 0.0))
        p.orbit = int(prob.get("orbit", 0))
        for i, v in enumerate(prob.get("orbit_params", ())):
            p.orbit_params[i] = v
        p.stream = self.stream.cuda_stream
        dev, strm = self.device, self.stream

        def _alloc(nbytes, ctx):
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        p.dev_alloc = self._alloc_cb
        p.dev_free = self._free_cb
        self._prob = p
        self.tree = tree
        h = C.c_void_p()
        _check(L.lts_plan_create(tree.h, C.byref(p), C.byref(h)), "lts_plan_create")
        self.h = h
        self.stats_ = self.stats()
        self.n = self.stats_["n_octants"]
        self.nf = self.stats_["nf"]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lts_plan_destroy(self.h)
            self.h = None

    def stats(self):
        s = Stats()
        _check(_lib.lts_plan_stats(self.h, C.byref(s)), "lts_plan_stats")
        out = {k: getattr(s, k) for k, _ in Stats._fields_}
        out["octants_per_level"] = list(s.octants_per_level)
        return out

    def set_initial(self, t0=0.0):
        _check(_lib.lts_set_initial(self.h, t0), "lts_set_initial")

    def _buf(self, arr, writable):
        t = self.torch
        if isinstance(arr, t.Tensor):
            assert arr.dtype == t.float64 and arr.is_contiguous() and arr.numel() == self.nf * self.n * 343
            return C.c_void_p(arr.data_ptr()), 1 if arr.is_cuda else 0
        assert arr.dtype == np.float64 and arr.flags["C_CONTIGUOUS"] and arr.size == self.nf * self.n * 343
        return C.c_void_p(arr.ctypes.data), 0

    def set_state(self, u, t0=0.0):
        ptr, dev = self._buf(u, False)
        _check(_lib.lts_set_state(self.h, ptr, t0, dev), "lts_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((self.nf, self.n, 343))
        ptr, dev = self._buf(out, True)
        t = C.c_double()
        _check(_lib.lts_get_state(self.h, ptr, C.byref(t), dev), "lts_get_state")
        return out

    def get_stage(self, j, out=None):
        if out is None:
            out = np.zeros((self.nf, self.n, 343))
        ptr, dev = self._buf(out, True)
        _check(_lib.lts_get_stage(self.h, j, ptr, dev), "lts_get_stage")
        return out

    @property
    def time(self):
        return self.stats()["time"]

    def run_substeps(self, n):
        _check(_lib.lts_run_substeps(self.h, n), "lts_run_substeps")

    def advance(self, t_end):
        _check(_lib.lts_advance(self.h, t_end), "lts_advance")

    def gts_steps(self, n):
        _check(_lib.gts_steps(self.h, n), "gts_steps")

    def gts_advance(self, t_end):
        _check(_lib.gts_advance(self.h, t_end), "gts_advance")

    def export_o2o(self):
        out = np.zeros((self.n, 27, 8), np.int32)
        _check(_lib.lts_export_o2o(self.h, _i32(out)), "lts_export_o2o")
        return out

    def export_pad_map(self, octs):
        octs = np.ascontiguousarray(octs, dtype=np.int32)
        src = np.zeros((len(octs), 2197), np.int32)
        r = np.zeros((len(octs), 2197, 3), np.int32)
        _check(_lib.lts_export_pad_map(self.h, _i32(octs), len(octs), _i32(src), _i32(r)), "lts_export_pad_map")
        return src, r

    def export_pad_map_static(self, octs):
        """lts_export_pad_map without per-call device allocation (at most 32 octants)."""
        octs = np.ascontiguousarray(octs, dtype=np.int32)
        src = np.zeros((len(octs), 2197), np.int32)
        r = np.zeros((len(octs), 2197, 3), np.int32)
        _check(_lib.lts_export_pad_map_static(self.h, _i32(octs), len(octs), _i32(src), _i32(r)),
               "lts_export_pad_map_static")
        return src, r

    def export_node_map(self, octs):
        octs = np.ascontiguousarray(octs, dtype=np.int32)
        src = np.zeros((len(octs), 343), np.int32)
        r = np.zeros((len(octs), 343, 3), np.int32)
        _check(_lib.lts_export_node_map(self.h, _i32(octs), len(octs), _i32(src), _i32(r)), "lts_export_node_map")
        return src, r

    def set_blocking(self, on=True):
        """step complete sibling groups as 13^3-node blocks (default on; bit-identical results)"""
        _check(_lib.lts_set_blocking(self.h, 1 if on else 0), "lts_set_blocking")

    def set_profiling(self, on=True):
        _check(_lib.lts_set_profiling(self.h, 1 if on else 0), "lts_set_profiling")

    def kernel_stats(self, reset=True):
        n = C.c_int64()
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        ns = C.c_int64()
        _check(_lib.lts_kernel_stats(self.h, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by), C.byref(ns),
                                     1 if reset else 0), "lts_kernel_stats")
        return dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value, node_stages=ns.value)

    def prolong_stats(self, reset=True):
        n, src = C.c_int64(), C.c_int64()
        ms, fl = C.c_double(), C.c_double()
        _check(_lib.lts_prolong_stats(self.h, C.byref(n), C.byref(ms), C.byref(fl), C.byref(src),
                                      1 if reset else 0), "lts_prolong_stats")
        return dict(launches=n.value, ms=ms.value, flops=fl.value, sources=src.value)


class Batch:
    """lts_batch_*: several plans advanced together, one persistent launch per stage.
    Batch(plans) binds a fixed list; Batch.slots(n, stream, precision) creates an empty
    batch whose slots are filled and emptied with attach / detach."""

    def __init__(self, plans=None, _handle=None, _n=0):
        L = load()
        if _handle is not None:
            self.h = _handle
            self.plans = [None] * _n
            return
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.h.value for p in self.plans])
        h = C.c_void_p()
        _check(L.lts_batch_create(arr, len(self.plans), C.byref(h)), "lts_batch_create")
        self.h = h

    @classmethod
    def slots(cls, n, stream, precision=0):
        L = load()
        h = C.c_void_p()
        _check(L.lts_batch_create_slots(n, C.c_void_p(stream.cuda_stream), precision, C.byref(h)),
               "lts_batch_create_slots")
        return cls(_handle=h, _n=n)

    def attach(self, slot, plan):
        _check(_lib.lts_batch_attach(self.h, slot, plan.h), "lts_batch_attach")
        self.plans[slot] = plan

    def detach(self, slot):
        _check(_lib.lts_batch_detach(self.h, slot), "lts_batch_detach")
        self.plans[slot] = None

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lts_batch_destroy(self.h)
            self.h = None

    def run(self, substeps, graph=True):
        """advance plan i by substeps[i] substeps (asynchronous)"""
        arr = np.ascontiguousarray(substeps, dtype=np.int64)
        assert len(arr) == len(self.plans)
        _check(_lib.lts_batch_run(self.h, arr.ctypes.data_as(C.POINTER(C.c_int64)), 1 if graph else 0),
               "lts_batch_run")

    def set_grid(self, stage, prolong, sync):
        _check(_lib.lts_batch_set_grid(self.h, stage, prolong, sync), "lts_batch_set_grid")

    def set_mode(self, persistent=True, ctas_per_sm=1):
        """persistent: one cooperative launch per round (ctas_per_sm CTAs per SM); else
        the per-stage launches"""
        _check(_lib.lts_batch_set_mode(self.h, 1 if persistent else 0, int(ctas_per_sm)), "lts_batch_set_mode")

    def wait(self):
        """synchronise; raises LtsError (LTS_ETIMEOUT) if a round's grid barrier timed out"""
        _check(_lib.lts_batch_wait(self.h), "lts_batch_wait")

    def probe_barrier(self, absent_cta=-1, limit_s=0.05):
        """the grid barrier alone; returns the status (0 ok, LTS_ETIMEOUT when a CTA is absent)"""
        return _lib.lts_batch_probe_barrier(self.h, int(absent_cta), float(limit_s))

    def stats(self):
        n = C.c_int64()
        g = [C.c_int(), C.c_int(), C.c_int()]
        _check(_lib.lts_batch_stats(self.h, C.byref(n), *[C.byref(x) for x in g]), "lts_batch_stats")
        return dict(launches=n.value, grid_stage=g[0].value, grid_prolong=g[1].value, grid_sync=g[2].value)

    def autotune(self, rounds=4, candidates=None):
        """Choose the launch shape of the rounds by timing `rounds` rounds for each
        candidate: the persistent round kernel with 1 .. (resident) CTAs per SM, and the
        per-stage launches with grid sizes in multiples of the SMs (advances the plans:
        re-set their state afterwards).  Returns the best shape and every timing."""
        import time
        live = [p for p in self.plans if p is not None]
        torch = live[0].torch
        sms = torch.cuda.get_device_properties(live[0].device).multi_processor_count
        if candidates is None:
            candidates = [("persistent", k) for k in (1, 2, 3, 4)]
            candidates += [("per-stage", (sms * a, sms * b, sms * 8)) for a in (2, 4, 6) for b in (4, 6)]
        best, table = None, []
        for mode, shape in candidates:
            try:
                if mode == "persistent":
                    self.set_mode(True, shape)
                else:
                    self.set_mode(False)
                    self.set_grid(*shape)
            except LtsError:
                continue            # more CTAs per SM than the kernel keeps resident
            steps = [rounds if p is not None else 0 for p in self.plans]
            self.run(steps, graph=True)    # capture + warm
            self.wait()
            t0 = time.perf_counter()
            self.run(steps, graph=True)
            self.wait()
            dt = time.perf_counter() - t0
            table.append((mode, shape, dt))
            if best is None or dt < best[2]:
                best = (mode, shape, dt)
        mode, shape, dt = best
        if mode == "persistent":
            self.set_mode(True, shape)
        else:
            self.set_mode(False)
            self.set_grid(*shape)
        return dict(mode=mode, shape=shape, seconds=dt, table=table)
