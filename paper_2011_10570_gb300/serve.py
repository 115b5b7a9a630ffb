"""Continuous batching of LTS solves on one GPU.

Requests (an octree refinement spec, a problem and an end time) arrive over time.
The server keeps every admitted solve resident on the device (octree tables, RK
state) in a slot of a batch (``lts_batch_create_slots``), and advances all of them
together in rounds: each round performs one LTS substep (Alg. 2, Fig. blk_loop)
of every resident solve, with one persistent launch per RK stage covering the
active levels of all of them.  Between chunks of rounds the server
  * retires solves that reached their end time (result copied to the host,
    device memory returned, slot freed), and
  * admits waiting requests, first come first served, while a slot is free, the
    device-memory budget holds their estimated footprint, and the GPU is not yet
    saturated: the resident solves' mean active octants per substep (eq. w_nuts
    over the 2^(l_max - l_min) substeps of a macro step) stay within `saturation`.
    Batching adds throughput only while one substep of the resident solves does
    not fill the GPU; past that point sharing it would only stretch every
    request's latency, so further requests wait.
A single resident solve runs on its own plan's kernels (no batch indirection).
Latency is arrival to result; throughput is node-updates per second of wall time.

Two policies choose the order of admission and the solves each chunk advances:
  * ``fcfs``: requests are admitted in arrival order, and every resident solve
    advances in every chunk (saturation bounds the admissions, as above);
  * ``srpt``: shortest remaining work first.  Waiting requests are admitted in order
    of their work (node-updates to their end time, eq. w_nuts per macro step), and
    each chunk advances the resident solves with the least remaining work while
    their summed load stays within `saturation` (at least one).  The others stay
    resident and paused: their state does not move until they are scheduled again.
    Small solves that arrive behind a large one no longer wait for it to finish,
    at the same total work.

``serve_one_at_a_time`` solves the same stream first-come-first-served, one
request at a time, for comparison.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import ltsoct


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    work: dict              # {"spec": ..., "prob": ...}
    t_end: float


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    octants: int
    substeps: int
    node_updates: float
    state: np.ndarray = field(repr=False, default=None)
    t_requested: float = 0.0   # the request's end time
    t_reached: float = 0.0     # the time the solve reached (whole macro steps, see substeps_to)

    @property
    def latency(self):
        return self.finished - self.arrival


def state_bytes(n_octants, nf, precision, p=4):
    """Device bytes of a plan: state (2 copies, FP64), RK stages and 2 stage-input
    buffers in the stage type, prolonged inputs (at most one slot per octant), the
    padding map (4 bytes per padded point) and tables."""
    es = 4 if precision == 1 else 8
    per_octant = 343 * nf * (2 * 8 + (p + 2) * es) + 2197 * nf * es + 2197 * 4 + 27 * 4 + 64
    return int(n_octants * per_octant)


def substeps_to(plan, t_end):
    """whole macro steps from the plan's current time up to the macro-step boundary
    nearest t_end (at least one): the solve ends at that boundary, which Result
    records as t_reached next to the requested t_end"""
    st = plan.stats()
    n_macro = max(1, int(round((t_end - st["time"]) / st["dt_coarsest"])))
    return n_macro * (1 << (st["l_max"] - st["l_min"]))


def estimated_work(spec, prob, levels, t_end):
    """node-updates of a request before its plan exists: macro steps of the coarsest step
    dt_c = cfl * h_(l_min) (h the node spacing) to t_end, times the LTS work of one macro
    step, sum_l n_l 2^(l - l_min) octant-steps of 343 nodes (eq. w_nuts)"""
    levels = np.asarray(levels)
    lmin = int(levels.min())
    dt_c = prob["cfl"] * (spec["hi"] - spec["lo"]) / (6.0 * 2.0 ** lmin)
    n_macro = max(1, int(round(t_end / dt_c)))
    return float(n_macro * 343 * np.sum(np.ldexp(1.0, levels.astype(np.int64) - lmin)))


def mean_active_octants(levels):
    """octants stepping in an average substep: sum_l n_l 2^(l - l_max) (eq. w_nuts / 2^L)"""
    levels = np.asarray(levels)
    lmax = int(levels.max())
    return float(np.sum(np.ldexp(1.0, levels.astype(np.int64) - lmax)))


def node_updates(st, n_sub0, n):
    lmin, lmax = st["l_min"], st["l_max"]
    counts = st["octants_per_level"]
    total, k = 0, n_sub0
    for _ in range(n):
        lstar = next(l for l in range(lmin, lmax + 1) if k % (1 << (lmax - l)) == 0)
        total += 343 * sum(counts[lstar:lmax + 1])
        k = (k + 1) % (1 << (lmax - lmin))
    return float(total)


class Server:
    def __init__(self, slots=16, hbm_budget=64 << 30, chunk=8, precision=0, keep_results=True,
                 saturation=8192.0, policy="fcfs"):
        import torch
        if policy not in ("fcfs", "srpt"):
            raise ValueError("policy must be 'fcfs' or 'srpt'")
        self.policy = policy
        self.torch = torch
        self.stream = torch.cuda.current_stream()
        self.batch = ltsoct.Batch.slots(slots, self.stream, precision)
        self.nslots = slots
        self.budget = hbm_budget
        self.chunk = chunk
        self.precision = precision
        self.keep = keep_results
        self.saturation = saturation

    def serve(self, requests, realtime=True):
        """Serve `requests` (sorted by arrival).  With realtime, arrivals are honoured
        against the wall clock; otherwise every request is available at once."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        active = {}                      # slot -> [req, plan, remaining, admitted, est, updates, load]
        used = 0
        load = 0.0                       # mean active octants per substep of the resident solves
        results = []
        trees = {}                       # rid -> (octree, device bytes, load), built once per request
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        # wall time of the server's phases (seconds), for the bench report
        self.phases = collections.Counter()
        clock = [time.perf_counter()]

        def mark(phase):
            t = time.perf_counter()
            self.phases[phase] += t - clock[0]
            clock[0] = t

        def prepare(req):
            if req.rid not in trees:
                tree = ltsoct.Octree(req.work["spec"])
                nf = 2 if req.work["prob"]["pde"] == 1 else 1
                levels = tree.export()[1]
                trees[req.rid] = (tree, state_bytes(len(tree), nf, self.precision), mean_active_octants(levels),
                                  estimated_work(req.work["spec"], req.work["prob"], levels, req.t_end))
            return trees[req.rid]

        srpt = self.policy == "srpt"
        while pending or active:
            mark("idle_or_host")
            # admit while a slot is free and the budget holds
            while pending and (not realtime or pending[0].arrival <= now()) and len(active) < self.nslots:
                if srpt:
                    # the arrived request with the least work
                    arrived = [r for r in pending if not realtime or r.arrival <= now()]
                    req = min(arrived, key=lambda r: (prepare(r)[3], r.arrival))
                else:
                    req = pending[0]
                tree, est, ld, _ = prepare(req)
                if active and (used + est > self.budget or (not srpt and load + ld > self.saturation)):
                    break                # wait for memory to be freed or the GPU to have room
                pending.remove(req)
                del trees[req.rid]
                prob = dict(req.work["prob"], precision=self.precision)
                plan = ltsoct.Plan(tree, prob, stream=self.stream)
                plan.set_initial(0.0)
                n = substeps_to(plan, req.t_end)
                slot = next(s for s in range(self.nslots) if s not in active)
                self.batch.attach(slot, plan)
                active[slot] = [req, plan, n, now(), est, node_updates(plan.stats(), 0, n), ld, n]
                used += est
                load += ld
                mark("admit")
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now())))
                continue
            steps = [0] * self.nslots
            if srpt:
                # the resident solves with the least remaining work, within the saturation load
                order = sorted(active, key=lambda s: (active[s][5] * active[s][2] / active[s][7], active[s][0].arrival))
                run, ld_run = [], 0.0
                for s in order:
                    if run and ld_run + active[s][6] > self.saturation:
                        break
                    run.append(s)
                    ld_run += active[s][6]
                k = min(self.chunk, min(active[s][2] for s in run))
            else:
                run = list(active)
                k = min(self.chunk, min(a[2] for a in active.values()))
                if len(active) == 1 and load >= self.saturation:
                    # nothing can join a solve that fills the GPU: run it to its end in one go
                    k = next(iter(active.values()))[2]
            for s in run:
                steps[s] = min(k, active[s][2])
            if len(run) == 1:
                a0 = active[run[0]]
                a0[1].run_substeps(steps[run[0]])
            else:
                self.batch.run(steps, graph=True)
            mark("launch")
            # host work while the GPU runs the chunk: octrees of requests that have arrived
            for req in list(pending)[:self.nslots]:
                if realtime and req.arrival > now():
                    break
                prepare(req)
            mark("prepare")
            torch.cuda.current_stream().synchronize()
            mark("gpu_wait")
            for s in list(active):
                a = active[s]
                a[2] -= steps[s]
                if a[2] == 0:
                    req, plan = a[0], a[1]
                    state = plan.get_state() if self.keep else None
                    t = now()
                    st = plan.stats()
                    results.append(Result(req.rid, req.arrival, a[3], t, st["n_octants"],
                                          int(round(st["time"] / st["dt_finest"])), a[5], state,
                                          t_requested=req.t_end, t_reached=st["time"]))
                    self.batch.detach(s)
                    used -= a[4]
                    load -= a[6]
                    del active[s]
                    del plan
        return sorted(results, key=lambda r: r.rid), now()


def serve_one_at_a_time(requests, precision=0, realtime=True, keep_results=True):
    """First come, first served, one solve on the GPU at a time (no batching)."""
    import torch
    stream = torch.cuda.current_stream()
    results = []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime and req.arrival > now():
            time.sleep(req.arrival - now())
        admitted = now()
        plan = ltsoct.Plan(ltsoct.Octree(req.work["spec"]), dict(req.work["prob"], precision=precision),
                           stream=stream)
        plan.set_initial(0.0)
        n = substeps_to(plan, req.t_end)
        plan.run_substeps(n)
        stream.synchronize()             # a request is finished when its solve has run
        state = plan.get_state() if keep_results else None
        st = plan.stats()
        results.append(Result(req.rid, req.arrival, admitted, now(), st["n_octants"], n,
                              node_updates(st, 0, n), state, t_requested=req.t_end, t_reached=st["time"]))
        del plan
    return results, now()


def summary(results, wall):
    lat = np.array([r.latency for r in results])
    work = sum(r.node_updates for r in results)
    return {"requests": len(results), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
            "throughput_node_updates_per_s": work / wall, "requests_per_s": len(results) / wall,
            "wall_s": wall}
