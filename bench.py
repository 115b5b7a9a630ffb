"""Benchmark: LTS octant-node updates/s on one GB300 (wave equation, levels 4..9).

A step is one LTS macro step (Alg. 2): 2^(l_max - l_min) = 32 substeps of the
finest timestep, each running the RK stages of the active levels (Fig. blk_loop),
followed by the shared-node reconcile.  The metric counts one node of one
octant advanced one full RK step on its own level (eq. w_nuts times 343 nodes).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle on a bounded sample of the same workload
(the paper has no GPU implementation; the oracle is the reference arm).  Under
torchrun (N > 1) every rank runs an independent replica (the solve is not sharded
across GPUs) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LTS octant-node updates/s"
UNIT = "node-updates/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk/SM x flops/FMA x max clock
# DRAM bytes (read + write) per node-stage of stage_kernel<2, double> / <2, float>, from ncu
# captures of one stage launch on the levels 4..8 wave case; None whenever the kernel changes
STAGE_DRAM_BYTES_PER_NODE_STAGE = 88.3
STAGE_DRAM_BYTES_PER_NODE_STAGE_MIXED = 48.3
# FP64-pipe operations per node-stage of stage_kernel<2, double> on the wave equation:
# phi's dissipation 18 (15 pair-sum additions, 3 FMAs), the Laplacian's scaling and the
# two stage FMAs 3, two integer-to-FP64 conversions 2, the RK epilogue 3.5 on average;
# chi's 19 stencil inputs are summed exactly on the integer pipes
FP64_PIPE_OPS_PER_NODE_STAGE = 26.5


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        # replicas only: the collectives are a timing barrier and a max over ranks
        # of one float, on the host (gloo), for both arms
        import torch.distributed as dist
        dist.init_process_group(backend="gloo")
        pg = dist
    return world, rank, local, pg


class OracleSample:
    """The CPU oracle on a bounded sample of the workload: one LTS substep in which
    every level is active (substep 0), each octant advanced one full RK step on its
    own level.  The tree and the oracle's padding maps are built once (first call
    untimed); every timed call restarts from the initial data."""

    def __init__(self, w, threads=None):
        import oracle
        if threads:
            oracle.set_threads(threads)
        self.tree = oracle.Tree.build(w["spec"])
        self.sol = oracle.Solver(self.tree, w["spec"], w["prob"])
        self.n = len(self.tree)
        self.sol.set_initial(0.0)
        self.sol.lts_substeps(1)          # builds the padding maps

    def run(self):
        self.sol.set_initial(0.0)
        t0 = time.perf_counter()
        self.sol.lts_substeps(1)
        dt = time.perf_counter() - t0
        return self.n * 343 / dt, dt


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, w, world, rank, pg):
    if rank != 0:
        return
    threads = args.oracle_threads or host_threads()
    sample = OracleSample(w, threads)
    n = sample.n
    vals, times = [], []
    for _ in range(args.warmup):
        sample.run()
    for _ in range(args.steps):
        v, dt = sample.run()
        vals.append(v)
        times.append(dt)
    value = len(vals) / sum(1.0 / v for v in vals)
    sample = ("one LTS substep with every level active (substep 0: %d octants x 343 nodes, one RK4 step each) "
              "of the wave workload, per step" % n)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "octants": n, "levels": "%d..%d" % (w["spec"]["l_min"], w["spec"]["l_max"]),
                   "fields": 2, "rk": 4,
                   "parallelism": "replicas",
                   "l2": "state arrays (%d MB each) larger than L2" % round(2 * n * 343 * 8 / 1e6)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def schedule_work(st, n_sub0, rounds):
    """node-updates of `rounds` substeps of one plan starting at substep n_sub0 (Fig. blk_loop)"""
    lmin, lmax = st["l_min"], st["l_max"]
    counts = st["octants_per_level"]
    nsub = 2 ** (lmax - lmin)
    total, n = 0, n_sub0
    for _ in range(rounds):
        lstar = next(l for l in range(lmin, lmax + 1) if n % (2 ** (lmax - l)) == 0)
        total += 343 * sum(counts[lstar:lmax + 1])
        n = (n + 1) % nsub
    return total


def run_batch(args):
    """Batched instances (NEXT-2): one persistent launch per stage covers all instances;
    rounds replayed from a captured CUDA graph; grid shapes autotuned."""
    import numpy as np
    import torch

    from paper_2011_10570_gb300 import build, ltsoct, workloads
    build.build()
    torch.cuda.set_device(0)
    ws = workloads.batch_instances(seed=3, n=args.batch, f_range=(1.0, args.batch_fmax))
    stream = torch.cuda.current_stream()
    plans = [ltsoct.Plan(ltsoct.Octree(w["spec"]), w["prob"], stream=stream) for w in ws]
    sts = [p.stats() for p in plans]
    for p in plans:
        p.set_initial(0.0)
    batch = ltsoct.Batch(plans)
    tune = batch.autotune(rounds=4)
    batch.wait()
    rounds = args.rounds
    for p in plans:
        p.set_initial(0.0)
    batch.run([args.warmup] * len(plans))
    torch.cuda.synchronize()
    n0 = [p.stats()["substep"] for p in plans]
    work = sum(schedule_work(st, n, rounds) for st, n in zip(sts, n0))
    l0 = batch.stats()["launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        batch.run([rounds] * len(plans), graph=True)
        ev1.record(stream)
        torch.cuda.synchronize()
    batch.wait()
    ms = ev0.elapsed_time(ev1)
    launches = batch.stats()["launches"] - l0
    # the same work one instance at a time (per-plan launches, no batching)
    for p in plans:
        p.set_initial(0.0)
        p.run_substeps(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for p in plans:
        p.run_substeps(rounds)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_alone = e0.elapsed_time(e1)
    n_oct = [st["n_octants"] for st in sts]
    line = {
        "metric": "batched LTS octant-node updates/s", "value": work / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": rounds, "warmup": args.warmup, "ms_per_step": ms / rounds, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batch of %d instances (seed 3, f <= %g)" % (len(plans), args.batch_fmax),
                   "octants_min": min(n_oct),
                   "octants_median": int(np.median(n_oct)), "octants_max": max(n_oct),
                   "levels": "3..6-11", "step": "one round: one substep of every instance"},
        "gpu_launches": launches, "graph": True,
        "autotuned": {"mode": tune["mode"], "shape": tune["shape"],
                      "candidates_s": [[m, sh, round(t, 5)] for m, sh, t in tune["table"]]},
        "one_at_a_time": {"value": work / (ms_alone / 1e3), "ms_per_step": ms_alone / rounds},
        "batch_speedup": ms_alone / ms, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def serve_sample(args, n=32, rate=32.0):
    """A short served stream beside the main line (NEXT-3): n small shell solves (levels
    3..4, 736 to 3,536 octants, end times 0.5..5) arriving as a Poisson stream, served by
    continuous batching (shortest remaining work first) and by one solve at a time,
    first come first served; latency is arrival to the end of the solve on the GPU."""
    from paper_2011_10570_gb300 import serve, workloads
    raw = workloads.serving_requests(seed=4, n=n, rate=rate, lmax_choices=(4,))
    reqs = [serve.Request(r["rid"], r["arrival"], r["work"], r["t_end"]) for r in raw]
    out = {"requests": n, "rate_per_s": rate, "workload": "shell solves, levels 3..4 (seed 4)"}
    server = serve.Server(slots=16, chunk=8, keep_results=False, policy="srpt")
    res_b, wall_b = server.serve(reqs, realtime=True)
    out["continuous_batching_srpt"] = serve.summary(res_b, wall_b)
    res_1, wall_1 = serve.serve_one_at_a_time(reqs, realtime=True, keep_results=False)
    out["one_at_a_time_fcfs"] = serve.summary(res_1, wall_1)
    return out


def run_serve(args):
    """Serving (NEXT-3): a Poisson stream of wave solves, continuous batching against
    first-come-first-served one-at-a-time solving, per arrival rate."""
    import torch

    from paper_2011_10570_gb300 import build, serve, workloads
    build.build()
    torch.cuda.set_device(0)
    out = {"metric": "served LTS solves: p50/p99 latency and throughput", "n_gpus": 1, "dtype": "f64",
           "data": "synthetic", "rates": []}
    for rate in args.serve_rates:
        raw = workloads.serving_requests(seed=4, n=args.serve_n, rate=rate, lmax_choices=tuple(args.serve_lmax))
        reqs = [serve.Request(r["rid"], r["arrival"], r["work"], r["t_end"]) for r in raw]
        row = {"rate_per_s": rate}
        for policy in args.serve_policy:
            for sat in args.serve_saturation:
                server = serve.Server(slots=args.serve_slots, chunk=args.serve_chunk, keep_results=False,
                                      saturation=sat, policy=policy)
                res_b, wall_b = server.serve(reqs, realtime=True)
                row["continuous_batching_%s_sat%g" % (policy, sat)] = dict(
                    serve.summary(res_b, wall_b), phases_s={k: round(v, 4) for k, v in server.phases.items()})
                del server
        res_1, wall_1 = serve.serve_one_at_a_time(reqs, realtime=True, keep_results=False)
        octs = sorted(r.octants for r in res_1)
        row["one_at_a_time"] = serve.summary(res_1, wall_1)
        row["octants_min_median_max"] = [octs[0], octs[len(octs) // 2], octs[-1]]
        out["rates"].append(row)
        print(json.dumps(out["rates"][-1]), flush=True)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lts", choices=["lts", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="host threads of the oracle in the reference arm (default: all cores)")
    ap.add_argument("--no-gts", action="store_true",
                    help="skip the GTS comparison (GTS over the same physical time, and the LTS-GTS difference)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the short served stream beside the main line")
    ap.add_argument("--batch", type=int, default=0, help="batched mode: number of instances (64 for the C4 workload)")
    ap.add_argument("--rounds", type=int, default=64, help="batched mode: timed rounds")
    ap.add_argument("--batch-fmax", type=float, default=20.0,
                    help="batched mode: refinement radius range in finest-octant edges (20: 1k-50k octants)")
    ap.add_argument("--serve", action="store_true", help="serving mode: Poisson stream, continuous batching")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 2.0])
    ap.add_argument("--serve-n", type=int, default=16)
    ap.add_argument("--serve-lmax", type=int, nargs="+", default=[5, 6],
                    help="finest levels the request trees draw from (5 6: about 4k to 180k octants)")
    ap.add_argument("--serve-saturation", type=float, nargs="+", default=[8192.0],
                    help="admission limit on the resident solves' mean active octants per substep")
    ap.add_argument("--serve-policy", nargs="+", default=["fcfs", "srpt"], choices=["fcfs", "srpt"],
                    help="admission / scheduling policies of the continuous-batching server")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-chunk", type=int, default=8)
    ap.add_argument("--workload", default="shell", choices=["shell", "nonlinear", "orbit"],
                    help="shell: linear wave, levels 4..9 (the benchmark configuration); nonlinear: the same "
                         "with the -sin(2 chi)/r^2 source; orbit: two orbiting sources, levels 3..12")
    ap.add_argument("--orbit-lmax", type=int, default=12,
                    help="finest level of the orbit workload (12: the configuration; smaller for profiling)")
    ap.add_argument("--substeps", type=int, default=0,
                    help="substeps per step (default: a macro step; 64 for the orbit workload)")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="mixed: FP32 stages and right-hand side, FP64 state and time corrections")
    ap.add_argument("--lmax", type=int, default=9,
                    help="finest level of the wave workload (9: the benchmark configuration; 8: the profiling case)")
    args = ap.parse_args()

    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    from paper_2011_10570_gb300 import workloads
    if args.workload == "orbit":
        w = workloads.wave_orbit(l_max=args.orbit_lmax)
    elif args.workload == "nonlinear":
        w = workloads.wave_nonlinear(l_max=args.lmax)
    else:
        w = workloads.wave_shell(l_max=args.lmax)
    if args.precision is None:
        args.precision = "mixed" if args.workload == "orbit" else "fp64"
    w["prob"]["precision"] = 1 if args.precision == "mixed" else 0
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, w, world, rank, pg)
        if pg:
            pg.barrier()
            pg.destroy_process_group()
        return

    import numpy as np
    import torch

    from paper_2011_10570_gb300 import build, ltsoct
    build.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ltsoct.Octree(workloads.advection_gauss(l_min=2, l_max=3)["spec"])   # the build's kernels loaded
    torch.cuda.synchronize()
    t_tree = time.perf_counter()
    tree = ltsoct.Octree(w["spec"])            # refinement, 2:1 balance and o2o on the device
    t_plan = time.perf_counter()
    plan = ltsoct.Plan(tree, w["prob"], stream=stream)
    torch.cuda.synchronize()
    t_ready = time.perf_counter()
    st = plan.stats()
    n = st["n_octants"]
    L = st["l_max"] - st["l_min"]
    # a step: one macro step (2^L substeps), or a window of k substeps of it when a
    # macro step is too long to time several of (the orbit workload: 512 substeps)
    nsub = args.substeps if args.substeps else (64 if args.workload == "orbit" else 2 ** L)
    plan.set_initial(0.0)
    for _ in range(args.warmup):
        plan.run_substeps(nsub)
    torch.cuda.synchronize()
    n_sub0 = plan.stats()["substep"]
    work_timed = schedule_work(st, n_sub0, args.steps * nsub)   # node-updates of the timed substeps

    # device-resident timed region (CUDA events on the plan's stream)
    plan.set_profiling(True)
    plan.kernel_stats(reset=True)
    plan.prolong_stats(reset=True)
    launches0 = plan.stats()["kernel_launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            plan.run_substeps(nsub)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = plan.stats()["kernel_launches"] - launches0
    ks = plan.kernel_stats(reset=True)
    ps = plan.prolong_stats(reset=True)
    plan.set_profiling(False)
    if pg:
        t = torch.tensor([ms], dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = world * work_timed / (ms / 1e3)

    # end to end through the C ABI with host buffers: H2D of the state, one macro
    # step, D2H of the result, every step
    host_t = torch.empty((st["nf"], n, 343), dtype=torch.float64, pin_memory=True)
    out_t = torch.empty((st["nf"], n, 343), dtype=torch.float64, pin_memory=True)
    host, out = host_t.numpy(), out_t.numpy()
    plan.get_state(host)
    e2e_steps = 0 if args.no_e2e else max(1, args.steps)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.set_state(host, 0.0)
        plan.run_substeps(nsub)
        plan.get_state(out)
    torch.cuda.synchronize()
    e2e_s = max(time.perf_counter() - t0, 1e-30)
    if pg:
        t = torch.tensor([e2e_s], dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_s = float(t.item())
    # every e2e step restarts from a synchronised state: the first window of a macro step
    e2e_value = world * e2e_steps * schedule_work(st, 0, nsub) / e2e_s if e2e_steps else None
    state_bytes = host.nbytes

    # GTS (Alg. 1) over the same physical time: 2^L global steps of dt_f per macro step,
    # timed like the LTS steps; then the difference of the two solutions after one macro
    # step from the same initial data (LTS's interface error against GTS at equal dt_f)
    gts = None
    if not args.no_gts:
        plan.set_initial(0.0)
        plan.gts_steps(2)
        plan.set_initial(0.0)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        plan.gts_steps(nsub)
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1)
        # LTS: the timed steps; GTS: nsub global steps of dt_f (the same physical time
        # per step when a step is a macro step)
        gts = {"ms_per_step": gms, "lts_ms_per_step": ms / args.steps, "steps_of_dt_finest": nsub,
               "lts_speedup_measured": gms / (ms / args.steps), "lts_speedup_model": st["model_speedup"],
               "gts_node_updates_per_s": world * st["gts_work_per_macro"] * 343 * (nsub / 2 ** L) / (gms / 1e3)}
        if nsub == 2 ** L:
            u_g = plan.get_state(out)
            plan.set_initial(0.0)
            plan.run_substeps(nsub)
            u_l = plan.get_state(host)
            gts["lts_minus_gts_rel_linf"] = max(float(np.abs(u_l[f] - u_g[f]).max() / np.abs(u_g[f]).max())
                                                for f in range(st["nf"]))
            gts["lts_minus_gts_note"] = ("after one macro step from the same initial data, per field relative "
                                         "to the field's max, the larger of the two")
        else:
            gts["note"] = ("a step is %d of the %d substeps of a macro step: the LTS window also holds the "
                           "coarse levels' steps of substep 0 when it starts a macro step" % (nsub, 2 ** L))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32 stages / f64 state",
        "data": "synthetic",
        "config": {"workload": w["name"], "octants": n, "levels": "%d..%d" % (st["l_min"], st["l_max"]),
                   "fields": st["nf"], "rk": 4, "substeps_per_step": nsub, "substeps_per_macro_step": 2 ** L,
                   "parallelism": "replicas",
                   "l2": "inputs larger than L2 (state arrays %d MB each)" % round(st["nf"] * n * 343 * 8 / 1e6)},
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes},
        "clocks": clk.summary(),
        "lts_model_speedup": st["model_speedup"],
        "setup_s": {"octree_build": round(t_plan - t_tree, 4), "plan_create": round(t_ready - t_plan, 4),
                    "note": "octree_build: refinement, 2:1 balance, level order and o2o on the device, leaves "
                            "and o2o copied to the host; plan_create: tables, padding and node maps"},
    }
    if nsub == 2 ** L:
        # useful work at GTS's count (every octant at dt_f) per LTS wall second
        line["gts_equivalent_rate"] = world * args.steps * st["gts_work_per_macro"] * 343 / (ms / 1e3)
    if ks["launches"]:
        avg_ms = ks["ms"] / ks["launches"]
        flops_per_launch = ks["flops"] / ks["launches"]
        achieved = flops_per_launch / (avg_ms / 1e3) / 1e12
        per_ns = STAGE_DRAM_BYTES_PER_NODE_STAGE if args.precision == "fp64" else STAGE_DRAM_BYTES_PER_NODE_STAGE_MIXED
        traffic = per_ns * ks["node_stages"] / ks["launches"] if per_ns else None
        hbm_peak = measured_peaks().get("hbm_gbs")
        # DRAM bytes the kernel moves per launch (ncu's per-node-stage figure for this build)
        # over its live launch time: the HBM rate it reaches, beside the algorithmic one
        dram_gbs = traffic / (avg_ms / 1e3) / 1e9 if traffic else None
        if args.precision == "mixed":
            gbs = ks["bytes"] / (ks["ms"] / 1e3) / 1e9
            line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                "frac": gbs / hbm_peak if hbm_peak else None, "traffic": traffic,
                                "traffic_source": "ncu dram bytes per node-stage (levels 4..8 capture) x node-stages per launch",
                                "kernel": "stage_kernel<2, float>", "peak_source": "measured (MEASURED_PEAKS.json)",
                                "fp64_tflops_algorithmic": achieved, "stage_share_of_step": ks["ms"] / ms,
                                "dram_gbs_measured_bytes": dram_gbs,
                                "dram_frac_measured_bytes": dram_gbs / hbm_peak if dram_gbs and hbm_peak else None}
        else:
            fl = flops_per_launch / (ks["node_stages"] / ks["launches"])
            line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                              "flops_per_node_stage": fl,
                              "flops_note": "FP64-equivalent operations counted from the kernel's formulas, FMA = 2 "
                                            "(an estimate of 65 per node-stage gives frac %.3f); chi's stencil sums "
                                            "run as exact integer arithmetic on the integer pipes, so frac is the "
                                            "FP64-equivalent rate against the FP64 pipe's peak, and "
                                            "fp64_pipe_frac the pipe's own load" % (achieved * 65 / fl / FP64_PEAK_TFLOPS),
                              "frac_vs_fma_probe": achieved / 1.20,
                              "fma_probe_note": "1.20 TFLOP/s: an FP64 FMA loop measured on a GB300 of this pool",
                              "traffic_source": "ncu dram bytes per node-stage (levels 4..8 capture) x node-stages per launch",
                              "kernel": "stage_kernel<2>", "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz",
                              "hbm_gbs_algorithmic": ks["bytes"] / (ks["ms"] / 1e3) / 1e9,
                              "hbm_peak_gbs": hbm_peak,
                              "dram_gbs_measured_bytes": dram_gbs,
                              "fp64_ops_per_node_stage": FP64_PIPE_OPS_PER_NODE_STAGE,
                              "fp64_pipe_frac": FP64_PIPE_OPS_PER_NODE_STAGE * ks["node_stages"] / (ks["ms"] / 1e3) /
                                                (152 * 2 * 2.070e9),
                              "stage_share_of_step": ks["ms"] / ms}
    if ps["launches"] and "roofline" in line:
        # the second kernel of the step: the prolongation, FP64-equivalent flops as directly
        # evaluated over its live event-timed launches
        pro = {"launches": ps["launches"], "ms_per_launch": ps["ms"] / ps["launches"],
               "sources_per_launch": ps["sources"] / ps["launches"], "share_of_step": ps["ms"] / ms}
        if args.precision == "fp64":
            p_tf = ps["flops"] / (ps["ms"] / 1e3) / 1e12
            pro.update({"kernel": "prolong_kernel<2, double>", "bound": "alu", "achieved": p_tf, "unit": "TFLOP/s",
                        "peak": FP64_PEAK_TFLOPS, "frac": p_tf / FP64_PEAK_TFLOPS,
                        "note": "flops: the interpolation's multiply-adds of the plan's cost model (7 per odd "
                                "half-node position) and the time-corrected inputs, FMA = 2; the kernel evaluates "
                                "mirrored pairs with fewer FP64 operations, so frac is an FP64-equivalent rate"})
        else:
            pro.update({"kernel": "prolong_kernel<2, float>",
                        "note": "FP32 interpolation after FP64 time corrections: bound by instruction issue "
                                "(ncu), no single-pipe peak applies"})
        line["roofline"]["prolong"] = pro
    if gts:
        line["gts"] = gts
    if not args.no_serve and rank == 0:
        line["serving"] = serve_sample(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        del plan
        torch.cuda.empty_cache()
        samp = OracleSample(w, host_threads())
        v, dt = samp.run()
        nn = samp.n
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
                                "sample": "one LTS substep with every level active (%d octants, one RK4 step each), "
                                          "%.1f s" % (nn, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
