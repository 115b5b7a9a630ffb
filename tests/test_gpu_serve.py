"""Continuous batching: requests that arrive while others run are admitted into
free slots and advanced together; each request's result is the same as when it is
solved alone (relative L-infinity <= 1e-13) and, for the small trees, the same as the
CPU oracle's solve to the same time (1e-12), under both scheduling policies
(first come first served, shortest remaining work first with paused solves); the
server respects its slot count and device-memory budget."""
import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_10570_gb300 import build, ltsoct, serve
    build.build()
    ltsoct.load()
    return serve


def small_requests():
    # mixed sizes and end times; advection and wave; arrivals staggered in time
    ws = [W.advection_gauss(l_min=2, l_max=4), W.wave_planar(l_min=2, l_max=4),
          W.wave_shell(l_min=3, l_max=5, half=4.0, radius=1.5, width=0.2), W.advection_gauss(l_min=2, l_max=3),
          W.wave_shell(l_min=2, l_max=4, half=4.0, radius=1.5, width=0.2)]
    t_ends = [0.06, 0.05, 0.3, 0.09, 0.4]
    return ws, t_ends


@pytest.mark.parametrize("policy", ["fcfs", "srpt"])
def test_results_same_alone_and_in_the_mix(srv, policy):
    ws, t_ends = small_requests()
    reqs = [srv.Request(i, 0.002 * i, dict(spec=w["spec"], prob=w["prob"]), t) for i, (w, t) in
            enumerate(zip(ws, t_ends))]
    server = srv.Server(slots=3, chunk=4, policy=policy)   # fewer slots than requests: some must wait
    mixed, wall = server.serve(reqs, realtime=True)
    alone, _ = srv.serve_one_at_a_time(reqs, realtime=False)
    assert [r.rid for r in mixed] == [r.rid for r in alone] == list(range(len(reqs)))
    for a, b in zip(alone, mixed):
        assert a.substeps == b.substeps
        err = np.abs(a.state - b.state).max() / np.abs(a.state).max()
        assert err <= 1e-13, (a.rid, err)
    # requests 3 and 4 could only start after a slot was freed
    assert max(r.admitted for r in mixed) > min(r.finished for r in mixed) - 1e-9
    s = srv.summary(mixed, wall)
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_budget_limits_resident_solves(srv):
    ws, t_ends = small_requests()
    reqs = [srv.Request(i, 0.0, dict(spec=w["spec"], prob=w["prob"]), t) for i, (w, t) in
            enumerate(zip(ws[:3], t_ends[:3]))]
    from paper_2011_10570_gb300 import ltsoct
    sizes = [srv.state_bytes(len(ltsoct.Octree(r.work["spec"])), 2 if r.work["prob"]["pde"] == 1 else 1, 0)
             for r in reqs]
    # room for the largest request alone: whenever a request is admitted, the solves
    # resident at that moment and it fit the budget together
    budget = max(sizes)
    server = srv.Server(slots=4, chunk=4, hbm_budget=budget)
    res, _ = server.serve(reqs, realtime=False)
    size = {r.rid: sz for r, sz in zip(reqs, sizes)}
    for r in res:
        resident = [q for q in res if q.rid != r.rid and q.admitted <= r.admitted < q.finished]
        assert sum(size[q.rid] for q in resident) + size[r.rid] <= budget or not resident
    assert len(res) == 3


def test_saturated_gpu_serves_first_come_first_served(srv):
    """With a saturation threshold below any one solve's load, a request is admitted
    only when the GPU is free: the server degenerates to one solve at a time, and the
    results are still those of solving each request alone."""
    ws, t_ends = small_requests()
    reqs = [srv.Request(i, 0.0, dict(spec=w["spec"], prob=w["prob"]), t) for i, (w, t) in
            enumerate(zip(ws[:3], t_ends[:3]))]
    server = srv.Server(slots=4, chunk=4, saturation=1.0)
    res, _ = server.serve(reqs, realtime=False)
    spans = sorted((r.admitted, r.finished) for r in res)
    for (a0, f0), (a1, f1) in zip(spans[:-1], spans[1:]):
        assert a1 >= f0 - 1e-9
    alone, _ = srv.serve_one_at_a_time(reqs, realtime=False)
    for a, b in zip(alone, res):
        assert np.array_equal(a.state, b.state)


@pytest.mark.parametrize("policy", ["fcfs", "srpt"])
def test_served_results_match_the_oracle(srv, orc, policy):
    """Every served solve on a small tree (levels up to 4) equals the CPU oracle's LTS
    solve over the same substeps, and the reached time is that of the oracle."""
    ws, t_ends = small_requests()
    reqs = [srv.Request(i, 0.0, dict(spec=w["spec"], prob=w["prob"]), t) for i, (w, t) in
            enumerate(zip(ws, t_ends))]
    server = srv.Server(slots=3, chunk=4, policy=policy, saturation=1500.0)
    served, _ = server.serve(reqs, realtime=False)
    checked = 0
    for r, w in zip(served, ws):
        assert r.t_requested == t_ends[r.rid]
        if w["spec"]["l_max"] > 4:
            continue
        ot = orc.Tree.build(w["spec"])
        sol = orc.Solver(ot, w["spec"], w["prob"])
        sol.set_initial(0.0)
        sol.lts_substeps(r.substeps)
        ref = sol.state()
        err = np.abs(r.state - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (r.rid, err)
        assert r.t_reached == pytest.approx(sol.time, rel=1e-13)
        checked += 1
    assert checked == 4
