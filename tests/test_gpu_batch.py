"""Batching (many independent solves advanced together; a round is one persistent
cooperative launch, or a launch per stage; rounds captured in a CUDA graph): every
instance ends exactly where it ends when run alone, for instances of different PDEs,
RK schemes, level ranges and substep counts (whole and partial macro steps), in both
modes and every autotuned shape; the grid barrier of the persistent round gives up
after its time limit and reports LTS_ETIMEOUT (a CTA that never arrives)."""
import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_10570_gb300 import build, ltsoct
    build.build()
    ltsoct.load()
    return ltsoct


def instances():
    return [W.advection_gauss(l_min=2, l_max=4), W.advection_gauss(l_min=2, l_max=3, rk=3),
            W.wave_planar(l_min=2, l_max=4), W.wave_shell(l_min=3, l_max=5, half=4.0, radius=1.5, width=0.2),
            W.advection_gauss(l_min=1, l_max=6, radius=1e-3),
            W.wave_nonlinear(l_min=2, l_max=4, half=4.0, radius=1.5, width=0.2),
            W.wave_orbit(l_min=2, l_max=4, band=0.2, half=2.0, omega=3.0, precision=0)]


@pytest.mark.parametrize("graph,mode", [(True, ("persistent", 2)), (False, ("persistent", 1)),
                                        (True, ("per-stage", None)), (False, ("per-stage", None))])
def test_batch_equals_instances_alone(lt, graph, mode):
    ws = instances()
    substeps = [9, 7, 16, 5, 40, 6, 11]
    alone, batched = [], []
    for w in ws:
        a = lt.Plan(lt.Octree(w["spec"]), w["prob"])
        b = lt.Plan(lt.Octree(w["spec"]), w["prob"])
        a.set_initial(0.0)
        b.set_initial(0.0)
        alone.append(a)
        batched.append(b)
    for p, n in zip(alone, substeps):
        p.run_substeps(n)
    batch = lt.Batch(batched)
    if mode[0] == "persistent":
        batch.set_mode(True, mode[1])
    else:
        batch.set_mode(False)
    batch.run(substeps[:2] + [0] * (len(ws) - 2), graph=graph)     # a first call, some plans idle
    batch.run([0, 0] + substeps[2:], graph=graph)
    batch.wait()
    if mode[0] == "persistent":
        assert batch.stats()["launches"] == max(substeps[:2]) + max(substeps[2:])   # one launch per round
    for a, b, n in zip(alone, batched, substeps):
        assert a.stats()["time"] == b.stats()["time"]
        assert a.stats()["substep"] == b.stats()["substep"]
        ua, ub = a.get_state(), b.get_state()
        err = np.abs(ua - ub).max() / np.abs(ua).max()
        assert err <= 1e-13, err
    # the plans continue normally after the batch
    for a, b in zip(alone, batched):
        a.run_substeps(3)
        b.run_substeps(3)
        assert np.abs(a.get_state() - b.get_state()).max() <= 1e-13 * np.abs(a.get_state()).max()


def test_batch_matches_oracle(lt, orc):
    ws = instances()[:3]
    plans = [lt.Plan(lt.Octree(w["spec"]), w["prob"]) for w in ws]
    for p in plans:
        p.set_initial(0.0)
    batch = lt.Batch(plans)
    tune = batch.autotune(rounds=2)
    assert tune["mode"] in ("persistent", "per-stage") and len(tune["table"]) >= 2
    refs = []
    for w in ws:
        sol = orc.Solver(orc.Tree.build(w["spec"]), w["spec"], w["prob"])
        sol.set_initial(0.0)
        sol.lts_substeps(8)
        refs.append(sol.state())
    # the tuned shape, then every shape the autotuner timed
    for mode, shape, _ in [(tune["mode"], tune["shape"], 0.0)] + tune["table"]:
        if mode == "persistent":
            batch.set_mode(True, shape)
        else:
            batch.set_mode(False)
            batch.set_grid(*shape)
        for p in plans:
            p.set_initial(0.0)
        batch.run([8, 8, 8])
        batch.wait()
        for p, ref in zip(plans, refs):
            assert np.abs(p.get_state() - ref).max() / np.abs(ref).max() <= 1e-12, (mode, shape)


def test_grid_barrier_time_limit(lt):
    """The persistent round's grid barrier gives up after its limit: with one CTA that
    never arrives, every other CTA's wait runs out and LTS_ETIMEOUT comes back; the
    batch is usable afterwards."""
    w = W.advection_gauss(l_min=2, l_max=3)
    plan = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    plan.set_initial(0.0)
    batch = lt.Batch([plan])
    assert batch.probe_barrier(-1, 0.5) == 0                 # all arrive
    assert batch.probe_barrier(3, 0.05) == lt.LTS_ETIMEOUT   # CTA 3 never arrives
    batch.wait()                                             # the error word was cleared
    ref = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    ref.set_initial(0.0)
    ref.run_substeps(4)
    batch.run([4])
    batch.wait()
    assert np.array_equal(plan.get_state(), ref.get_state())


def test_batch_rejects_mixed_streams_or_precision(lt):
    w = W.advection_gauss(l_min=2, l_max=3)
    a = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    b = lt.Plan(lt.Octree(w["spec"]), dict(w["prob"], precision=1))
    with pytest.raises(lt.LtsError):
        lt.Batch([a, b])


@pytest.mark.parametrize("mode", [("persistent", 3), ("per-stage", None)])
def test_mixed_precision_batch_equals_instances_alone(lt, mode):
    """Mixed-precision plans (FP32 stages, FP64 state) batched in either mode end where
    they end alone."""
    ws = [W.advection_gauss(l_min=2, l_max=4), W.wave_planar(l_min=2, l_max=4),
          W.wave_shell(l_min=3, l_max=5, half=4.0, radius=1.5, width=0.2)]
    for w in ws:
        w["prob"]["precision"] = 1
    substeps = [8, 12, 4]
    alone, batched = [], []
    for w, n in zip(ws, substeps):
        a = lt.Plan(lt.Octree(w["spec"]), w["prob"])
        b = lt.Plan(lt.Octree(w["spec"]), w["prob"])
        a.set_initial(0.0)
        b.set_initial(0.0)
        a.run_substeps(n)
        alone.append(a)
        batched.append(b)
    batch = lt.Batch(batched)
    if mode[0] == "persistent":
        batch.set_mode(True, mode[1])
    batch.run(substeps)
    batch.wait()
    for a, b in zip(alone, batched):
        ua, ub = a.get_state(), b.get_state()
        assert np.abs(ua - ub).max() <= 1e-12 * np.abs(ua).max()
