"""Mixed precision (RK stages, stage inputs, padded block and right-hand side in
FP32; state, RK update and the time corrections of eqs. fc_1 / fc_2 in FP64)
against the FP64 oracle.

The error is that of FP32 finite differences: tile values carry a relative
rounding of eps32 = 6e-8, so a second difference at spacing h has a relative
error of about eps32 * 8 (sigma/h)^2 for a pulse of width sigma, and a first
difference about eps32 * 2 sigma/h.  Bounds below are stated per workload from
that estimate over the steps taken, and each run prints its measured error.
"""
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


def mixed(w):
    w = dict(w)
    w["prob"] = dict(w["prob"], precision=1)
    return w


CASES = [
    # name, workload, macro steps, bound on the relative L-infinity error
    ("adv_l2-4", lambda: W.advection_gauss(l_min=2, l_max=4), 2, 1e-5),
    ("wave_planar_l2-4", lambda: W.wave_planar(l_min=2, l_max=4), 2, 1e-4),
    ("wave_shell_l3-6", lambda: W.wave_shell(l_min=3, l_max=6, half=4.0, radius=1.5, width=0.2), 1, 1e-4),
]


@pytest.mark.parametrize("name,mk,nmacro,bound", CASES)
def test_mixed_lts_against_fp64_oracle(lt, orc, name, mk, nmacro, bound):
    w = mixed(mk())
    plan = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    sol = orc.Solver(orc.Tree.build(w["spec"]), w["spec"], w["prob"])
    plan.set_initial(0.0)
    sol.set_initial(0.0)
    st = plan.stats()
    n = nmacro * 2 ** (st["l_max"] - st["l_min"])
    plan.run_substeps(n)
    sol.lts_substeps(n)
    ref = sol.state()
    err = np.abs(plan.get_state() - ref).max() / np.abs(ref).max()
    print("mixed %s: %d substeps, relative Linf error vs FP64 oracle %.3e (bound %.0e)" % (name, n, err, bound))
    assert err <= bound
    assert err > 1e-12          # the mode really computes in FP32


@pytest.mark.parametrize("name,mk,nmacro,bound", CASES[:2])
def test_mixed_gts_against_fp64_oracle(lt, orc, name, mk, nmacro, bound):
    w = mixed(mk())
    plan = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    sol = orc.Solver(orc.Tree.build(w["spec"]), w["spec"], w["prob"])
    plan.set_initial(0.0)
    sol.set_initial(0.0)
    plan.gts_steps(4)
    sol.gts_steps(4)
    ref = sol.state()
    err = np.abs(plan.get_state() - ref).max() / np.abs(ref).max()
    print("mixed GTS %s: 4 steps, relative Linf error vs FP64 oracle %.3e" % (name, err))
    assert err <= bound


def test_mixed_full_wave_first_substeps_sampled(lt, orc):
    """The benchmark workload (levels 4..9, 154,400 octants) in mixed precision: the
    first two substeps at sampled octants against the FP64 oracle's dependency cones."""
    from test_gpu_parity import cone, ring
    w = mixed(W.wave_shell())
    plan = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    plan.set_initial(0.0)
    plan.run_substeps(2)
    u = plan.get_state()
    ot = orc.Tree.build(w["spec"])
    _, lev = ot.export()
    n = len(lev)
    o2o = ot.o2o()
    rng = np.random.default_rng(21)
    S1 = np.zeros(n, bool)
    S1[rng.choice(np.where(lev == 9)[0], 4, replace=False)] = True
    need1 = cone(o2o, lev == 9, S1, 4)
    X0 = ring(o2o, need1.any(axis=0))
    need0 = cone(o2o, np.ones(n, bool), X0, 4)
    sol = orc.Solver(ot, w["spec"], w["prob"])
    sol.set_initial(0.0)
    sol.lts_substep_masked(need0.astype(np.uint8), X0.astype(np.uint8))
    sol.lts_substep_masked(need1.astype(np.uint8), S1.astype(np.uint8))
    idx = np.where(S1)[0]
    err = np.abs(u[:, idx] - sol.state()[:, idx]).max() / np.abs(u).max()
    print("mixed full wave: 2 substeps, sampled relative Linf error vs FP64 oracle %.3e" % err)
    # level 9: sigma/h = 34, eps32 * 8 * 34^2 = 5.5e-4 relative on the Laplacian, times
    # two steps of dt * |lap| / |u| ~ 0.0016 * 20
    assert err <= 1e-4
