"""LTS (Alg. 2) against GTS (Alg. 1) at equal accuracy on the GPU (Sec. 3.7: LTS takes
fewer octant-steps for the same finest step).

A shell of unmodulated Gaussian data is evolved on a four-level tree refined around
it, with LTS and with GTS at the finest step, both through the C ABI.  Their errors
against the spherical closed form chi = [(r - t) F(r - t) + (r + t) F(r + t)] / (2r)
(evaluated by the CPU oracle, whose closed form is pinned against sympy) must agree
within 10 %: LTS adds only the interface error of its time corrections (eqs. fc_1,
fc_2), which is below the scheme's own truncation error here.  The wall times of both
are printed beside the errors.
"""
import time

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


def shell_case(precision):
    w = W.wave_shell(l_min=3, l_max=6, amp=0.0, half=4.0, radius=1.5, width=0.1, band=0.3)
    w["prob"]["precision"] = precision
    return w


def state_error(u, ex):
    """largest error over both fields, each relative to the field's own size"""
    return max(np.abs(u[f] - ex[f]).max() / np.abs(ex[f]).max() for f in range(u.shape[0]))


@pytest.mark.parametrize("precision", [0, 1])
def test_lts_and_gts_equally_accurate_on_the_shell_closed_form(lt, orc, precision):
    import torch
    w = shell_case(precision)
    gt = lt.Octree(w["spec"])
    ot = orc.Tree.build(w["spec"])
    ref = orc.Solver(ot, w["spec"], w["prob"])
    plan = lt.Plan(gt, w["prob"])
    st = plan.stats()
    nsub = 2 ** (st["l_max"] - st["l_min"])
    macro = 4
    out = {}
    for mode in ("lts", "gts"):
        plan.set_initial(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (plan.run_substeps if mode == "lts" else plan.gts_steps)(macro * nsub)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        t_end = plan.time
        assert t_end == pytest.approx(macro * nsub * st["dt_finest"], rel=1e-13)
        out[mode] = (state_error(plan.get_state(), ref.exact(t_end)), wall)
    (el, wl), (eg, wg) = out["lts"], out["gts"]
    print("precision %d: %d octants, t = %.4f, error vs closed form LTS %.3e GTS %.3e (ratio %.3f); "
          "wall LTS %.1f ms GTS %.1f ms" % (precision, st["n_octants"], t_end, el, eg, el / eg, 1e3 * wl, 1e3 * wg))
    assert el <= 1.1 * eg and eg <= 1.1 * el, (el, eg)
    assert el < 1e-3
