"""Pins for the oracle's time stepping: GTS (Alg. 1), LTS (Alg. 2 with the schedule
of Fig. blk_loop and the corrections of eqs. fc_1 / fc_2) and the shared-node sync.

* a uniform tree has one level, so Alg. 2 reduces to Alg. 1: LTS == GTS bitwise;
* polynomial patch: with cubic data every ingredient is exact (FD, KO, Lagrange
  padding, RK4 in time, the Taylor stage corrections, exact boundary data), so LTS
  and GTS reproduce the closed-form solution to rounding;
* closed forms: Gaussian advection and the 1-D wave (Sec. 4.3) converge at the
  scheme's order under refinement in space and time;
* dependency cones: a substep restricted to the octants a sample depends on gives
  the same sample bitwise (this is what the full-size GPU checks rely on).
"""
import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W


def run(orc, w, mode, nsub, tree=None):
    t = tree or orc.Tree.build(w["spec"])
    s = orc.Solver(t, w["spec"], w["prob"])
    s.set_initial(0.0)
    if mode == "lts":
        s.lts_substeps(nsub)
    else:
        s.gts_steps(nsub)
    return t, s


@pytest.mark.parametrize("pde", [W.PDE_ADVECTION, W.PDE_WAVE])
def test_lts_equals_gts_on_uniform_tree(orc, pde):
    w = W.uniform(2, pde=pde)
    t = orc.Tree.build(w["spec"])
    assert len(t) == 64
    _, a = run(orc, w, "lts", 3, t)
    _, b = run(orc, w, "gts", 3, t)
    assert a.time == b.time
    assert np.array_equal(a.state(), b.state())


@pytest.mark.parametrize("mk,tol", [(lambda: W.advection_poly(5), 1e-13), (lambda: W.advection_poly(11, rk=3), 1e-13),
                                    (lambda: W.wave_poly(7), 1e-12)])
def test_polynomial_patch_exact(orc, mk, tol):
    w = mk()
    t = orc.Tree.build(w["spec"])
    _, lev = t.export()
    assert lev.max() - lev.min() == 2            # three levels, two kinds of interfaces
    L = int(lev.max() - lev.min())
    for mode in ("lts", "gts"):
        _, s = run(orc, w, mode, 2 * 2 ** L, t)
        u, ex = s.state(), s.exact(s.time)
        assert np.abs(u - ex).max() <= tol * np.abs(ex).max(), mode


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_patch_test_catches_planted_mistakes(orc, mutation):
    """Negative controls: a wrong time correction, nearest-node instead of Lagrange
    padding, a sign error in the RHS, or the step-end state for a half-way coarse
    source each break the exact reproduction of the cubic solution."""
    w = W.advection_poly(5)
    t = orc.Tree.build(w["spec"])
    _, lev = t.export()
    L = int(lev.max() - lev.min())
    try:
        orc.set_mutation(mutation)
        _, s = run(orc, w, "lts", 2 * 2 ** L, t)
        err = np.abs(s.state() - s.exact(s.time)).max() / np.abs(s.exact(s.time)).max()
    finally:
        orc.set_mutation(0)
    assert err > 1e-9, err


def convergence(orc, mk, levels, t_end, mode):
    errs = []
    for lmin, lmax in levels:
        w = mk(lmin, lmax)
        t = orc.Tree.build(w["spec"])
        s = orc.Solver(t, w["spec"], w["prob"])
        s.set_initial(0.0)
        n = int(round(t_end / s.dt_f))
        assert abs(n * s.dt_f - t_end) < 1e-12
        (s.lts_substeps if mode == "lts" else s.gts_steps)(n)
        errs.append(np.abs(s.state()[0] - s.exact(s.time)[0]).max())
    return np.array(errs)


@pytest.mark.parametrize("mode", ["lts", "gts"])
def test_advection_gauss_convergence(orc, mode):
    mk = lambda a, b: W.advection_gauss(l_min=a, l_max=b, radius=0.3, width=0.2)
    e = convergence(orc, mk, [(2, 3), (3, 4), (4, 5)], 1.0 / 24, mode)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order > 3.4), (e, order)
    assert e[-1] < 2e-6


@pytest.mark.parametrize("mode", ["lts", "gts"])
def test_planar_wave_convergence(orc, mode):
    mk = lambda a, b: W.wave_planar(l_min=a, l_max=b, width=0.2)
    e = convergence(orc, mk, [(2, 3), (3, 4), (4, 5)], 1.0 / 24, mode)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order > 3.4), (e, order)


def test_config1_advection_accuracy_and_lts_vs_gts(orc):
    w = W.advection_gauss()                       # levels 3..5, t = 0.25 in 24 macro steps
    t = orc.Tree.build(w["spec"])
    _, lev = t.export()
    assert lev.min() == 3 and lev.max() == 5
    s = orc.Solver(t, w["spec"], w["prob"])
    s.set_initial(0.0)
    nsub = int(round(w["t_end"] / s.dt_f))
    assert nsub == 96
    s.lts_substeps(nsub)
    assert s.time == pytest.approx(0.25, abs=1e-14)
    err = np.abs(s.state() - s.exact(s.time)).max()
    assert err < 2e-4                       # the pulse is under-resolved at level 3 (sigma ~ 4 h)
    # LTS error stays within 10% of GTS at equal finest step (first two macro steps)
    _, a = run(orc, w, "lts", 8, t)
    _, g = run(orc, w, "gts", 8, t)
    ea = np.abs(a.state() - a.exact(a.time)).max()
    eg = np.abs(g.state() - g.exact(g.time)).max()
    assert ea < 1.1 * eg and eg < 1.1 * ea


def test_sync_properties(orc):
    w = W.advection_poly(5)
    t = orc.Tree.build(w["spec"])
    s = orc.Solver(t, w["spec"], w["prob"])
    s.set_initial(0.0)
    u = s.state()
    su = s.sync(u)
    # a continuous cubic is reproduced at hanging nodes by the degree-6 interpolation
    assert np.abs(su - u).max() < 1e-14 * np.abs(u).max()
    rng = np.random.default_rng(4)
    v = rng.standard_normal(u.shape)
    sv = s.sync(v)
    assert np.array_equal(s.sync(sv), sv)          # idempotent
    xyz, lev = t.export()
    for b in rng.choice(len(lev), 20, replace=False):
        src, r = t.node_map(int(b))
        for n in range(343):
            if src[n] == b:
                assert sv[0, b, n] == v[0, b, n]
            elif np.all(r[n] % 2 == 0):
                assert sv[0, b, n] == v[0, src[n], r[n, 0] // 2 + 7 * (r[n, 1] // 2) + 49 * (r[n, 2] // 2)]
            else:
                assert lev[src[n]] == lev[b] - 1   # hanging nodes are fed by the coarser side


def cone_masks(o2o, active, first_rings, p, n):
    """stage j needs stage j-1 on the one-ring of every octant that needs stage j"""
    need = np.zeros((p, n), bool)
    cur = np.zeros(n, bool)
    cur[first_rings] = True
    for st in range(p - 1, -1, -1):
        need[st] = cur & active
        nb = np.unique(o2o[np.where(cur)[0]].reshape(-1))
        nb = nb[nb >= 0]
        nxt = cur.copy()
        nxt[nb] = True
        cur = nxt
    return need


def test_masked_substep_matches_full(orc):
    w = W.advection_gauss(l_min=3, l_max=5)
    t = orc.Tree.build(w["spec"])
    _, lev = t.export()
    o2o = t.o2o()
    full = orc.Solver(t, w["spec"], w["prob"])
    full.set_initial(0.0)
    full.lts_substeps(1)
    rng = np.random.default_rng(5)
    sample = rng.choice(len(lev), 3, replace=False)
    active = np.ones(len(lev), bool)             # substep 0: every level is active
    need = cone_masks(o2o, active, sample, 4, len(lev))
    assert need[0].sum() < len(lev)              # the cone is a strict subset
    part = orc.Solver(t, w["spec"], w["prob"])
    part.set_initial(0.0)
    fmask = np.zeros(len(lev), np.uint8)
    fmask[sample] = 1
    part.lts_substep_masked(need.astype(np.uint8), fmask)
    assert np.array_equal(part.state()[:, sample], full.state()[:, sample])
