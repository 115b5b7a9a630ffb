"""Pins for the oracle's source terms and the orbit-circle refinement.

* eq. phi's non-linear term -c sin(2 chi)/r^2: on a constant state the Laplacian and
  the Kreiss-Oliger terms vanish, so the first RK stage of phi is the term itself;
  on shell data it is the difference between runs with c = 1 and c = 0;
* the orbiting Gaussian sources: from rest, the first two RK stages of phi are the
  source at the stage times t_b + c_s dt_l of each level (c = 0, 1/2 for RK4 and
  0, 1 for SSPRK3), written out here independently;
* a one-level tree still makes LTS and GTS identical bit for bit with both sources;
* the circle predicate agrees with a brute-force distance from the box to a dense
  sampling of the circle.
"""
import math

import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W

ROOT = 1 << 20


def node_positions(tree, spec):
    """x, y, z of every node [N][343] and a mask of the nodes on the domain boundary"""
    xyz, lev = tree.export()
    e = (ROOT >> lev.astype(np.int64))[:, None]
    i = np.arange(343)
    ijk = np.stack([i % 7, (i // 7) % 7, i // 49])
    P = 6 * xyz.astype(np.int64)[:, :, None] + ijk[None, :, :] * e[:, None, :]
    x = spec["lo"] + (spec["hi"] - spec["lo"]) * (P / (6.0 * ROOT))
    bnd = ((P == 0) | (P == 6 * ROOT)).any(axis=1)
    return x, bnd, lev


def test_nonlinear_term_on_constant_state(orc):
    w = W.uniform(2, pde=W.PDE_WAVE)
    w["prob"]["nl_c"] = 1.0
    t = orc.Tree.build(w["spec"])
    s = orc.Solver(t, w["spec"], w["prob"])
    u = np.zeros((2, len(t), 343))
    u[0] = 0.3
    s.set_state(u, 0.0)
    s.gts_steps(1)
    k0 = s.stage(0)
    x, bnd, _ = node_positions(t, w["spec"])
    r2 = (x ** 2).sum(axis=1)
    want = np.where(r2 > 0, -np.sin(0.6) / np.where(r2 > 0, r2, 1.0), 0.0)
    inner = ~bnd
    assert (r2[inner] == 0).any()                      # the origin is a node: the r = 0 reading
    assert np.abs(k0[0][inner]).max() <= 1e-15          # Kreiss-Oliger of a constant: rounding only
    assert np.abs(k0[1][inner] - want[inner]).max() <= 1e-14 * np.abs(want).max()


def test_nonlinear_term_is_the_difference_of_two_runs(orc):
    w1 = W.wave_nonlinear(l_min=2, l_max=3, half=4.0, radius=1.5, width=0.2)
    w0 = W.wave_shell(l_min=2, l_max=3, half=4.0, radius=1.5, width=0.2)
    t = orc.Tree.build(w1["spec"])
    _, lev = t.export()
    assert lev.min() < lev.max()
    k = []
    for w in (w1, w0):
        s = orc.Solver(t, w["spec"], w["prob"])
        s.set_initial(0.0)
        u0 = s.state()
        s.lts_substeps(1)                                # substep 0: every level steps
        k.append(s.stage(0))
    x, bnd, _ = node_positions(t, w1["spec"])
    r2 = (x ** 2).sum(axis=1)
    want = np.where(r2 > 0, -np.sin(2 * u0[0]) / np.where(r2 > 0, r2, 1.0), 0.0)
    d = k[0][1] - k[1][1]
    assert np.abs(d[~bnd] - want[~bnd]).max() <= 1e-13 * np.abs(want).max()
    assert np.array_equal(k[0][0], k[1][0])              # chi_t = phi is untouched


def orbit_source(x, t, R, om, wd, A):
    c = np.array([R * math.cos(om * t), R * math.sin(om * t), 0.0])
    d1 = ((x - c[None, :, None]) ** 2).sum(axis=1)
    d2 = ((x + c[None, :, None]) ** 2).sum(axis=1)
    return A * (np.exp(-d1 / wd) + np.exp(-d2 / wd))


@pytest.mark.parametrize("rk,c1", [(4, 0.5), (3, 1.0)])
def test_orbit_source_at_stage_times(orc, rk, c1):
    w = W.wave_orbit(l_min=2, l_max=4, band=0.3, half=2.0, omega=3.0, ko_sigma=0.0, rk=rk, precision=0)
    t = orc.Tree.build(w["spec"])
    _, lev = t.export()
    assert lev.max() - lev.min() == 2
    s = orc.Solver(t, w["spec"], w["prob"])
    t0 = 0.7
    s.set_state(np.zeros((2, len(t), 343)), t0)
    s.lts_substeps(1)
    x, bnd, lev = node_positions(t, w["spec"])
    dt = s.dt_f * 2.0 ** (lev.max() - lev)[:, None]
    R, om, wd, A = w["prob"]["orbit_params"]
    k0, k1 = s.stage(0), s.stage(1)
    want0 = orbit_source(x, t0, R, om, wd, A)
    assert np.abs(want0).max() > 0.5
    assert np.abs(k0[1] - want0)[~bnd].max() <= 1e-14
    assert np.array_equal(k0[0][~bnd], np.zeros((~bnd).sum()))
    # stage 1 at t0 + c1 dt_l, per level
    want1 = np.empty_like(want0)
    for l in np.unique(lev):
        m = lev == l
        want1[m] = orbit_source(x[m], t0 + c1 * s.dt_f * 2.0 ** (lev.max() - l), R, om, wd, A)
    assert np.abs(k1[1] - want1)[~bnd].max() <= 1e-14
    # a different stage time would be visible
    assert np.abs(want1 - want0)[~bnd].max() > 1e-6


def test_lts_equals_gts_on_uniform_tree_with_sources(orc):
    w = W.uniform(2, pde=W.PDE_WAVE)
    w["prob"].update(nl_c=1.0, orbit=1, orbit_params=[1.0, 0.5, 0.05, 1.0])
    t = orc.Tree.build(w["spec"])
    out = []
    for mode in ("lts", "gts"):
        s = orc.Solver(t, w["spec"], w["prob"])
        s.set_initial(0.0)
        (s.lts_substeps if mode == "lts" else s.gts_steps)(3)
        out.append(s.state())
    assert np.array_equal(out[0], out[1])


def sampled_circle_distance(box_lo, edge, c, R, n=20001):
    th = np.linspace(0.0, 2 * np.pi, n)
    pts = np.stack([c[0] + R * np.cos(th), c[1] + R * np.sin(th), np.full(n, float(c[2]))], axis=1)
    lo = np.asarray(box_lo, float)
    q = np.clip(pts, lo, lo + edge)
    return np.sqrt(((pts - q) ** 2).sum(axis=1)).min()


def test_circle_predicate_against_sampled_distance(orc):
    rng = np.random.Generator(np.random.PCG64(11))
    spec = W.wave_orbit(l_min=0, l_max=12, band=0.3, half=2.0)["spec"]
    scale = ROOT / (spec["hi"] - spec["lo"])
    R, b = spec["radius"] * scale, spec["band"] * scale
    c = [round((0.0 - spec["lo"]) * scale)] * 3
    seen = {True: 0, False: 0}
    for _ in range(400):
        level = int(rng.integers(2, 9))
        edge = ROOT >> level
        # anchors near the circle
        th = rng.uniform(0, 2 * np.pi)
        p = np.array([c[0] + R * np.cos(th), c[1] + R * np.sin(th), c[2]]) + rng.normal(0, 2 * b, 3)
        a = [int(np.clip(v // edge, 0, (ROOT // edge) - 1)) * edge for v in p]
        d = sampled_circle_distance(a, edge, c, R)
        if abs(d - b) < 1e-3 * R:
            continue
        got = bool(orc.refine_pred(spec, a[0], a[1], a[2], level))
        assert got == (d <= b), (a, level, d, b)
        seen[got] += 1
    assert seen[True] > 50 and seen[False] > 50


def test_circle_tree_is_balanced_and_refined_around_the_orbit(orc):
    w = W.wave_orbit(l_min=2, l_max=5, band=0.2, half=2.0)
    t = orc.Tree.build(w["spec"])
    xyz, lev = t.export()
    spec = w["spec"]
    for q in range(len(t)):
        if lev[q] < spec["l_max"]:
            assert not orc.refine_pred(spec, int(xyz[q, 0]), int(xyz[q, 1]), int(xyz[q, 2]), int(lev[q]))
    # the finest octants lie within the band of the circle
    scale = ROOT / (spec["hi"] - spec["lo"])
    fin = np.flatnonzero(lev == spec["l_max"])
    assert len(fin) > 0
    R, b = spec["radius"] * scale, spec["band"] * scale
    c = [round(-spec["lo"] * scale)] * 3
    e = ROOT >> spec["l_max"]
    for q in fin[:: max(1, len(fin) // 40)]:
        pq = xyz[q].astype(float)
        # a finest octant is a child of a split box that came within the band: within
        # the band plus the parent's diagonal 2 sqrt(3) e
        assert sampled_circle_distance(pq, e, c, R) <= b + 2 * math.sqrt(3) * e
