"""Pins for the oracle's outer boundary on the wave equation (Sec. 4.2, eqs. chi, phi
with the radiative condition) and for its spherical closed form.

The radiative condition is read as the outgoing-wave form: at a node on the domain
boundary, df/dt = -(x^i/r) d_i f - k f / r, with k = 1 for chi and k = 2 for phi (the
paper's fall-off powers), the derivatives centred, and the exterior ghosts of the
padded block filled by cubic extrapolation along each axis (x, then y, then z).

What fixes each part, independently of the oracle's code:

* cubic extrapolation: the unzipped block of a tensor-product cubic (degree <= 3 in
  each variable) reproduces that cubic at every exterior ghost, on face, edge and
  corner octants alike, since each one-dimensional extrapolation is exact for cubics;
* first RK stage on cubic data: at interior nodes the right-hand side is exactly
  (phi, lap chi) (4th-order differences exact, Kreiss-Oliger zero), including nodes
  whose stencils reach extrapolated ghosts;
* the radiative formula: any f = g(r - t) / r^k satisfies df/dt = -d_r f - k f / r
  exactly, so on chi = g(r)/r and phi = h(r)/r^2 the boundary right-hand side must
  converge to -g'(r)/r and -h'(r)/r^2 as the octants are refined; a swapped k or a
  flipped sign leaves an O(1) error that does not shrink;
* the spherical closed form chi = [(r - t) F(r - t) + (r + t) F(r + t)] / (2r): an LTS
  solve of shell data with exact boundary values converges to it at 4th order.
"""
import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W

ROOT = 2 ** 20


def wave_problem(bc=W.BC_RADIATIVE):
    return dict(pde=W.PDE_WAVE, adv=(0.0, 0.0, 0.0), cfl=0.25, ko_sigma=0.1, rk=4, bc=bc,
                ic=W.IC_WAVE_REST, ic_params=[])


def corner_tree_spec():
    """[-1,1]^3 on levels 2..3, refined near one corner: face, edge and corner octants
    on both levels, and level interfaces that meet the boundary."""
    return dict(lo=-1.0, hi=1.0, l_min=2, l_max=3, kind=W.REFINE_BALLS, centers=[(0.6, 0.6, 0.6)],
                radius=0.3, band=0.0)


def tensor_cubic(seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (4, 4, 4))       # c[i, j, k] x^i y^j z^k, degree <= 3 per variable


def eval_tc(c, X, Y, Z):
    v = np.zeros_like(X)
    for i in range(4):
        for j in range(4):
            for k in range(4):
                v += c[i, j, k] * X ** i * Y ** j * Z ** k
    return v


def grad_lap_tc(c, X, Y, Z):
    g = [np.zeros_like(X) for _ in range(3)]
    lap = np.zeros_like(X)
    for i in range(4):
        for j in range(4):
            for k in range(4):
                cv = c[i, j, k]
                if i:
                    g[0] += cv * i * X ** (i - 1) * Y ** j * Z ** k
                if j:
                    g[1] += cv * j * X ** i * Y ** (j - 1) * Z ** k
                if k:
                    g[2] += cv * k * X ** i * Y ** j * Z ** (k - 1)
                if i > 1:
                    lap += cv * i * (i - 1) * X ** (i - 2) * Y ** j * Z ** k
                if j > 1:
                    lap += cv * j * (j - 1) * X ** i * Y ** (j - 2) * Z ** k
                if k > 1:
                    lap += cv * k * (k - 1) * X ** i * Y ** j * Z ** (k - 2)
    return g, lap


def node_coords(xyz, lev, lo, hi, offsets):
    """physical coordinates [N][len(offsets)^3] of lattice points 6A + i e (i in offsets),
    in node order i + n j + n^2 k"""
    e = (ROOT >> lev).astype(np.float64)[:, None]
    o = np.asarray(offsets, np.float64)
    K, J, I = np.meshgrid(o, o, o, indexing="ij")
    I, J, K = I.reshape(-1)[None], J.reshape(-1)[None], K.reshape(-1)[None]
    scale = (hi - lo) / (6.0 * ROOT)
    X = lo + scale * (6.0 * xyz[:, 0:1] + I * e)
    Y = lo + scale * (6.0 * xyz[:, 1:2] + J * e)
    Z = lo + scale * (6.0 * xyz[:, 2:3] + K * e)
    return X, Y, Z


def boundary_kind(xyz, lev):
    """number of domain faces each octant touches (1 face, 2 edge, 3 corner)"""
    e = (ROOT >> lev)[:, None]
    return ((xyz == 0) | (xyz + e == ROOT)).sum(axis=1)


def set_cubic_state(orc, c_chi, c_phi):
    spec = corner_tree_spec()
    t = orc.Tree.build(spec)
    xyz, lev = t.export()
    s = orc.Solver(t, spec, wave_problem())
    X, Y, Z = node_coords(xyz, lev, spec["lo"], spec["hi"], range(7))
    u = np.stack([eval_tc(c_chi, X, Y, Z), eval_tc(c_phi, X, Y, Z)])
    s.set_state(u, 0.0)
    return spec, t, xyz, lev, s, (X, Y, Z)


@pytest.mark.parametrize("mutation", [0, 7])
def test_extrapolated_ghosts_reproduce_tensor_cubics(orc, mutation):
    c_chi, c_phi = tensor_cubic(21), tensor_cubic(22)
    spec, t, xyz, lev, s, _ = set_cubic_state(orc, c_chi, c_phi)
    kinds = boundary_kind(xyz, lev)
    for kind in (1, 2, 3):                       # face, edge and corner octants on both levels
        for l in (2, 3):
            assert np.any((kinds == kind) & (lev == l)), (kind, l)
    X, Y, Z = node_coords(xyz, lev, spec["lo"], spec["hi"], range(-3, 10))
    worst = 0.0
    n_ghost = 0
    try:
        orc.set_mutation(mutation)
        for b in np.where(kinds > 0)[0]:
            T = s.tile(b).reshape(2, -1)
            ex = [eval_tc(c_chi, X[b], Y[b], Z[b]), eval_tc(c_phi, X[b], Y[b], Z[b])]
            outside = (np.abs(X[b]) > 1.0) | (np.abs(Y[b]) > 1.0) | (np.abs(Z[b]) > 1.0)
            n_ghost += outside.sum()
            for f in range(2):
                scale = np.abs(ex[f]).max()
                worst = max(worst, np.abs(T[f] - ex[f]).max() / scale)
    finally:
        orc.set_mutation(0)
    assert n_ghost > 0
    if mutation == 0:
        # exterior ghosts and interior padding alike; a corner ghost is extrapolated three
        # times with weights of absolute sum up to 111 (position -3: 20, -45, 36, -10), so
        # rounding grows to about 111^3 * 2^-52 = 3e-10 of the values there
        assert worst < 1e-9, worst
    else:
        assert worst > 1e-3, worst               # a wrong extrapolation row is caught


def test_first_stage_on_cubics_at_and_near_the_boundary(orc):
    c_chi, c_phi = tensor_cubic(31), tensor_cubic(32)
    spec, t, xyz, lev, s, (X, Y, Z) = set_cubic_state(orc, c_chi, c_phi)
    s.lts_substeps(1)                            # substep 0: every level active, stage 1 = F(u)
    k1 = s.stage(0)
    chi, phi = eval_tc(c_chi, X, Y, Z), eval_tc(c_phi, X, Y, Z)
    (gc, lap_chi), (gp, _) = grad_lap_tc(c_chi, X, Y, Z), grad_lap_tc(c_phi, X, Y, Z)
    on_bnd = (np.abs(np.abs(X) - 1.0) < 1e-14) | (np.abs(np.abs(Y) - 1.0) < 1e-14) | (np.abs(np.abs(Z) - 1.0) < 1e-14)
    assert on_bnd.any() and (~on_bnd).any()
    # interior nodes: chi_t = phi, phi_t = lap chi exactly (stencils reach exterior ghosts
    # on octants at the boundary)
    assert np.abs(k1[0][~on_bnd] - phi[~on_bnd]).max() < 1e-11 * np.abs(phi).max()
    assert np.abs(k1[1][~on_bnd] - lap_chi[~on_bnd]).max() < 1e-10 * np.abs(lap_chi).max()
    # boundary nodes: the outgoing-wave condition with k = 1 (chi) and k = 2 (phi)
    r = np.where(on_bnd, np.sqrt(X ** 2 + Y ** 2 + Z ** 2), 1.0)   # r >= 1 on the boundary
    rd_chi = (X * gc[0] + Y * gc[1] + Z * gc[2]) / r
    rd_phi = (X * gp[0] + Y * gp[1] + Z * gp[2]) / r
    want_chi = -rd_chi - 1.0 * chi / r
    want_phi = -rd_phi - 2.0 * phi / r
    assert np.abs(k1[0][on_bnd] - want_chi[on_bnd]).max() < 1e-10 * np.abs(want_chi[on_bnd]).max()
    assert np.abs(k1[1][on_bnd] - want_phi[on_bnd]).max() < 1e-10 * np.abs(want_phi[on_bnd]).max()
    # one boundary node written out by hand: the corner (1, 1, 1) of the cube
    b = int(np.argmax((xyz[:, 0] + (ROOT >> lev) == ROOT) & (xyz[:, 1] + (ROOT >> lev) == ROOT)
                      & (xyz[:, 2] + (ROOT >> lev) == ROOT)))
    n = 342                                      # node (6, 6, 6)
    assert X[b, n] == 1.0 and Y[b, n] == 1.0 and Z[b, n] == 1.0
    # at (1,1,1): chi = sum c, x.grad chi = sum (i + j + k) c, r = sqrt 3
    cs, ds = c_chi.sum(), sum((i + j + k) * c_chi[i, j, k] for i in range(4) for j in range(4) for k in range(4))
    ps, qs = c_phi.sum(), sum((i + j + k) * c_phi[i, j, k] for i in range(4) for j in range(4) for k in range(4))
    r3 = np.sqrt(3.0)
    assert k1[0, b, n] == pytest.approx(-ds / r3 - 1.0 * cs / r3, rel=1e-11)
    assert k1[1, b, n] == pytest.approx(-qs / r3 - 2.0 * ps / r3, rel=1e-11)


def outgoing_error(orc, level, mutation=0, half=2.0, s0=2.6, w=0.5):
    """chi = g(r)/r, phi = h(r)/r^2 on a uniform tree of [-half, half]^3; returns the
    largest error of the first RK stage at boundary nodes against d/dt of the outgoing
    waves g(r - t)/r and h(r - t)/r^2, relative to their size there."""
    spec = dict(lo=-half, hi=half, l_min=level, l_max=level, kind=W.REFINE_BALLS, centers=[(0.0, 0.0, 0.0)],
                radius=0.0, band=0.0)
    t = orc.Tree.build(spec)
    xyz, lev = t.export()
    s = orc.Solver(t, spec, wave_problem())
    X, Y, Z = node_coords(xyz, lev, -half, half, range(7))
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    g = np.exp(-(r - s0) ** 2 / w)
    dg = -2.0 * (r - s0) / w * g
    h = 0.7 * np.exp(-(r - s0 - 0.2) ** 2 / w)
    dh = -2.0 * (r - s0 - 0.2) / w * h
    far = r > 1.0                                # values near the origin never reach the boundary
    rs = np.where(far, r, 1.0)
    s.set_state(np.stack([np.where(far, g / rs, 0.0), np.where(far, h / rs ** 2, 0.0)]), 0.0)
    try:
        orc.set_mutation(mutation)
        s.lts_substeps(1)
    finally:
        orc.set_mutation(0)
    k1 = s.stage(0)
    on_bnd = (np.abs(np.abs(X) - half) < 1e-12) | (np.abs(np.abs(Y) - half) < 1e-12) | (np.abs(np.abs(Z) - half) < 1e-12)
    want = [-dg / rs, -dh / rs ** 2]
    return np.array([np.abs(k1[f][on_bnd] - want[f][on_bnd]).max() / np.abs(want[f][on_bnd]).max()
                     for f in range(2)])


def test_radiative_condition_converges_on_outgoing_waves(orc):
    e = np.array([outgoing_error(orc, lv) for lv in (2, 3, 4)])
    order = np.log2(e[:-1] / e[1:])
    # one-sided differences through cubic-extrapolated ghosts: third order at the boundary
    assert np.all(order > 2.5), (e, order)
    assert np.all(e[-1] < 2e-3), e


@pytest.mark.parametrize("mutation", [5, 6])
def test_radiative_condition_catches_planted_mistakes(orc, mutation):
    """k of chi and phi swapped, or the sign of the x^i/r term flipped: the boundary
    right-hand side no longer approaches d/dt of the outgoing waves."""
    e = np.array([outgoing_error(orc, lv, mutation) for lv in (2, 3)])
    assert np.all(e[-1] > 0.05), e
    assert np.all(e[0] / e[1] < 2.0), e


def test_shell_closed_form_convergence(orc):
    """LTS solves of shell data (no modulation, exact boundary values) on trees refined
    around the shell converge to the spherical closed form at 4th order."""
    errs = []
    for a, b in [(2, 3), (3, 4), (4, 5)]:
        w = W.wave_shell(l_min=a, l_max=b, amp=0.0, bc=W.BC_EXACT, half=2.0, radius=1.0, width=0.05, band=0.6)
        t = orc.Tree.build(w["spec"])
        _, lev = t.export()
        assert lev.min() == a and lev.max() == b
        s = orc.Solver(t, w["spec"], w["prob"])
        s.set_initial(0.0)
        n = int(round((1.0 / 24) / s.dt_f))
        assert abs(n * s.dt_f - 1.0 / 24) < 1e-14
        s.lts_substeps(n)
        ex = s.exact(s.time)
        errs.append(np.abs(s.state() - ex).max(axis=(1, 2)) / np.abs(ex).max(axis=(1, 2)))
    e = np.array(errs)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order >= 3.5), (e, order)
