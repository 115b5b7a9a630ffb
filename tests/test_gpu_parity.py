"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

* octrees (geometric predicates and the wavelet criterion) and maps (o2o, padding
  sources, shared-node owners) bit-exact;
* FP64 fields within a relative L-infinity error of 1e-12 of the oracle, for LTS
  (Alg. 2) and GTS (Alg. 1), advection and wave, exact and radiative boundaries;
* LTS == GTS bitwise on a one-level tree (Alg. 2 reduces to Alg. 1);
* FP64 wave right-hand sides (exact integer stencil sums) on data spanning 10^-300 to
  10^200, each node within a few units of 2^-52 of its own stencil scale; NaN and infinite
  inputs non-finite at exactly the oracle's nodes;
* at the full wave configuration (levels 4..9, 154,400 octants): the octree, the
  o2o map, sampled padding maps, and the first two LTS substeps at sampled octants
  (the oracle runs only the dependency cone of the sample).
"""
import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def lt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_10570_gb300 import build, ltsoct
    build.build()
    ltsoct.load()
    return ltsoct


def rel_linf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def stage_err(plan, sol, gt, j):
    """error of RK stage j as its contribution to the state: dt_l * |dK| against max|u|
    (a stage is a time derivative; FD rounding is amplified by 1/h^2 in it)"""
    st = plan.stats()
    _, lev = gt.export()
    dtl = st["dt_finest"] * 2.0 ** (st["l_max"] - lev)
    dk = np.abs(plan.get_stage(j) - sol.stage(j)) * dtl[None, :, None]
    return dk.max() / np.abs(sol.state()).max()


def both(lt, orc, w):
    gt = lt.Octree(w["spec"])
    plan = lt.Plan(gt, w["prob"])
    ot = orc.Tree.build(w["spec"])
    sol = orc.Solver(ot, w["spec"], w["prob"])
    return gt, plan, ot, sol


SMALL = [
    ("adv_l2-4", lambda: W.advection_gauss(l_min=2, l_max=4)),
    ("adv_l2-4_rk3", lambda: W.advection_gauss(l_min=2, l_max=4, rk=3)),
    ("wave_planar_l2-4", lambda: W.wave_planar(l_min=2, l_max=4)),
    ("wave_shell_l3-6", lambda: W.wave_shell(l_min=3, l_max=6, half=4.0, radius=1.5, width=0.2)),
    ("wave_shell_l2-5_rk3", lambda: W.wave_shell(l_min=2, l_max=5, half=4.0, radius=1.5, width=0.2, rk=3)),
    # wavelet refinement (Sec. 3.2.2) of the advected pulse
    ("adv_wavelet_l2-5", lambda: W.wavelet_spec(W.advection_gauss(l_min=2, l_max=5), eps=1e-7)),
]


@pytest.mark.parametrize("name,mk", SMALL)
def test_maps_bit_exact(lt, orc, name, mk):
    w = mk()
    gt, plan, ot, _ = both(lt, orc, w)
    xa, la = gt.export()
    xb, lb = ot.export()
    assert np.array_equal(xa, xb) and np.array_equal(la, lb)
    assert np.array_equal(plan.export_o2o(), ot.o2o())
    octs = np.arange(len(lb), dtype=np.int32)
    src, r = plan.export_pad_map(octs)
    nsrc, nr = plan.export_node_map(octs)
    for b in range(len(lb)):
        s, rr = ot.pad_map(b)
        assert np.array_equal(src[b], s), b
        m = s >= 0
        assert np.array_equal(r[b][m], rr[m]), b
        s, rr = ot.node_map(b)
        assert np.array_equal(nsrc[b], s) and np.array_equal(nr[b], rr), b


@pytest.mark.parametrize("name,mk", SMALL)
def test_lts_fields_match_oracle(lt, orc, name, mk):
    w = mk()
    gt, plan, ot, sol = both(lt, orc, w)
    plan.set_initial(0.0)
    sol.set_initial(0.0)
    assert rel_linf(plan.get_state(), sol.state()) <= 1e-14   # synced initial data (rounding of the interpolation)
    st = plan.stats()
    nsub = 2 ** (st["l_max"] - st["l_min"])
    # one substep (all levels), the rest of the macro step (finest-only and partial
    # substeps, half-way coarse sources), then a second macro step after reconcile
    for chunk in (1, nsub - 1, nsub):
        plan.run_substeps(chunk)
        sol.lts_substeps(chunk)
        assert plan.time == sol.time
        err = rel_linf(plan.get_state(), sol.state())
        assert err <= TOL, (name, chunk, err)
    for j in range(st["p"]):
        assert stage_err(plan, sol, gt, j) <= TOL


@pytest.mark.parametrize("name,mk", SMALL[:4])
def test_gts_fields_match_oracle(lt, orc, name, mk):
    w = mk()
    gt, plan, ot, sol = both(lt, orc, w)
    plan.set_initial(0.0)
    sol.set_initial(0.0)
    for chunk in (1, 3):
        plan.gts_steps(chunk)
        sol.gts_steps(chunk)
        err = rel_linf(plan.get_state(), sol.state())
        assert err <= TOL, (name, chunk, err)


@pytest.mark.parametrize("pde", [W.PDE_ADVECTION, W.PDE_WAVE])
def test_lts_equals_gts_bitwise_on_uniform_tree(lt, pde):
    w = W.uniform(3, pde=pde)
    a = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    b = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    a.set_initial(0.0)
    b.set_initial(0.0)
    a.run_substeps(3)
    b.gts_steps(3)
    assert a.time == b.time
    assert np.array_equal(a.get_state(), b.get_state())


def test_config1_advection_to_t_end(lt, orc):
    """levels 3..5 around the pulse, RK4, CFL 0.25, LTS to t = 0.25 (24 macro steps)."""
    w = W.advection_gauss()
    gt, plan, ot, sol = both(lt, orc, w)
    plan.set_initial(0.0)
    sol.set_initial(0.0)
    plan.advance(w["t_end"])
    sol.lts_substeps(96)
    assert plan.time == pytest.approx(0.25, abs=1e-14)
    err = rel_linf(plan.get_state(), sol.state())
    assert err <= TOL, err
    # accuracy against the closed form, and the LTS/GTS work model
    assert np.abs(plan.get_state() - sol.exact(sol.time)).max() < 2e-4
    st = plan.stats()
    s_model, wl, wg = ot.work_model()
    assert st["model_speedup"] == pytest.approx(s_model, rel=1e-14)


def test_single_octant_tree(lt, orc):
    """degenerate tree: one octant, every ghost comes from the boundary data"""
    w = W.advection_gauss(l_min=0, l_max=0, radius=0.0, width=0.5)
    gt, plan, ot, sol = both(lt, orc, w)
    assert len(gt) == 1
    plan.set_initial(0.0)
    sol.set_initial(0.0)
    plan.run_substeps(2)
    sol.lts_substeps(2)
    assert rel_linf(plan.get_state(), sol.state()) <= TOL


def test_deep_narrow_tree(lt, orc):
    """ten levels of refinement towards one point (2:1 grading through every level)"""
    w = W.advection_gauss(l_min=1, l_max=10, radius=1e-4, width=0.05)
    gt, plan, ot, sol = both(lt, orc, w)
    _, lev = gt.export()
    assert lev.min() == 2 and lev.max() == 10 and len(set(lev)) == 9
    plan.set_initial(0.0)
    sol.set_initial(0.0)
    plan.run_substeps(3)
    sol.lts_substeps(3)
    assert rel_linf(plan.get_state(), sol.state()) <= TOL


def stencil_scale(tile):
    """largest |input| among each node's 19 stencil points (centre and the 6 x 3 axis
    neighbours), over both fields: [343] in node order (i fastest) from a padded tile
    [nf][13][13][13] in (k, j, i) order"""
    a = np.abs(tile).max(axis=0)
    c = slice(3, 10)
    m = a[c, c, c].copy()
    for s in (1, 2, 3):
        for lo in (3 - s, 3 + s):
            sl = slice(lo, lo + 7)
            m = np.maximum(m, a[sl, c, c])
            m = np.maximum(m, a[c, sl, c])
            m = np.maximum(m, a[c, c, sl])
    return m.reshape(-1)


def test_fp64_wave_rhs_on_wide_range_data(lt, orc):
    """FP64 wave right-hand sides partly come from exact integer stencil sums on a per-node
    grid (floating point for magnitudes outside [2^-968, 2^500), infinities and NaNs).
    State with a magnitude class per octant and field (1 down to 1e-300, up to 1e200, zero,
    subnormal), random signs, scattered zeros and subnormals: every node's first stage
    agrees with the oracle's FP64 evaluation to a few units of 2^-52 of the node's own
    stencil scale, not of the global maximum (Sec. 4 wave equation, KO dissipation)."""
    w = W.wave_shell(l_min=2, l_max=4, half=4.0, radius=1.5, width=0.2)
    gt, plan, ot, sol = both(lt, orc, w)
    st = plan.stats()
    n = st["n_octants"]
    rng = np.random.default_rng(11)
    mags = np.array([1.0, 1e-5, 1e-20, 1e-100, 1e-290, 1e-300, 1e140, 1e200, 0.0, 4e-320])
    cls = rng.integers(0, len(mags), size=(2, n))
    u = rng.standard_normal((2, n, 343)) * mags[cls][:, :, None]
    u[rng.random(u.shape) < 0.1] = 0.0
    sub = rng.random(u.shape) < 0.02
    u[sub] = 3e-320 * np.where(rng.random(int(sub.sum())) < 0.5, -1.0, 1.0)
    plan.set_state(u)
    sol.set_state(u)
    scale = np.stack([stencil_scale(sol.tile(b)) for b in range(n)])  # [n][343]
    plan.run_substeps(1)
    sol.lts_substeps(1)
    _, lev = gt.export()
    half = w["spec"]["hi"]
    h = 2.0 * half / (6.0 * 2.0 ** lev)
    kos = w["prob"]["ko_sigma"] / (64.0 * h)
    # bound of the operators' coefficients acting on the inputs: Laplacian and dissipation
    # (192 = the sums of the integer weights' magnitudes), the radiative gradient at the
    # boundary (|x| <= half * sqrt(3), 18 / (12 h), plus 2 / r)
    coef = 192.0 * (1.0 / (12.0 * h * h) + kos) + 3.0 * half * 18.0 / (12.0 * h) + 4.0
    kg, ko = plan.get_stage(0), sol.stage(0)
    err = np.abs(kg - ko) / (coef[None, :, None] * scale[None] + 1e-320)
    assert np.isfinite(kg).all()
    assert err.max() <= 64 * 2.0 ** -52
    # octants of tiny and of huge magnitudes are both present and checked on their own scale
    assert (scale < 1e-280).any() and (scale > 1e180).any()


def test_fp64_nonfinite_inputs_propagate(lt, orc):
    """A NaN or an infinity in the state is never turned into a finite value by the exact
    integer paths (stencil sums, prolongation lines): nodes whose inputs reach one take the
    floating-point formula, so the GPU's first RK stage is non-finite at exactly the nodes
    where the oracle's is."""
    w = W.wave_shell(l_min=2, l_max=4, half=4.0, radius=1.5, width=0.2)
    gt, plan, ot, sol = both(lt, orc, w)
    n = plan.stats()["n_octants"]
    rng = np.random.default_rng(5)
    u = rng.standard_normal((2, n, 343))
    picks = rng.choice(n, size=6, replace=False)
    for t, b in enumerate(picks):
        node = 3 + 7 * 3 + 49 * 3 if t % 2 == 0 else int(rng.integers(0, 343))
        u[t % 2, b, node] = (np.nan, np.inf, -np.inf)[t % 3]
    plan.set_state(u)
    sol.set_state(u)
    plan.run_substeps(1)
    sol.lts_substeps(1)
    for j in range(2):
        kg, ko = plan.get_stage(j), sol.stage(j)
        fg, fo = np.isfinite(kg), np.isfinite(ko)
        assert (~fo).any()
        assert np.array_equal(fg, fo), j
        assert np.abs(kg[fo] - ko[fo]).max() <= 1e-9 * np.abs(ko[fo]).max()


def test_invalid_calls_fail_loudly(lt):
    w = W.advection_gauss(l_min=2, l_max=3)
    plan = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    plan.set_initial(0.0)
    with pytest.raises(lt.LtsError):
        plan.advance(0.123456)            # not a whole number of macro steps
    plan.run_substeps(1)
    with pytest.raises(lt.LtsError):
        plan.advance(1.0)                 # inside a macro step
    bad = dict(w["prob"], bc=W.BC_RADIATIVE)
    with pytest.raises(lt.LtsError):
        lt.Plan(lt.Octree(w["spec"]), bad)


# ---------------------------------------------------------------------------
# full wave configuration: sampled checks
# ---------------------------------------------------------------------------

def ring(o2o, members):
    nb = o2o[np.where(members)[0]].reshape(-1)
    out = members.copy()
    out[nb[nb >= 0]] = True
    return out


def cone(o2o, active, targets, p):
    need = np.zeros((p, len(active)), bool)
    cur = targets.copy()
    for st in range(p - 1, -1, -1):
        need[st] = cur & active
        cur = ring(o2o, cur)
    return need


@pytest.fixture(scope="module")
def full_wave(lt, orc):
    w = W.wave_shell()
    gt = lt.Octree(w["spec"])
    ot = orc.Tree.build(w["spec"])
    return w, gt, ot


def test_full_wave_maps(lt, orc, full_wave):
    w, gt, ot = full_wave
    xa, la = gt.export()
    xb, lb = ot.export()
    assert len(la) == 154400
    assert np.array_equal(xa, xb) and np.array_equal(la, lb)
    plan = lt.Plan(gt, w["prob"])
    assert np.array_equal(plan.export_o2o(), ot.o2o())
    rng = np.random.default_rng(11)
    # every level, and octants at level interfaces
    sample = np.concatenate([rng.choice(np.where(lb == l)[0], 8, replace=False) for l in range(4, 10)])
    src, r = plan.export_pad_map(sample.astype(np.int32))
    nsrc, nr = plan.export_node_map(sample.astype(np.int32))
    for i, b in enumerate(sample):
        s, rr = ot.pad_map(int(b))
        assert np.array_equal(src[i], s)
        m = s >= 0
        assert np.array_equal(r[i][m], rr[m])
        s, rr = ot.node_map(int(b))
        assert np.array_equal(nsrc[i], s) and np.array_equal(nr[i], rr)


def test_full_wave_first_substeps_sampled(lt, orc, full_wave):
    """Substep 0 (all levels step, fine<->coarse corrections of eq. fc_1) and
    substep 1 (finest level only, half-way coarse sources of eq. fc_2) of the
    benchmark workload, compared at sampled octants of every level."""
    w, gt, ot = full_wave
    plan = lt.Plan(gt, w["prob"])
    plan.set_initial(0.0)
    plan.run_substeps(2)
    u_gpu = plan.get_state()
    k_gpu = [plan.get_stage(j) for j in range(4)]
    _, lev = ot.export()
    n = len(lev)
    o2o = ot.o2o()
    rng = np.random.default_rng(12)
    fine = np.where(lev == 9)[0]
    S1 = np.zeros(n, bool)
    S1[rng.choice(fine, 6, replace=False)] = True
    # substep 1: only level 9 is active
    act1 = lev == 9
    need1 = cone(o2o, act1, S1, 4)
    # everything substep 1 reads must be final after substep 0
    X0 = ring(o2o, need1.any(axis=0))
    # plus sampled octants of every level checked after substep 0 itself
    S0 = np.zeros(n, bool)
    for l in range(4, 9):
        S0[rng.choice(np.where(lev == l)[0], 3, replace=False)] = True
    X0 |= S0
    need0 = cone(o2o, np.ones(n, bool), X0, 4)
    sol = orc.Solver(ot, w["spec"], w["prob"])
    sol.set_initial(0.0)
    sol.lts_substep_masked(need0.astype(np.uint8), X0.astype(np.uint8))
    u0 = sol.state()
    idx0 = np.where(S0)[0]
    sol.lts_substep_masked(need1.astype(np.uint8), S1.astype(np.uint8))
    u1 = sol.state()
    idx1 = np.where(S1)[0]
    # relative L-infinity over the state vector (both fields), as elsewhere; sampled
    # octants far from the shell hold values near zero
    def err(a, b, full):
        return np.abs(a - b).max() / np.abs(full).max()
    assert err(u_gpu[:, idx1], u1[:, idx1], u_gpu) <= TOL
    # levels 4..8 stepped once in substep 0 and then rested
    assert err(u_gpu[:, idx0], u0[:, idx0], u_gpu) <= TOL
    st = plan.stats()
    dtl = st["dt_finest"] * 2.0 ** (st["l_max"] - lev)
    for j in range(4):
        kj = sol.stage(j)
        for idx in (idx1, idx0):
            dk = np.abs(k_gpu[j][:, idx] - kj[:, idx]) * dtl[None, idx, None]
            assert dk.max() / np.abs(u_gpu).max() <= TOL


@pytest.mark.parametrize("name,mk", SMALL + [
    ("nonlinear_l3-5", lambda: W.wave_nonlinear(l_min=3, l_max=5, half=4.0, radius=1.5, width=0.2)),
    ("uniform_l3_wave", lambda: W.uniform(3, pde=W.PDE_WAVE)),
    ("orbit_l2-5", lambda: W.wave_orbit(l_min=2, l_max=5, band=0.3, half=2.0, omega=3.0, precision=0)),
    ("planar_mixed", lambda: dict(W.wave_planar(l_min=2, l_max=4),
                                  prob=dict(W.wave_planar(l_min=2, l_max=4)["prob"], precision=1)))])
def test_blocking_is_bit_identical(lt, name, mk):
    """Sec. 3.2.5 blocks: stepping complete sibling groups as 13^3-node blocks gives the
    same bits as stepping every octant alone, under LTS (all substep kinds, reconcile)
    and GTS."""
    w = mk()
    gt = lt.Octree(w["spec"])
    a, b = lt.Plan(gt, w["prob"]), lt.Plan(gt, w["prob"])
    b.set_blocking(False)
    st = a.stats()
    if name.startswith(("uniform", "orbit")):
        assert st["blocked_octants"] > 0
    if name.startswith("uniform"):
        assert st["blocked_octants"] == st["n_octants"]
    nsub = 2 ** (st["l_max"] - st["l_min"])
    for p in (a, b):
        p.set_initial(0.0)
        p.run_substeps(nsub + 3)
    assert np.array_equal(a.get_state(), b.get_state())
    for j in range(st["p"]):
        assert np.array_equal(a.get_stage(j), b.get_stage(j))
    for p in (a, b):
        p.gts_steps(2)
    assert np.array_equal(a.get_state(), b.get_state())


def test_profiling_counts_stage_and_prolongation_launches(lt):
    """lts_kernel_stats / lts_prolong_stats: one substep with every level active is 4 RK
    stages, each one stage launch and one prolongation launch over every coarser source;
    LTS counts the time-corrected inputs in the prolongation's flops, GTS does not."""
    w = W.wave_shell(l_min=3, l_max=6, half=4.0, radius=1.5, width=0.2)
    plan = lt.Plan(lt.Octree(w["spec"]), w["prob"])
    plan.set_initial(0.0)
    plan.set_profiling(True)
    plan.kernel_stats(reset=True)
    plan.prolong_stats(reset=True)
    plan.run_substeps(1)
    ks, ps = plan.kernel_stats(reset=True), plan.prolong_stats(reset=True)
    st = plan.stats()
    assert ks["launches"] == 4 and ks["node_stages"] == 4 * st["n_octants"] * 343
    assert ps["launches"] == 4 and ps["ms"] > 0 and ps["sources"] > 0 and ps["sources"] % 4 == 0
    assert 0 < ps["sources"] // 4 < st["n_octants"]
    lts_flops = ps["flops"]
    plan.gts_steps(1)
    gs = plan.prolong_stats(reset=True)
    plan.set_profiling(False)
    assert gs["launches"] == 4 and gs["sources"] == ps["sources"]
    # the interpolation alone under GTS: fewer flops than with the time corrections
    assert 0 < gs["flops"] < lts_flops
