"""Pins for the oracle's spatial operators, RK tableaus, LTS stage corrections and
closed forms.

* finite differences: exact on polynomials up to the stencil order (Sec. 3.3, a reading of the paper);
* Kreiss-Oliger: the 6th difference annihilates degree <= 5 and gives 6! h^6 on x^6;
* Lagrange 7 -> 13 interpolation (coarse-to-fine padding, Fig. unzip) reproduces degree <= 6;
* omega tables (eqs. rk_crrection, fc_1, fc_2): a ghost built from a source's RK
  stages equals the requester's own RK stage input exactly for u' = J u with J
  nilpotent (the Taylor reconstruction is then exact), for every relation;
* closed forms: time derivatives against sympy.
"""
import math

import numpy as np
import pytest


def poly_tile(c, h, origin=(0.3, -0.2, 0.1)):
    """values of sum c[i,j,k] x^i y^j z^k on the 13^3 padded lattice with spacing h"""
    idx = np.arange(-3, 10)
    x = origin[0] + h * idx
    y = origin[1] + h * idx
    z = origin[2] + h * idx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    v = np.zeros_like(X)
    for (i, j, k), cv in c.items():
        v += cv * X ** i * Y ** j * Z ** k
    return v, (X, Y, Z)


def interior(a):
    return a[3:10, 3:10, 3:10].reshape(-1)


@pytest.mark.parametrize("h", [0.05, 0.013])
def test_fd_exact_on_polynomials(orc, h):
    rng = np.random.default_rng(1)
    # total degree <= 4 for D1 (4th order), per-axis degree <= 5 for D2, <= 5 for KO
    c = {(i, j, k): rng.uniform(-1, 1) for i in range(5) for j in range(5) for k in range(5) if i + j + k <= 4}
    v, (X, Y, Z) = poly_tile(c, h)
    d1, d2, ko = orc.tile_ops(v, h)
    ex = {0: np.zeros_like(X), 1: np.zeros_like(X), 2: np.zeros_like(X)}
    ex2 = {0: np.zeros_like(X), 1: np.zeros_like(X), 2: np.zeros_like(X)}
    for (i, j, k), cv in c.items():
        if i:
            ex[0] += cv * i * X ** (i - 1) * Y ** j * Z ** k
        if j:
            ex[1] += cv * j * X ** i * Y ** (j - 1) * Z ** k
        if k:
            ex[2] += cv * k * X ** i * Y ** j * Z ** (k - 1)
        if i > 1:
            ex2[0] += cv * i * (i - 1) * X ** (i - 2) * Y ** j * Z ** k
        if j > 1:
            ex2[1] += cv * j * (j - 1) * X ** i * Y ** (j - 2) * Z ** k
        if k > 1:
            ex2[2] += cv * k * (k - 1) * X ** i * Y ** j * Z ** (k - 2)
    scale = np.abs(v).max()
    for a in range(3):
        assert np.allclose(d1[a], interior(ex[a]), atol=1e-9 * scale / h, rtol=0)
        assert np.allclose(d2[a], interior(ex2[a]), atol=1e-8 * scale / h ** 2, rtol=0)
        assert np.allclose(ko[a], 0.0, atol=1e-10 * scale)
    # 6th difference of x^6 is 6! h^6 (the leading KO term)
    v6, _ = poly_tile({(6, 0, 0): 1.0}, h)
    _, _, ko6 = orc.tile_ops(v6, h)
    assert np.allclose(ko6[0], 720.0 * h ** 6, rtol=1e-6)
    # fourth-order accuracy of D1 on sin: error ~ h^4 / 30 * |f^(5)|
    vs = np.sin(poly_tile({}, h)[1][0])
    d1s, d2s, _ = orc.tile_ops(vs, h)
    X = poly_tile({}, h)[1][0]
    assert np.abs(d1s[0] - interior(np.cos(X))).max() < h ** 4 / 30 * 1.01
    assert np.abs(d2s[0] + interior(np.sin(X))).max() < h ** 4 / 90 * 1.01


def test_lagrange_interpolation(orc):
    W = orc.interp_weights()
    for r in range(0, 13, 2):
        assert np.array_equal(W[r], np.eye(7)[r // 2])
    xs = np.arange(7.0)
    for deg in range(7):
        vals = xs ** deg
        for r in range(13):
            assert abs(W[r] @ vals - (0.5 * r) ** deg) < 1e-9 * max(1.0, (0.5 * r) ** deg)
    # reflection x -> 6 - x maps the nodes onto themselves and position r / 2 onto
    # (12 - r) / 2: the weights of mirrored positions are reversed copies (the CUDA
    # prolongation evaluates mirrored pairs from symmetric and antisymmetric sums)
    for r in range(13):
        assert np.allclose(W[12 - r], W[r][::-1], rtol=0, atol=1e-15)
    rng = np.random.default_rng(2)
    c = rng.uniform(-1, 1, (4, 4, 4))
    node = np.arange(7.0)
    Zs, Ys, Xs = np.meshgrid(node, node, node, indexing="ij")
    v = sum(c[i, j, k] * Xs ** i * Ys ** j * Zs ** k for i in range(4) for j in range(4) for k in range(4))
    for _ in range(50):
        rx, ry, rz = (int(q) for q in rng.integers(0, 13, 3))
        ex = sum(c[i, j, k] * (rx / 2) ** i * (ry / 2) ** j * (rz / 2) ** k
                 for i in range(4) for j in range(4) for k in range(4))
        assert abs(orc.interp_point(v.reshape(-1), rx, ry, rz) - ex) < 1e-10 * max(1, abs(ex))


@pytest.mark.parametrize("rk", [4, 3])
def test_tableau_order_conditions(orc, rk):
    p, a, w, c = orc.tableau(rk)
    assert p == (4 if rk == 4 else 3)
    assert np.allclose(a.sum(axis=1), c)
    assert abs(w.sum() - 1) < 1e-15
    assert abs(w @ c - 0.5) < 1e-15
    assert abs(w @ c ** 2 - 1 / 3) < 1e-15
    assert abs(w @ a @ c - 1 / 6) < 1e-15
    if rk == 4:
        assert abs(w @ c ** 3 - 1 / 4) < 1e-15
        assert abs(w @ (c * (a @ c)) - 1 / 8) < 1e-15
        assert abs(w @ a @ c ** 2 - 1 / 12) < 1e-15
        assert abs(w @ a @ a @ c - 1 / 24) < 1e-15


def rk_stage_inputs(J, u0, dt, a):
    p = a.shape[0]
    K = []
    U = []
    for s in range(p):
        us = u0 + dt * sum(a[s, j] * K[j] for j in range(s)) if s else u0.copy()
        U.append(us)
        K.append(J @ us)
    return np.array(U), np.array(K)


def expm_nilpotent(J, t):
    n = J.shape[0]
    out = np.eye(n)
    term = np.eye(n)
    for m in range(1, n + 1):
        term = term @ J * t / m
        out = out + term
    return out


@pytest.mark.parametrize("rk", [4, 3])
@pytest.mark.parametrize("theta,rho", [(0.0, 1.0), (0.0, 2.0), (0.0, 0.5), (0.5, 0.5)])
def test_omega_exact_on_nilpotent_system(orc, rk, theta, rho):
    """eqs. fc_1/fc_2: for u' = J u with J^(p+1) = 0 the source's stages determine the
    solution's Taylor polynomial exactly, so the corrected ghost equals the stage
    input the requester computes itself."""
    p, a, w, c = orc.tableau(rk)
    n = p + 1
    J = np.diag(np.ones(n - 1), 1) * 0.7            # nilpotent shift, J^n = 0
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1, 1, n)
    dtN = 0.37
    _, KN = rk_stage_inputs(J, u0, dtN, a)
    om = orc.omega(rk, theta, rho)
    ub = expm_nilpotent(J, theta * dtN) @ u0        # exact solution at the requester's step start
    Ub, _ = rk_stage_inputs(J, ub, rho * dtN, a)    # the requester's own stage inputs
    for s in range(p):
        ghost = u0 + dtN * sum(om[s, j] * KN[j] for j in range(p))
        assert np.allclose(ghost, Ub[s], rtol=0, atol=1e-13), (s, ghost, Ub[s])
    # causality: an active source's stage j >= s is never needed at stage s
    if theta == 0.0:
        assert np.all(np.triu(om) == 0.0)


def test_omega_special_rows(orc):
    p, a, w, c = orc.tableau(4)
    assert np.array_equal(orc.omega(4, 0.0, 1.0), a)            # same level: the tableau itself
    assert np.allclose(orc.omega(4, 1.0, 1.0)[0], w, atol=1e-15)  # theta = 1 shift = RK weights
    om = orc.omega(4, 0.5, 0.5) * 96
    assert np.allclose(om, [[25, 16, 6, 1], [27, 28, 14, 3], [18, 28, 20, 6], [17, 28, 34, 17]], atol=1e-12)
    assert np.allclose(orc.omega(4, 0.0, 2.0), [[0, 0, 0, 0], [1, 0, 0, 0], [-1, 2, 0, 0], [-2, -4, 8, 0]],
                       atol=1e-14)
    assert np.allclose(orc.omega(4, 0.0, 0.5) * 8, [[0, 0, 0, 0], [2, 0, 0, 0], [1, 1, 0, 0], [2, 1, 1, 0]],
                       atol=1e-14)


@pytest.mark.parametrize("rk", [4, 3])
def test_stage_taylor_matches_linear_rk(orc, rk):
    p, a, w, c = orc.tableau(rk)
    g = orc.stage_taylor(rk)
    lam, dt = -0.8, 0.3
    U, _ = rk_stage_inputs(np.array([[lam]]), np.array([1.0]), dt, a)
    for s in range(p):
        val = 1.0 + sum(g[s, m] * (dt * lam) ** (m + 1) for m in range(p))
        assert abs(val - U[s, 0]) < 1e-15


def test_exact_derivatives_against_sympy(orc):
    sp = pytest.importorskip("sympy")
    from paper_2011_10570_gb300 import workloads as W
    x, y, z, t = sp.symbols("x y z t", real=True)
    X = (0.31, -0.17, 0.22)
    cases = []
    w = W.advection_gauss()
    p = w["prob"]["ic_params"]
    a = w["prob"]["adv"]
    cases.append((w["prob"], [sp.exp(-((x - p[0] - a[0] * t) ** 2 + (y - p[1] - a[1] * t) ** 2
                                        + (z - p[2] - a[2] * t) ** 2) / p[3])]))
    w = W.wave_planar()
    s0, wd = w["prob"]["ic_params"][:2]
    f = lambda s: sp.exp(-(s - s0) ** 2 / wd)
    chi = (f(x - t) + f(x + t)) / 2
    cases.append((w["prob"], [chi, sp.diff(chi, t)]))
    w = W.advection_poly(5)
    cc = w["prob"]["ic_params"]
    a = w["prob"]["adv"]
    poly = sum(cc[i + 4 * j + 16 * k] * (x - a[0] * t) ** i * (y - a[1] * t) ** j * (z - a[2] * t) ** k
               for i in range(4) for j in range(4) for k in range(4))
    cases.append((w["prob"], [poly]))
    w = W.wave_poly(7)
    P = w["prob"]["ic_params"][:64]
    Q = w["prob"]["ic_params"][64:128]
    Pp = sum(P[i + 4 * j + 16 * k] * x ** i * y ** j * z ** k for i in range(4) for j in range(4) for k in range(4))
    Qp = sum(Q[i + 4 * j + 16 * k] * x ** i * y ** j * z ** k for i in range(4) for j in range(4) for k in range(4))
    lap = lambda e: sp.diff(e, x, 2) + sp.diff(e, y, 2) + sp.diff(e, z, 2)
    chi = Pp + t * Qp + t ** 2 / 2 * lap(Pp) + t ** 3 / 6 * lap(Qp)
    assert sp.simplify(sp.diff(chi, t, 2) - lap(chi)) == 0          # it solves the wave equation
    cases.append((w["prob"], [chi, sp.diff(chi, t)]))
    w = W.wave_shell(amp=0.0)
    R, wd = w["prob"]["ic_params"][:2]
    r = sp.sqrt(x ** 2 + y ** 2 + z ** 2)
    F = lambda s: s * sp.exp(-(s - R) ** 2 / wd)
    chi = (F(r - t) + F(r + t)) / (2 * r)
    cases.append((w["prob"], [chi, sp.diff(chi, t)]))
    for prob, fields in cases:
        for tt in (0.0, 0.13, 0.4):
            d = orc.exact_derivs(prob, X, tt)
            for fi, e in enumerate(fields):
                for m in range(4):
                    ex = float(sp.diff(e, t, m).subs({x: X[0], y: X[1], z: X[2], t: tt}).evalf(30))
                    assert abs(d[fi, m] - ex) <= 1e-11 * max(1.0, abs(ex)), (prob["ic"], fi, m, d[fi, m], ex)
