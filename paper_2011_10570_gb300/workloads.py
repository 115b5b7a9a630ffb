"""Seeded synthetic workloads: refinement specs, problem parameters and initial data.

This module only describes inputs (plain dictionaries of numbers and seeded
random draws).  It holds none of the method's arithmetic, and it is the one
module that both the library binding and the CPU oracle read, so that both see
exactly the same inputs.

Workloads follow the paper's experiments (Sec. 4.2, Sec. 4.4):
  * ``advection_gauss``  -- 3-D linear advection of a Gaussian, a = (1,1,1)/sqrt(3),
    domain [-1,1]^3, levels 3..5 refined around the pulse, RK4, CFL 0.25.
  * ``wave_shell``       -- scalar wave equation in first-order form (eqs. chi, phi
    with c = 0) on [-10,10]^3, levels 4..9 refined around a Gaussian shell of
    radius 2, radiative outer boundary, seeded 1e-3 amplitude modulation.
  * small variants of both for parity tests, and polynomial data for exactness tests.
"""
from __future__ import annotations

import math

import numpy as np

PDE_ADVECTION, PDE_WAVE = 0, 1
BC_EXACT, BC_RADIATIVE = 0, 1
IC_ADV_GAUSS, IC_ADV_POLY, IC_WAVE_SHELL, IC_WAVE_PLANAR, IC_WAVE_POLY, IC_WAVE_REST = 0, 1, 2, 3, 4, 5
REFINE_BALLS, REFINE_SHELL, REFINE_CIRCLE, REFINE_WAVELET = 0, 1, 2, 3


def advection_gauss(l_min=3, l_max=5, radius=0.3, t_end=0.25, cfl=0.25, ko_sigma=0.1, rk=4, width=0.05):
    """Linear advection u_t + a.grad u = 0 of exp(-|x-x0|^2/w), x0 = (-0.3,-0.3,-0.3)."""
    x0 = (-0.3, -0.3, -0.3)
    spec = dict(lo=-1.0, hi=1.0, l_min=l_min, l_max=l_max, kind=REFINE_BALLS, centers=[x0],
                radius=radius, band=0.0)
    s3 = 1.0 / math.sqrt(3.0)
    prob = dict(pde=PDE_ADVECTION, adv=(s3, s3, s3), cfl=cfl, ko_sigma=ko_sigma, rk=rk,
                bc=BC_EXACT, ic=IC_ADV_GAUSS, ic_params=[x0[0], x0[1], x0[2], width])
    return dict(name="advection_gauss_l%d-%d" % (l_min, l_max), spec=spec, prob=prob, t_end=t_end)


def shell_modes(seed, nmodes=4):
    """Seeded modulation of the shell amplitude: eps_i in [-1,1], integer k_i in [1,3]^3,
    phases theta_i in [0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    modes = []
    for _ in range(nmodes):
        eps = float(rng.uniform(-1.0, 1.0))
        k = [float(v) for v in rng.integers(1, 4, size=3)]
        theta = float(rng.uniform(0.0, 2.0 * math.pi))
        modes.append((eps, k[0], k[1], k[2], theta))
    return modes


def wave_shell(l_min=4, l_max=9, band=0.0, seed=1, amp=1e-3, radius=2.0, width=0.1, t_end=5.0,
               cfl=0.25, ko_sigma=0.1, rk=4, bc=BC_RADIATIVE, half=10.0):
    """Wave equation chi_t = phi, phi_t = lap chi on [-half,half]^3 around a Gaussian shell
    chi_0 = exp(-(r-R)^2/w) (1 + amp sum_i eps_i sin(kscale k_i.x + theta_i)), phi_0 = 0."""
    spec = dict(lo=-half, hi=half, l_min=l_min, l_max=l_max, kind=REFINE_SHELL, centers=[(0.0, 0.0, 0.0)],
                radius=radius, band=band)
    modes = shell_modes(seed) if amp != 0.0 else []
    params = [radius, width, amp, float(len(modes)), math.pi / half]
    for m in modes:
        params.extend(m)
    prob = dict(pde=PDE_WAVE, adv=(0.0, 0.0, 0.0), cfl=cfl, ko_sigma=ko_sigma, rk=rk, bc=bc,
                ic=IC_WAVE_SHELL, ic_params=params)
    return dict(name="wave_shell_l%d-%d" % (l_min, l_max), spec=spec, prob=prob, t_end=t_end)


def wave_nonlinear(l_min=4, l_max=9, c=1.0, **kw):
    """The shell data of ``wave_shell`` evolved with the non-linear source -c sin(2 chi)/r^2
    of eq. phi (the paper's non-linear runs use c = 1)."""
    w = wave_shell(l_min=l_min, l_max=l_max, **kw)
    w["prob"]["nl_c"] = c
    w["name"] = "wave_nonlinear_l%d-%d" % (l_min, l_max)
    return w


def wave_orbit(l_min=3, l_max=12, band=0.042, half=10.0, radius=1.0, omega=0.5, width=0.05, amp=1.0,
               t_end=1.0, cfl=0.25, ko_sigma=0.1, rk=4, precision=1):
    """Wave equation at rest driven by two Gaussian sources on a circular orbit:
    phi_t += amp sum_i exp(-|x - x_i(t)|^2 / width), x_1 = radius (cos omega t, sin omega t, 0),
    x_2 = -x_1, on [-half,half]^3 with levels l_min..l_max refined within `band` of the orbit
    circle, radiative outer boundary, mixed precision by default."""
    spec = dict(lo=-half, hi=half, l_min=l_min, l_max=l_max, kind=REFINE_CIRCLE, centers=[(0.0, 0.0, 0.0)],
                radius=radius, band=band)
    prob = dict(pde=PDE_WAVE, adv=(0.0, 0.0, 0.0), cfl=cfl, ko_sigma=ko_sigma, rk=rk, bc=BC_RADIATIVE,
                ic=IC_WAVE_REST, ic_params=[], orbit=1, orbit_params=[radius, omega, width, amp],
                precision=precision)
    return dict(name="wave_orbit_l%d-%d" % (l_min, l_max), spec=spec, prob=prob, t_end=t_end)


def wavelet_spec(w, eps=1e-5):
    """The refinement of workload `w` replaced by the wavelet criterion of Sec. 3.2.2 on its
    initial pulse: a Gaussian bump (advection) or shell (wave) of the same centre, radius and
    width, refined while a box's largest wavelet coefficient exceeds eps."""
    prob, spec = w["prob"], dict(w["spec"])
    p = prob["ic_params"]
    if prob["ic"] == IC_ADV_GAUSS:
        spec.update(kind=REFINE_WAVELET, centers=[(p[0], p[1], p[2])], radius=0.0, band=p[3], eps=eps)
    elif prob["ic"] == IC_WAVE_SHELL:
        spec.update(kind=REFINE_WAVELET, centers=[spec["centers"][0]], radius=p[0], band=p[1], eps=eps)
    else:
        raise ValueError("wavelet refinement is defined for Gaussian bump or shell data")
    return dict(w, spec=spec, name=w["name"] + "_wavelet")


def random_cubic(seed, scale=1.0):
    """Coefficients c[i + 4j + 16k] of a random polynomial of total degree <= 3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.zeros(64)
    for k in range(4):
        for j in range(4):
            for i in range(4):
                if i + j + k <= 3:
                    c[i + 4 * j + 16 * k] = scale * rng.uniform(-1.0, 1.0)
    return c


def advection_poly(seed, l_min=2, l_max=4, radius=0.35, center=(-0.3, 0.2, 0.1), rk=4, cfl=0.25,
                   ko_sigma=0.1):
    """Advection of a random cubic with exact boundary data (polynomial patch test)."""
    spec = dict(lo=-1.0, hi=1.0, l_min=l_min, l_max=l_max, kind=REFINE_BALLS, centers=[center],
                radius=radius, band=0.0)
    s = (0.6, -0.48, 0.64)
    prob = dict(pde=PDE_ADVECTION, adv=s, cfl=cfl, ko_sigma=ko_sigma, rk=rk, bc=BC_EXACT,
                ic=IC_ADV_POLY, ic_params=list(random_cubic(seed)))
    return dict(name="advection_poly", spec=spec, prob=prob)


def wave_poly(seed, l_min=2, l_max=4, radius=0.35, center=(0.2, -0.1, 0.3), rk=4, cfl=0.25, ko_sigma=0.1):
    """Wave equation with chi = P + tQ + t^2/2 lap P + t^3/6 lap Q (P, Q random cubics)."""
    spec = dict(lo=-1.0, hi=1.0, l_min=l_min, l_max=l_max, kind=REFINE_BALLS, centers=[center],
                radius=radius, band=0.0)
    params = list(random_cubic(seed)) + list(random_cubic(seed + 1000))
    prob = dict(pde=PDE_WAVE, adv=(0.0, 0.0, 0.0), cfl=cfl, ko_sigma=ko_sigma, rk=rk, bc=BC_EXACT,
                ic=IC_WAVE_POLY, ic_params=params)
    return dict(name="wave_poly", spec=spec, prob=prob)


def wave_planar(l_min=2, l_max=4, radius=0.4, s0=0.0, width=0.1, rk=4, cfl=0.25, ko_sigma=0.1):
    """1-D wave chi = (f(x-t)+f(x+t))/2 in 3-D (Sec. 4.3), f Gaussian, exact boundary data."""
    spec = dict(lo=-1.0, hi=1.0, l_min=l_min, l_max=l_max, kind=REFINE_BALLS, centers=[(s0, 0.0, 0.0)],
                radius=radius, band=0.0)
    prob = dict(pde=PDE_WAVE, adv=(0.0, 0.0, 0.0), cfl=cfl, ko_sigma=ko_sigma, rk=rk, bc=BC_EXACT,
                ic=IC_WAVE_PLANAR, ic_params=[s0, width])
    return dict(name="wave_planar", spec=spec, prob=prob)


def uniform(level, pde=PDE_ADVECTION, rk=4):
    """Single-level tree: LTS reduces to GTS (Alg. 2 with one block set)."""
    if pde == PDE_ADVECTION:
        w = advection_gauss(l_min=level, l_max=level, radius=0.0)
    else:
        w = wave_shell(l_min=level, l_max=level, band=0.0, half=4.0, radius=1.5, width=0.2)
    w["spec"]["radius"] = 0.0 if pde == PDE_ADVECTION else w["spec"]["radius"]
    w["prob"]["rk"] = rk
    w["name"] = "uniform_l%d_%s" % (level, "adv" if pde == PDE_ADVECTION else "wave")
    return w


def batch_instances(seed=3, n=64, lmax_range=(6, 11), f_range=(1.0, 20.0)):
    """Independent instances for batching: each is advection of a Gaussian or the 1-D
    wave, on [-1,1]^3 with levels 3..l_max (l_max uniform in lmax_range) refined within
    f finest-octant edges of a random centre (f log-uniform in f_range, which gives
    trees of roughly 1k to 50k octants)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        L = int(rng.integers(lmax_range[0], lmax_range[1] + 1))
        f = float(np.exp(rng.uniform(np.log(f_range[0]), np.log(f_range[1]))))
        c = tuple(float(v) for v in rng.uniform(-0.5, 0.5, 3))
        r = f * 2.0 / 2 ** L
        if rng.uniform() < 0.5:
            w = advection_gauss(l_min=3, l_max=L, radius=r, width=0.02)
            w["spec"]["centers"] = [c]
            w["prob"]["ic_params"] = [c[0], c[1], c[2], 0.02]
        else:
            w = wave_planar(l_min=3, l_max=L, radius=r, s0=c[0], width=0.02)
            w["spec"]["centers"] = [c]
        w["name"] = "batch%02d_%s_l3-%d" % (i, "adv" if w["prob"]["pde"] == PDE_ADVECTION else "wave", L)
        out.append(w)
    return out


def serving_requests(seed=4, n=24, rate=1.0, lmax_choices=(5, 6)):
    """A Poisson stream of wave-equation solves: arrivals with exponential gaps of mean
    1/rate seconds; each a shell of radius R in [2,6] on [-10,10]^3, refined on levels
    3..l_max around a band in [0,5] (about 1k to 200k octants), end time in [0.5, 5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        L = int(rng.choice(lmax_choices))
        R = float(rng.uniform(2.0, 6.0))
        band = float(rng.uniform(0.0, 5.0))
        t_end = float(rng.uniform(0.5, 5.0))
        w = wave_shell(l_min=3, l_max=L, radius=R, band=band, seed=seed * 1000 + i)
        out.append(dict(rid=i, arrival=t, work=dict(spec=w["spec"], prob=w["prob"]), t_end=t_end,
                        name="req%02d_l3-%d" % (i, L)))
    return out
