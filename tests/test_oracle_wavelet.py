"""Pins for the oracle's wavelet refinement criterion (Sec. 3.2.2: the wavelet coefficient
measures how badly the field is interpolated from the coarser level).

* the coefficient of a box equals an independent numpy evaluation: the field on the
  13^3 half-node grid, minus its degree-6 tensor Lagrange interpolant from the 7^3 nodes
  (basis polynomials built here with numpy), maximised over the odd points;
* it decays like h^7 (a degree-6 interpolant) under refinement of a smooth field;
* the tree it builds refines around the pulse only, and every leaf coarser than l_max
  has its coefficient at or below the tolerance.
"""
import numpy as np

from paper_2011_10570_gb300 import workloads as W

ROOT = 1 << 20


def field(spec, x):
    f = np.zeros(x.shape[:-1])
    for c in spec["centers"]:
        r = np.sqrt(((x - np.asarray(c)) ** 2).sum(axis=-1)) - spec["radius"]
        f += np.exp(-r * r / spec["band"])
    return f


def lagrange_matrix():
    """M[k, j] = L_j(k / 2), L_j the Lagrange basis polynomial of the nodes 0..6"""
    nodes = np.arange(7.0)
    M = np.zeros((13, 7))
    for j in range(7):
        others = np.delete(nodes, j)
        coef = np.poly(others) / np.prod(j - others)
        M[:, j] = np.polyval(coef, np.arange(13) / 2.0)
    return M


def numpy_coeff(spec, anchor, level):
    e = ROOT >> level
    k = np.arange(13)
    P = [6 * a + k * (e // 2) for a in anchor]
    g = [spec["lo"] + (spec["hi"] - spec["lo"]) * (p / (6.0 * ROOT)) for p in P]
    X = np.stack(np.meshgrid(g[0], g[1], g[2], indexing="ij"), axis=-1)    # [kx][ky][kz]
    F = field(spec, X)
    M = lagrange_matrix()
    I = np.einsum("ai,bj,ck,ijk->abc", M, M, M, F[::2, ::2, ::2])
    odd = (k[:, None, None] % 2) | (k[None, :, None] % 2) | (k[None, None, :] % 2)
    return np.abs(F - I)[odd.astype(bool)].max()


def test_coefficient_matches_numpy(orc):
    rng = np.random.default_rng(5)
    for w in (W.wavelet_spec(W.advection_gauss(l_min=2, l_max=6)),
              W.wavelet_spec(W.wave_shell(l_min=3, l_max=6, half=4.0, radius=1.5, width=0.2))):
        spec = w["spec"]
        for _ in range(12):
            level = int(rng.integers(2, 7))
            e = ROOT >> level
            a = [int(v) * e for v in rng.integers(0, ROOT // e, 3)]
            ours = orc.wavelet_coeff(spec, a[0], a[1], a[2], level)
            ref = numpy_coeff(spec, a, level)
            assert abs(ours - ref) <= 1e-9 * max(ref, 1e-6), (level, a, ours, ref)


def test_coefficient_decays_like_h7(orc):
    spec = W.wavelet_spec(W.advection_gauss(l_min=2, l_max=8))["spec"]
    x0 = np.array(spec["centers"][0])
    c = (x0 - spec["lo"]) / (spec["hi"] - spec["lo"]) * ROOT
    maxima = []
    for level in (3, 4, 5):
        e = ROOT >> level
        # every box of this level within 0.25 of the bump centre
        lo = np.floor((c - 0.125 * ROOT) / e).astype(int)
        hi = np.floor((c + 0.125 * ROOT) / e).astype(int)
        m = 0.0
        for i in range(lo[0], hi[0] + 1):
            for j in range(lo[1], hi[1] + 1):
                for k in range(lo[2], hi[2] + 1):
                    m = max(m, orc.wavelet_coeff(spec, i * e, j * e, k * e, level))
        maxima.append(m)
    for a, b in zip(maxima[:-1], maxima[1:]):
        assert 2.0 ** 5.5 < a / b < 2.0 ** 8.5, maxima


def test_wavelet_tree(orc):
    w = W.wavelet_spec(W.wave_shell(l_min=3, l_max=6, half=4.0, radius=1.5, width=0.2), eps=1e-7)
    spec = w["spec"]
    t = orc.Tree.build(spec)
    xyz, lev = t.export()
    assert lev.max() == 6 and lev.min() == 3
    # refined around the shell |x| = 1.5, coarse far from it
    e = (ROOT >> lev).astype(float)
    ctr = spec["lo"] + (spec["hi"] - spec["lo"]) * (xyz + e[:, None] / 2) / ROOT
    r = np.sqrt((ctr ** 2).sum(axis=1))
    assert np.abs(r[lev == 6] - 1.5).max() < 2.0
    assert (lev[np.abs(r - 1.5) > 3.0] == 3).all() and (np.abs(r - 1.5) > 3.0).any()
    for q in np.flatnonzero(lev < spec["l_max"])[::17]:
        assert orc.wavelet_coeff(spec, *[int(v) for v in xyz[q]], int(lev[q])) <= spec["eps"]
