"""Pins for the oracle's octree, balance and maps (Sec. 3.2.2-3.2.4, Sec. 3.3).

Every check here is brute force over all leaves on small trees, or an invariant
the paper states (2:1 balance across faces, edges and corners; leaves tile the
domain; the o2o neighbour relation; padding sources coarsest-first)."""
import numpy as np
import pytest

D = 20
ROOT = 1 << D


def py_morton(x, y, z):
    k = 0
    for b in range(21):
        k |= ((x >> b) & 1) << (3 * b)
        k |= ((y >> b) & 1) << (3 * b + 1)
        k |= ((z >> b) & 1) << (3 * b + 2)
    return k


def random_spec(seed, l_min=1, l_max=4, kind=0):
    rng = np.random.default_rng(seed)
    nc = int(rng.integers(1, 4))
    cents = [tuple(float(v) for v in rng.uniform(-0.9, 0.9, 3)) for _ in range(nc)]
    return dict(lo=-1.0, hi=1.0, l_min=l_min, l_max=l_max, kind=kind, centers=cents,
                radius=float(rng.uniform(0.05, 0.4)), band=float(rng.uniform(0.02, 0.1)))


def edges(lev):
    return (ROOT >> lev.astype(np.int64)).astype(np.int64)


def touching_pairs(xyz, lev):
    e = edges(lev)
    lo = xyz.astype(np.int64)
    hi = lo + e[:, None]
    t = np.ones((len(lev), len(lev)), bool)
    for a in range(3):
        t &= (lo[:, None, a] <= hi[None, :, a]) & (lo[None, :, a] <= hi[:, None, a])
    np.fill_diagonal(t, False)
    return t


def test_morton_matches_bit_interleave(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        x, y, z = (int(v) for v in rng.integers(0, ROOT, 3))
        assert orc.morton(x, y, z) == py_morton(x, y, z)
    assert orc.morton(1, 0, 0) == 1 and orc.morton(0, 1, 0) == 2 and orc.morton(0, 0, 1) == 4


@pytest.mark.parametrize("seed", range(6))
def test_tree_tiles_domain_and_is_level_ordered(orc, seed):
    spec = random_spec(seed, kind=seed % 2)
    t = orc.Tree.build(spec)
    xyz, lev = t.export()
    e = edges(lev)
    assert np.all(xyz % e[:, None] == 0)                  # anchors aligned to their size
    assert int((e.astype(object) ** 3).sum()) == ROOT ** 3  # volumes sum to the domain
    keys = [py_morton(*map(int, p)) for p in xyz]
    order = sorted(range(len(lev)), key=lambda i: (lev[i], keys[i]))
    assert order == list(range(len(lev)))                 # (level, Morton) order
    # no overlaps: in Morton order every leaf ends before the next begins
    mo = sorted(range(len(lev)), key=lambda i: keys[i])
    for a, b in zip(mo[:-1], mo[1:]):
        ea = int(e[a]) ** 3
        assert keys[a] + ea <= keys[b]


@pytest.mark.parametrize("seed", range(6))
def test_balance_26_neighbours(orc, seed):
    spec = random_spec(seed, l_max=5 if seed % 2 else 4, kind=seed % 2)
    t = orc.Tree.build(spec)
    xyz, lev = t.export()
    tp = touching_pairs(xyz, lev)
    dl = np.abs(lev[:, None] - lev[None, :])
    assert not np.any(tp & (dl > 1)), "2:1 balance violated"


@pytest.mark.parametrize("seed", range(6))
def test_balance_refines_and_is_minimal(orc, seed):
    spec = random_spec(seed, l_max=5 if seed % 2 else 4, kind=seed % 2)
    ref = orc.Tree.refine_only(spec)
    bal = orc.Tree.build(spec)
    rx, rl = ref.export()
    bx, bl = bal.export()
    # every balanced leaf lies inside a refine-only leaf of level <= its own
    for p, l in zip(bx, bl):
        j = ref.find_leaf(*map(int, p))
        assert rl[j] <= l
    # refine-only leaves that were never split keep their exact box
    # minimality: no complete sibling group could be merged
    e = edges(bl)
    key = {(int(p[0]), int(p[1]), int(p[2]), int(l)) for p, l in zip(bx, bl)}
    parents = {}
    for p, l in zip(bx, bl):
        if l == 0:
            continue
        pe = ROOT >> (int(l) - 1)
        par = (int(p[0]) // pe * pe, int(p[1]) // pe * pe, int(p[2]) // pe * pe, int(l) - 1)
        parents.setdefault(par, 0)
        parents[par] += 1
    lo = bx.astype(np.int64)
    hi = lo + e[:, None]
    for par, cnt in parents.items():
        if cnt != 8:
            continue
        px, py, pz, pl = par
        if pl < spec["l_min"] or (pl < spec["l_max"] and orc.refine_pred(spec, px, py, pz, pl)):
            continue  # refinement forces the split
        pe = ROOT >> pl
        plo = np.array([px, py, pz])
        phi = plo + pe
        touch = np.all((lo <= phi) & (plo <= hi), axis=1)
        inside = np.all((lo >= plo) & (hi <= phi), axis=1)
        forced = np.any(touch & ~inside & (bl > pl + 1))
        assert forced, "sibling group %s could be merged: balance is not minimal" % (par,)


@pytest.mark.parametrize("seed", range(4))
def test_find_leaf_and_o2o_brute_force(orc, seed):
    spec = random_spec(seed, l_max=4, kind=seed % 2)
    t = orc.Tree.build(spec)
    xyz, lev = t.export()
    e = edges(lev)
    lo = xyz.astype(np.int64)
    hi = lo + e[:, None]
    rng = np.random.default_rng(seed)
    for _ in range(300):
        c = rng.integers(0, ROOT, 3)
        inside = np.all((lo <= c) & (c < hi), axis=1)
        assert inside.sum() == 1
        assert t.find_leaf(*map(int, c)) == int(np.argmax(inside))
    o2o = t.o2o()
    for b in range(len(lev)):
        for d in range(27):
            dx, dy, dz = d % 3 - 1, (d // 3) % 3 - 1, d // 9 - 1
            blo = lo[b] + np.array([dx, dy, dz]) * e[b]
            ent = o2o[b, d]
            if np.any(blo < 0) or np.any(blo >= ROOT):
                assert ent[0] == -2
                continue
            bhi = blo + e[b]
            cover = np.all((lo <= blo) & (bhi <= hi), axis=1)      # leaves containing the box
            within = np.all((blo <= lo) & (hi <= bhi), axis=1)     # leaves inside the box
            if cover.any():
                j = int(np.argmax(cover))
                assert ent[0] == j and np.all(ent[1:] == -1)
                assert lev[j] in (lev[b], lev[b] - 1) or d == 13
            else:
                kids = [-1] * 8
                h = e[b] // 2
                for c in range(8):
                    clo = blo + np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1]) * h
                    m = np.where(np.all(lo == clo, axis=1) & (lev == lev[b] + 1))[0]
                    kids[c] = int(m[0]) if len(m) else -1
                assert list(ent) == kids
                assert within.any()


def brute_source(lo6, hi6, P):
    inside = np.all((lo6 <= P) & (P <= hi6), axis=1)
    if not inside.any():
        return -1
    return int(np.argmax(inside))  # smallest level-order index = coarsest, then smallest Morton


@pytest.mark.parametrize("seed", range(4))
def test_padding_and_node_sources_brute_force(orc, seed):
    spec = random_spec(seed + 10, l_max=4, kind=seed % 2)
    t = orc.Tree.build(spec)
    xyz, lev = t.export()
    e = edges(lev)
    lo6 = 6 * xyz.astype(np.int64)
    hi6 = lo6 + 6 * e[:, None]
    rng = np.random.default_rng(seed)
    bs = rng.choice(len(lev), size=min(12, len(lev)), replace=False)
    for b in bs:
        src, r = t.pad_map(int(b))
        for q in range(13 ** 3):
            i, j, k = q % 13 - 3, (q // 13) % 13 - 3, q // 169 - 3
            P = lo6[b] + np.array([i, j, k]) * e[b]
            if 0 <= i <= 6 and 0 <= j <= 6 and 0 <= k <= 6:
                assert src[q] == b
                continue
            s = brute_source(lo6, hi6, P)
            assert src[q] == s
            if s >= 0:
                rr = 2 * (P - lo6[s]) // e[s]
                assert np.all(2 * (P - lo6[s]) % e[s] == 0)
                assert np.all(r[q] == rr)
                assert abs(int(lev[s]) - int(lev[b])) <= 1
                if lev[s] >= lev[b]:
                    assert np.all(r[q] % 2 == 0)   # same level and finer sources are copies
        nsrc, nr = t.node_map(int(b))
        for n in range(343):
            i, j, k = n % 7, (n // 7) % 7, n // 49
            P = lo6[b] + np.array([i, j, k]) * e[b]
            s = brute_source(lo6, hi6, P)
            assert nsrc[n] == s
            assert np.all(nr[n] == 2 * (P - lo6[s]) // e[s])
            if 1 <= i <= 5 and 1 <= j <= 5 and 1 <= k <= 5:
                assert s == b


def test_refine_predicate_semantics(orc):
    # balls: an octant is refined iff its box comes within `radius` of a center
    spec = dict(lo=-1.0, hi=1.0, l_min=0, l_max=6, kind=0, centers=[(0.0, 0.0, 0.0)], radius=0.1, band=0.0)
    half = ROOT // 2
    assert orc.refine_pred(spec, 0, 0, 0, 1)                     # touches the centre
    e3 = ROOT >> 3
    # box [0.75, 1]^3 in physical units is far from the centre
    assert not orc.refine_pred(spec, 7 * e3, 7 * e3, 7 * e3, 3)
    # a box whose nearest corner is at distance 0.0625*sqrt(3) ~ 0.108 > 0.1
    e5 = ROOT >> 5
    assert not orc.refine_pred(spec, half + e5, half + e5, half + e5, 5)
    # nearest face at distance 0.0625 < 0.1
    assert orc.refine_pred(spec, half + e5, half, half, 5)
    # shell: |x| in [R - band, R + band]
    sh = dict(spec, kind=1, radius=0.5, band=0.01)
    assert not orc.refine_pred(sh, half, half, half, 6)          # box at the centre (inside the shell)
    e6 = ROOT >> 6
    # box [0.5, 0.53125] x [0, 0.03125]^2 straddles r = 0.5
    assert orc.refine_pred(sh, half + 16 * e6, half, half, 6)
