"""Pins for the LTS schedule (Fig. blk_loop) and the speedup model (eqs. w_nuts,
w_uts, invS) against the paper's printed example and brute-force counting."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig_blk_loop.txt")


def read_golden():
    sets, work = {}, {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0].startswith("W_"):
            work[tok[0]] = int(tok[1])
        else:
            sets[int(tok[0])] = sorted(int(v) for v in tok[1:])
    return sets, work


def test_fig_blk_loop_schedule(orc):
    sets, work = read_golden()
    l_min, l_max = 0, 2          # b_4h at level 0, b_2h at 1, b_h at 2
    for n, sizes in sets.items():
        lstar = orc.active_level(l_min, l_max, n)
        active = sorted(2 ** (l_max - l) for l in range(lstar, l_max + 1))
        assert active == sizes
    # block-steps executed in one coarsest step equal W_lts of eq. w_nuts
    steps = sum(len(v) for v in sets.values())
    assert steps == work["W_lts"]


@pytest.mark.parametrize("seed", range(5))
def test_work_model_matches_schedule_count(orc, seed):
    from test_oracle_octree import random_spec
    spec = random_spec(seed, l_min=1, l_max=4 + seed % 2, kind=seed % 2)
    t = orc.Tree.build(spec)
    _, lev = t.export()
    S, wl, wg = t.work_model()
    lmin, lmax = int(lev.min()), int(lev.max())
    L = lmax - lmin
    counts = np.bincount(lev, minlength=lmax + 1)
    # octant-steps executed by the substep schedule of one macro step
    executed = 0
    for n in range(2 ** L):
        lstar = orc.active_level(lmin, lmax, n)
        executed += int(counts[lstar:lmax + 1].sum())
    assert executed == wl
    assert wg == 2 ** L * len(lev)
    assert abs(S - wg / wl) < 1e-12
    assert S < len(lev) / counts[lmax] + 1e-12      # S < |W| / alpha_0 (Sec. 3.7)


def test_work_model_fig_example(orc):
    # eqs. w_nuts / w_uts on alpha = (1, 1, 1), L = 2
    _, work = read_golden()
    alpha = [1, 1, 1]
    L = 2
    assert sum(2 ** (L - l) * a for l, a in enumerate(alpha)) == work["W_lts"]
    assert 2 ** L * sum(alpha) == work["W_gts"]
