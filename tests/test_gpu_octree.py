"""The octree build on the device (Sec. 3.2.2 refinement, Sec. 3.2.3 2:1 balance, level
order) and its o2o table (Sec. 3.2.4), bit for bit against the CPU oracle: the
geometric predicates of the workloads (balls, shells, the orbit circle), the wavelet
criterion, random specs, one-octant and deep narrow trees, and the full wave
(154,400 octants) and orbit (492,584 octants) configurations."""
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


def same_tree(lt, orc, spec):
    xa, la = lt.Octree(spec).export()
    xb, lb = orc.Tree.build(spec).export()
    assert len(la) == len(lb)
    assert np.array_equal(la, lb) and np.array_equal(xa, xb)
    return len(la)


@pytest.mark.parametrize("mk", [lambda: W.advection_gauss(), lambda: W.advection_gauss(l_min=2, l_max=4),
                                lambda: W.advection_poly(5), lambda: W.wave_shell(l_min=3, l_max=6, half=10.0),
                                lambda: W.wave_orbit(l_min=2, l_max=6, band=0.3, half=2.0),
                                lambda: W.wavelet_spec(W.advection_gauss(l_min=2, l_max=5), 1e-4),
                                lambda: W.wavelet_spec(W.wave_shell(l_min=2, l_max=5, half=4.0, radius=1.5,
                                                                    width=0.1), 1e-4),
                                lambda: W.uniform(0), lambda: W.uniform(3),
                                lambda: W.advection_gauss(l_min=1, l_max=9, radius=1e-3)])
def test_octree_bit_exact_vs_oracle(lt, orc, mk):
    same_tree(lt, orc, mk()["spec"])


def test_octree_bit_exact_random_specs(lt, orc):
    from test_oracle_octree import random_spec
    for seed in range(16):
        spec = random_spec(seed, l_min=seed % 3, l_max=3 + seed % 4, kind=seed % 2)
        same_tree(lt, orc, spec)


def test_o2o_bit_exact_random_trees(lt, orc):
    from test_oracle_octree import random_spec
    for seed in range(6):
        spec = random_spec(100 + seed, l_min=1, l_max=4, kind=seed % 2)
        w = W.advection_gauss()
        w["spec"] = spec
        plan = lt.Plan(lt.Octree(spec), w["prob"])
        assert np.array_equal(plan.export_o2o(), orc.Tree.build(spec).o2o()), seed


def test_octree_bit_exact_full_configs(lt, orc):
    assert same_tree(lt, orc, W.wave_shell()["spec"]) == 154400
    assert same_tree(lt, orc, W.wave_orbit()["spec"]) == 492584
