"""The C ABI: the library loads, exports every entry point include/ltsoct.h
declares, and its host-side octree construction (Sec. 3.2.2-3.2.3) matches the
oracle bit for bit.  No GPU needed."""
import os
import re

import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lt():
    from paper_2011_10570_gb300 import build, ltsoct
    build.build()
    ltsoct.load()
    return ltsoct


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(", txt, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(lt):
    import ctypes
    names = declared_functions()
    assert {"octree_build", "lts_plan_create", "lts_advance", "gts_advance", "lts_run_substeps"} <= names
    lib = ctypes.CDLL(lt.library_path())
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(lt.EXPORTS) <= names


def test_error_reporting_without_gpu(lt):
    bad = dict(W.advection_gauss()["spec"], l_max=1, l_min=3)
    with pytest.raises(lt.LtsError) as ei:
        lt.Octree(bad)
    assert ei.value.status == 1 and "octree_build" in str(ei.value)
    assert lt.load().lts_strerror(5).decode() == "octree is not 2:1 balanced"


@pytest.mark.parametrize("mk", [lambda: W.advection_gauss(), lambda: W.advection_gauss(l_min=2, l_max=4),
                                lambda: W.advection_poly(5), lambda: W.wave_shell(l_min=3, l_max=6, half=10.0)])
def test_octree_bit_exact_vs_oracle(lt, orc, mk):
    w = mk()
    a = lt.Octree(w["spec"])
    b = orc.Tree.build(w["spec"])
    xa, la = a.export()
    xb, lb = b.export()
    assert np.array_equal(la, lb) and np.array_equal(xa, xb)


def test_octree_bit_exact_random_specs(lt, orc):
    from test_oracle_octree import random_spec
    for seed in range(12):
        spec = random_spec(seed, l_min=seed % 3, l_max=3 + seed % 4, kind=seed % 2)
        xa, la = lt.Octree(spec).export()
        xb, lb = orc.Tree.build(spec).export()
        assert np.array_equal(la, lb) and np.array_equal(xa, xb), seed


@pytest.mark.slow
def test_octree_bit_exact_full_wave_config(lt, orc):
    w = W.wave_shell()
    xa, la = lt.Octree(w["spec"]).export()
    xb, lb = orc.Tree.build(w["spec"]).export()
    assert len(la) == 154400
    assert np.array_equal(la, lb) and np.array_equal(xa, xb)
