"""The C ABI: the library loads, exports every entry point include/ltsoct.h declares,
and rejects an invalid refinement spec before touching a device.  No GPU needed (the
octree build itself runs on the device: tests/test_gpu_octree.py)."""
import os
import re

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
