"""The C-ABI library builds, loads without a GPU and exports every function of include/hom.h."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "hom.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(hom_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1412_3228_gb300 import _build_lib
    return _build_lib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["hom_filter_build", "hom_solve", "hom_effective_stiffness"]:
        assert f in names, names


def test_library_exports_every_declared_function(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (hom_\w+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    import paper_1412_3228_gb300 as hom
    L = hom.lib()
    assert L.hom_version() >= 100
    for f in declared_functions():
        assert hasattr(L, f)
    assert set(hom.EXPORTED) <= set(declared_functions())
