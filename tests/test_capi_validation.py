"""Host-side option validation of hom_solve through the C ABI, without a GPU: every check below
returns before the library touches a device, so the codes and messages can be read on the CPU."""
import ctypes
import os
import shutil

import numpy as np
import pytest

hom = pytest.importorskip("paper_1412_3228_gb300")

HOM_ERR_INVALID_ARG = 1
HOM_ERR_NOT_IMPL = 9


@pytest.fixture(scope="module")
def L():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    return hom.lib()


def _call(L, **opt):
    cells = hom._marshal_cells([__import__("hom_inputs").centred_disk_cell(15)])
    mat = hom.hom_material()  # not built: the option checks come first
    E = np.eye(3)
    c0 = np.array([[1.0, 1.0]])
    ms = np.zeros((1, 3, 3))
    res = hom.hom_result(mean_sigma=ms.ctypes.data)
    base = dict(precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=1e-6, max_iter=10)
    base.update(opt)
    o = hom.hom_solve_opts(**base)
    code = L.hom_solve(cells.cells, 1, ctypes.byref(mat), E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 3,
                       c0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(o), ctypes.byref(res), None)
    return code, L.hom_last_error().decode()


def test_unknown_scheme_is_invalid(L):
    code, msg = _call(L, scheme=7)
    assert code == HOM_ERR_INVALID_ARG and "scheme" in msg


@pytest.mark.parametrize("opt", [dict(scheme=1, green=1), dict(scheme=1, refine=2, precision=0)])
def test_eyre_milton_combinations_not_implemented(L, opt):
    code, msg = _call(L, **opt)
    assert code == HOM_ERR_NOT_IMPL and "Eyre-Milton" in msg


@pytest.mark.parametrize("opt", [dict(warm_start=1, refine=2, precision=0), dict(warm_start=1, scheme=1)])
def test_warm_start_combinations_not_implemented(L, opt):
    code, msg = _call(L, **opt)
    assert code == HOM_ERR_NOT_IMPL and "warm start" in msg


def test_warm_start_needs_a_device_field(L):
    code, msg = _call(L, warm_start=1)  # out->eps is NULL
    assert code == HOM_ERR_INVALID_ARG and "device memory" in msg


@pytest.mark.parametrize("opt,word", [(dict(passes=5), "passes"), (dict(max_radix=16), "max_radix"),
                                      (dict(green=3), "Green"), (dict(refine=-1), "refine"),
                                      (dict(stall_window=-2), "negative")])
def test_other_options(L, opt, word):
    code, msg = _call(L, **opt)
    assert code == HOM_ERR_INVALID_ARG and word in msg, msg


def test_build_flags_of_the_release_library(L):
    assert L.hom_build_flags() == 0
