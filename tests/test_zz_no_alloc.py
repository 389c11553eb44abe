"""hom_solve_noalloc: the fixed-point solve for callers that cannot allocate device memory (a
framework that reserved the GPU's memory for its own allocator, a hard memory budget, or code
that cannot afford the device-wide synchronisation of cudaFree).  It runs the same kernels as
hom_solve (the specialised FP32 passes included) with all scratch in one fixed 64 MiB array inside
the library, so its results must match hom_solve's, call after call, even though every call reuses
the array left by the previous one.

This file is collected last on purpose: a failure here cannot hide the other GPU tests."""
import numpy as np
import pytest
import torch

import hom_inputs as H

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("precision,tol,tol_rel", [(0, 1e-6, 1e-5), (1, 1e-8, 1e-10)], ids=["fp32", "fp64"])
def test_noalloc_matches_hom_solve_on_two_calls(precision, tol, tol_rel):
    """Two hom_solve_noalloc calls in a row agree with hom_solve (uneven two-cell batch; the 27^2
    cell has no specialised plan, so both entry points run the generic passes)."""
    base = [H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER), H.centred_disk_cell(27, rule=H.RULE_VOIGT)]
    phases, cells = [], []
    for cell, contrast in zip(base, (10.0, 0.1)):
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(contrast))
    c0 = [H.mean_lame(phases[0:2]), H.mean_lame(phases[2:4])]
    E = np.eye(3)
    mat = hom.hom_filter_build(cells, phases)
    crit = hom.HOM_CRIT_EN if precision == hom.HOM_FP32 else hom.HOM_CRIT_E
    kw = dict(precision=precision, criterion=crit, tol=tol, max_iter=2000)
    ref = hom.hom_solve(mat, E, c0, **kw)
    assert ref["code"] == hom.HOM_OK
    for _ in range(2):
        got = hom.hom_solve_noalloc(mat, E, c0, **kw)
        assert got["code"] == hom.HOM_OK
        np.testing.assert_array_equal(got["iterations"], ref["iterations"])
        assert _rel(got["mean_sigma"], ref["mean_sigma"]) < tol_rel
        assert _rel(got["eps"].cpu().numpy(), ref["eps"].cpu().numpy()) < tol_rel
        assert _rel(got["sigma"].cpu().numpy(), ref["sigma"].cpu().numpy()) < tol_rel


def test_noalloc_runs_the_specialised_passes():
    """An FP32 batch of specialised sizes only (45^2 and 135^2): hom_solve runs the specialised
    passes, and so must hom_solve_noalloc, with its plan tables in the fixed array.  The same
    kernels on the same inputs give bit-identical results (the reductions have a fixed order), on
    two calls in a row; the generic passes round differently, which shows which kernels ran."""
    base = [H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER), H.centred_disk_cell(135, rule=H.RULE_REUSS)]
    phases, cells = [], []
    for cell, contrast in zip(base, (10.0, 0.1)):
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(contrast))
    c0 = [H.mean_lame(phases[0:2]), H.mean_lame(phases[2:4])]
    E = np.eye(3)
    mat = hom.hom_filter_build(cells, phases)
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-6, max_iter=2000)
    ref = hom.hom_solve(mat, E, c0, **kw)
    gen = hom.hom_solve(mat, E, c0, passes=hom.HOM_PASSES_GENERIC, **kw)
    assert ref["code"] == hom.HOM_OK and gen["code"] == hom.HOM_OK
    assert not np.array_equal(gen["eps"].cpu().numpy(), ref["eps"].cpu().numpy())
    for _ in range(2):
        got = hom.hom_solve_noalloc(mat, E, c0, **kw)
        assert got["code"] == hom.HOM_OK
        np.testing.assert_array_equal(got["iterations"], ref["iterations"])
        np.testing.assert_array_equal(got["mean_sigma"], ref["mean_sigma"])
        np.testing.assert_array_equal(got["eps"].cpu().numpy(), ref["eps"].cpu().numpy())
        np.testing.assert_array_equal(got["sigma"].cpu().numpy(), ref["sigma"].cpu().numpy())


def test_noalloc_rejects_a_batch_beyond_its_scratch():
    """A 1215^2 cell with three loads needs about 195 MB of scratch: refused with a clear error."""
    cells = [H.centred_disk_cell(1215, rule=H.RULE_NONE)]
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build(cells, phases)
    with pytest.raises(hom.HomError) as err:
        hom.hom_solve_noalloc(mat, np.eye(3), H.mean_lame(phases), precision=hom.HOM_FP32, tol=1e-6, max_iter=10)
    assert err.value.code == 2
    assert "scratch" in str(err.value) and "bytes" in str(err.value)


def test_noalloc_refuses_graphs_and_timing():
    cells = [H.centred_disk_cell(15, rule=H.RULE_VOIGT)]
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build(cells, phases)
    for kw in (dict(use_graph=True), dict(stats=True)):
        with pytest.raises(hom.HomError) as err:
            hom.hom_solve_noalloc(mat, np.eye(3), H.mean_lame(phases), precision=hom.HOM_FP64, **kw)
        assert err.value.code == 1
