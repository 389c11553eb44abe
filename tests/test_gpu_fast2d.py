"""GPU tests of the specialised FP32 2D passes: every specialised grid size, ragged row groups and
odd kx counts, output fields, batches with more phases than a one-byte label can name, and
agreement with the generic passes (passes=HOM_PASSES_GENERIC) on the same inputs.

The oracle is the FP64 CPU implementation (FP64, tight tolerance); the FP32 bar is 1e-5 relative
on C_eff, with local-field L2 errors stated."""

import numpy as np
import pytest
import torch

import hom_inputs as H
import oracle as O

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")
from gpu_helpers import cell_fields  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _solve(mat, E, c0, generic=False, **kw):
    passes = hom.HOM_PASSES_GENERIC if generic else hom.HOM_PASSES_AUTO
    return hom.hom_solve(mat, E, c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, passes=passes, **kw)


def _batch(specs):
    phases, cells = [], []
    for cell, contrast in specs:
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(contrast))
    c0 = [H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(len(cells))]
    return cells, phases, c0


# Every specialised size.  Row groups of 4: 45 = 4*11 + 1, 75 = 4*18 + 3, 225 = 4*56 + 1 (ragged
# last group); kx counts (n + 1) / 2: 23 and 113 are odd (last Green tile has one column).
SIZES = [(45, H.RULE_VOIGT, 10.0), (75, H.RULE_TWO_LAYER, 0.1), (135, H.RULE_REUSS, 3.0),
         (225, H.RULE_NONE, 0.2), (405, H.RULE_VOIGT, 5.0)]


def test_every_specialised_size_matches_oracle():
    specs = [(H.centred_disk_cell(n, rule=rule), contrast) for n, rule, contrast in SIZES]
    cells, phases, c0 = _batch(specs)
    E = np.eye(3)
    mat = hom.hom_filter_build(cells, phases)
    res = _solve(mat, E, c0, tol=1e-6, max_iter=3000)
    assert (res["status"] == 0).all()
    eps = cell_fields(res, cells, 2, "eps")
    sig = cell_fields(res, cells, 2, "sigma")
    for i, cell in enumerate(cells):
        fb = O.filter_build(cell, phases)
        ref = O.solve(fb["ctilde"], 2, cell.n, c0[i][0], c0[i][1], E, tol=1e-9, max_iter=3000)
        C = hom.hom_effective_stiffness(E, res["mean_sigma"][i:i + 1], 2)[0]
        Cref = O.effective_stiffness(ref["mean_sigma"], E)
        assert _rel(C, Cref) < 1e-5, (cell.n, _rel(C, Cref))
        # output fields of the specialised output pass: L2 error relative to the field scale
        for got, want in ((eps[i], ref["eps"]), (sig[i], ref["sigma"])):
            d = got - want
            assert np.sqrt(np.mean(d ** 2)) / np.sqrt(np.mean(want ** 2)) < 2e-5, cell.n


def test_specialised_and_generic_passes_agree():
    specs = [(H.centred_disk_cell(n, rule=rule), contrast) for n, rule, contrast in SIZES[:4]]
    cells, phases, c0 = _batch(specs)
    E = np.eye(3)
    mat = hom.hom_filter_build(cells, phases)
    fast = _solve(mat, E, c0, tol=1e-6, max_iter=3000)
    gen = _solve(mat, E, c0, generic=True, tol=1e-6, max_iter=3000)
    assert _rel(fast["mean_sigma"], gen["mean_sigma"]) < 2e-6
    assert np.abs(fast["iterations"].astype(int) - gen["iterations"].astype(int)).max() <= 2
    ef, eg = fast["eps"].cpu().numpy(), gen["eps"].cpu().numpy()
    assert np.sqrt(np.mean((ef - eg) ** 2)) / np.sqrt(np.mean(eg ** 2)) < 1e-5


def test_batch_with_more_phases_than_a_byte():
    """130 cells with their own phase pairs: 260 phases in the table, two per cell."""
    specs = []
    rng = np.random.default_rng(7)
    for i in range(130):
        n = 45 if i % 2 else 75
        contrast = float(10.0 ** rng.uniform(-1.0, 1.0))
        rule = [H.RULE_VOIGT, H.RULE_REUSS, H.RULE_TWO_LAYER][i % 3]
        specs.append((H.centred_disk_cell(n, rule=rule, vf=float(rng.uniform(0.1, 0.3))), contrast))
    cells, phases, c0 = _batch(specs)
    assert len(phases) > 254
    E = np.eye(3)
    mat = hom.hom_filter_build(cells, phases)
    fast = _solve(mat, E, c0, tol=1e-6, max_iter=3000, fields=False)
    gen = _solve(mat, E, c0, generic=True, tol=1e-6, max_iter=3000, fields=False)
    assert (fast["status"] == 0).all()
    assert _rel(fast["mean_sigma"], gen["mean_sigma"]) < 2e-6
    for i in (0, 1, 64, 129):
        fb = O.filter_build(cells[i], phases)
        ref = O.solve(fb["ctilde"], 2, cells[i].n, c0[i][0], c0[i][1], E, tol=1e-9, max_iter=3000)
        C = hom.hom_effective_stiffness(E, fast["mean_sigma"][i:i + 1], 2)[0]
        assert _rel(C, O.effective_stiffness(ref["mean_sigma"], E)) < 1e-5


def test_mixed_batch_falls_back_to_generic_passes():
    """A size without a specialised plan (63) in the batch: every cell runs the generic passes."""
    specs = [(H.centred_disk_cell(45, rule=H.RULE_VOIGT), 10.0), (H.centred_disk_cell(63, rule=H.RULE_REUSS), 0.1)]
    cells, phases, c0 = _batch(specs)
    E = np.eye(3)
    mat = hom.hom_filter_build(cells, phases)
    res = _solve(mat, E, c0, tol=1e-6, max_iter=3000, fields=False)
    for i, cell in enumerate(cells):
        fb = O.filter_build(cell, phases)
        ref = O.solve(fb["ctilde"], 2, cell.n, c0[i][0], c0[i][1], E, tol=1e-9, max_iter=3000)
        C = hom.hom_effective_stiffness(E, res["mean_sigma"][i:i + 1], 2)[0]
        assert _rel(C, O.effective_stiffness(ref["mean_sigma"], E)) < 1e-5
