"""Defect correction of the FP32 basic scheme (hom_solve_opts.refine): the load cases whose FP32
iteration stalls at its rounding floor are corrected by FP32 solves of the correction's fixed point
driven by FP64 residuals (the oracle's solve_refined_one), so FP32 reaches tolerances the plain FP32
iteration cannot.  Checked against the FP64 oracle run to convergence (the same discrete solution)."""
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


@pytest.mark.parametrize("contrast", [100.0, 0.01])
def test_refined_fp32_reaches_tight_tolerance_2d(contrast):
    """A batch of two hard cells and a mild one (contrast 2, whose FP32 floor is near 5e-8): the plain
    FP32 iteration stalls above the tolerance for the hard ones; with corrections every load case ends
    converged at e_n < 1e-8 (FP64 check), C_eff within 1e-7 of the oracle and fields within 2e-6 of
    the oracle's (FP32 rounding of the FP64-corrected strain)."""
    base = [(H.centred_disk_cell(45, rule=H.RULE_VOIGT), contrast), (H.centred_disk_cell(75, rule=H.RULE_TWO_LAYER), contrast),
            (H.centred_disk_cell(45, rule=H.RULE_REUSS), 2.0)]
    phases, cells = [], []
    for cell, ctr in base:
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(ctr))
    c0 = [H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(len(cells))]
    mat = hom.hom_filter_build(cells, phases)
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, max_iter=5000)
    plain = hom.hom_solve(mat, np.eye(3), c0, tol=1e-8, stall_window=30, **kw)
    assert (plain["status"][:2] == 3).all()
    r = hom.hom_solve(mat, np.eye(3), c0, tol=1e-8, refine=6, **kw)
    assert r["code"] == hom.HOM_OK and (r["status"] == 0).all(), r["status"]
    assert (r["err_n"] < 1e-8).all()
    C = hom.hom_effective_stiffness(np.eye(3), r["mean_sigma"], 2)
    for i in range(3):
        ph = phases[2 * i:2 * i + 2]
        fb = O.filter_build(H.remap_phases(cells[i], -2 * i), ph)
        ref = O.solve(fb["ctilde"], 2, cells[i].n, c0[i][0], c0[i][1], np.eye(3), tol=1e-11, max_iter=40000,
                      criterion=O.CRIT_EN)
        assert _rel(C[i], O.effective_stiffness(ref["mean_sigma"], np.eye(3))) < 1e-7
        eps = cell_fields(r, cells, 2, "eps")[i].astype(np.float64)
        assert _rel(eps, ref["eps"]) < 2e-6


def test_refined_fp32_3d():
    cell = H.rsa_spheres_cell(15, seed=1015, vf=0.15, rmin=0.1, rmax=0.15, subgrid=6, gap_voxels=1.0)
    phases = H.two_phases(100.0)
    c0 = H.mean_lame(phases)
    mat = hom.hom_filter_build([cell], phases)
    r = hom.hom_solve(mat, np.eye(6)[:3], c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-8,
                      max_iter=8000, refine=6)
    assert (r["status"] == 0).all() and (r["err_n"] < 1e-8).all()
    fb = O.filter_build(cell, phases)
    ref = O.solve(fb["ctilde"], 3, 15, c0[0], c0[1], np.eye(6)[:3], tol=1e-11, max_iter=40000, criterion=O.CRIT_EN)
    assert _rel(r["mean_sigma"][0], ref["mean_sigma"]) < 1e-7
