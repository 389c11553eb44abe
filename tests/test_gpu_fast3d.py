"""GPU tests of the specialised FP32 3D passes: sizes 27 and 45 against the FP64 oracle (C_eff,
output fields), and 81 against the generic 3D passes (passes=HOM_PASSES_GENERIC)."""

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


CASES = [
    # 27 = 3 x 9 (last row group of 3, 14 kx: 7 pairs), 45 = 5 x 9 (last group of 1, 23 kx: odd)
    ("sph27-2layer", lambda: H.rsa_spheres_cell(27, seed=27, vf=0.2, rmin=0.1, rmax=0.15, subgrid=4,
                                                gap_voxels=1.0), 10.0),
    ("sph45-voigt", lambda: H.rsa_spheres_cell(45, seed=45, vf=0.25, rmin=0.1, rmax=0.15, rule=H.RULE_VOIGT,
                                               subgrid=2, gap_voxels=1.0), 0.1),
]


@pytest.mark.parametrize("name,make,contrast", CASES, ids=[c[0] for c in CASES])
def test_specialised_3d_matches_oracle(name, make, contrast):
    cell = make()
    phases = H.two_phases(contrast)
    c0 = [H.mean_lame(phases)]
    E = np.eye(6)
    mat = hom.hom_filter_build([cell], phases)
    res = _solve(mat, E, c0, tol=1e-6, max_iter=3000)
    assert (res["status"] == 0).all()
    fb = O.filter_build(cell, phases)
    ref = O.solve(fb["ctilde"], 3, cell.n, c0[0][0], c0[0][1], E, tol=1e-9, max_iter=3000)
    C = hom.hom_effective_stiffness(E, res["mean_sigma"], 3)[0]
    assert _rel(C, O.effective_stiffness(ref["mean_sigma"], E)) < 1e-5
    eps = cell_fields(res, [cell], 3, "eps")[0]
    sig = cell_fields(res, [cell], 3, "sigma")[0]
    for got, want in ((eps, ref["eps"]), (sig, ref["sigma"])):
        d = got - want
        assert np.sqrt(np.mean(d ** 2)) / np.sqrt(np.mean(want ** 2)) < 2e-5


def test_specialised_and_generic_3d_agree_81():
    cell = H.rsa_spheres_cell(81, seed=1081, vf=0.3, rmin=0.05, rmax=0.1, rule=H.RULE_TWO_LAYER, radius_px=1.0,
                              subgrid=8, gap_voxels=81 / 243.0)
    phases = H.two_phases(10.0)
    c0 = [H.mean_lame(phases)]
    E = np.eye(6)
    mat = hom.hom_filter_build([cell], phases)
    fast = _solve(mat, E, c0, tol=1e-6, max_iter=3000)
    gen = _solve(mat, E, c0, generic=True, tol=1e-6, max_iter=3000)
    assert (fast["status"] == 0).all()
    assert _rel(fast["mean_sigma"], gen["mean_sigma"]) < 2e-6
    assert np.abs(fast["iterations"].astype(int) - gen["iterations"].astype(int)).max() <= 2
    ef, eg = fast["eps"].cpu().numpy(), gen["eps"].cpu().numpy()
    assert np.sqrt(np.mean((ef - eg) ** 2)) / np.sqrt(np.mean(eg ** 2)) < 1e-5
