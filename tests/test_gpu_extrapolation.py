"""GPU tests of hom_fourier_extrapolate (section 6, Fig. 4) against the oracle: element-by-element
parity in 2D and 3D (fine grids that are and are not multiples of n, several packed components,
a cell that is not the first of its batch), host and device outputs, m = n, argument errors, and the
paper's Fig. 4 statement computed on the GPU path."""
import math

import numpy as np
import pytest
import torch

import hom_inputs as H
import oracle as O

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


def _oracle(cell, phases, comp, m):
    ct = O.filter_build(cell, phases)["ctilde"]
    nc = ct.shape[-1]
    pairs = [(i, j) for i in range(nc) for j in range(i, nc)]
    i, j = pairs[comp]
    return O.fourier_extrapolate(ct[..., i, j], cell.dim, cell.n, m)


def _check(got, want):
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else got
    scale = np.abs(want).max()
    assert np.abs(got - want).max() < 1e-11 * scale, np.abs(got - want).max() / scale


CASES_2D = [
    # (cell, comp, m): m a multiple of n, m not a multiple, m < n, shear and normal components
    (lambda: H.centred_disk_cell(45, rule=H.RULE_VOIGT, radius_px=0.55, radius=math.pi / 15), 0, 135),
    (lambda: H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER, radius_px=1.0), 2, 100),
    (lambda: H.centred_disk_cell(27, rule=H.RULE_REUSS, radius_px=1.5), 1, 20),
    (lambda: H.centred_disk_cell(63, rule=H.RULE_NONE), 5, 189),
]


@pytest.mark.parametrize("k", range(len(CASES_2D)))
def test_2d_matches_oracle(k):
    make, comp, m = CASES_2D[k]
    cell = make()
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    _check(hom.hom_fourier_extrapolate(mat, 0, m, comp), _oracle(cell, phases, comp, m))


def test_3d_matches_oracle():
    cell = H.rsa_spheres_cell(27, seed=27, vf=0.2, rmin=0.1, rmax=0.15, subgrid=4, gap_voxels=1.0)
    phases = H.two_phases(0.1)
    mat = hom.hom_filter_build([cell], phases)
    for comp, m in ((0, 40), (hom.packed_index(3, 3, 3), 27), (hom.packed_index(0, 5, 3), 54)):
        _check(hom.hom_fourier_extrapolate(mat, 0, m, comp), _oracle(cell, phases, comp, m))


def test_later_cell_of_a_batch_and_host_output():
    cells = [H.centred_disk_cell(45, rule=H.RULE_VOIGT), H.centred_disk_cell(75, rule=H.RULE_TWO_LAYER, radius_px=0.55),
             H.centred_disk_cell(27, rule=H.RULE_REUSS)]
    phases = H.two_phases(1e3)
    mat = hom.hom_filter_build(cells, phases)
    want = _oracle(cells[1], phases, 0, 150)
    _check(hom.hom_fourier_extrapolate(mat, 1, 150, 0), want)
    host = torch.empty((150, 150), dtype=torch.float64)
    _check(hom.hom_fourier_extrapolate(mat, 1, 150, 0, out=host), want)
    _check(hom.hom_fourier_extrapolate(mat, 2, 27, 3), _oracle(cells[2], phases, 3, 27))


def test_same_grid_returns_the_filtered_values():
    cell = H.centred_disk_cell(45, rule=H.RULE_VOIGT)
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    ct = O.filter_build(cell, phases)["ctilde"][..., 0, 0]
    _check(hom.hom_fourier_extrapolate(mat, 0, 45, 0), ct)


def test_invalid_arguments_raise():
    cell = H.centred_disk_cell(15, rule=H.RULE_VOIGT)
    mat = hom.hom_filter_build([cell], H.two_phases(10.0))
    for kw in (dict(cell=1, m=15, comp=0), dict(cell=0, m=15, comp=6), dict(cell=0, m=0, comp=0),
               dict(cell=-1, m=15, comp=0)):
        with pytest.raises((hom.HomError, ValueError)):
            hom.hom_fourier_extrapolate(mat, kw["cell"], kw["m"], kw["comp"],
                                        out=torch.empty(max(kw["m"], 1) ** 2, dtype=torch.float64, device="cuda"))


def test_fig4_statement_on_the_gpu_path():
    """Fig. 4 (65^2, disk of radius pi/15, contrast 1e-3, Voigt): overshoot decreases from no filter to
    0.55 to 1.0; the L2 gap to the exact microstructure is smallest at 0.55 of (0.3, 0.55, 1.0, 1.5).
    All five cells in one filter build."""
    n, m = 65, 325
    phases = H.two_phases(1e-3)
    vals = [lam + 2 * mu for lam, mu in phases]
    span = max(vals) - min(vals)
    radii = [0.0, 0.3, 0.55, 1.0, 1.5]
    cells = [H.centred_disk_cell(n, rule=H.RULE_VOIGT if r else H.RULE_NONE, radius_px=r if r else 1.0,
                                 subgrid=16, radius=math.pi / 15) for r in radii]
    mat = hom.hom_filter_build(cells, phases)
    exact = O.exact_property(cells[0], vals, m)
    over, gap = {}, {}
    for i, r in enumerate(radii):
        f = hom.hom_fourier_extrapolate(mat, i, m, 0).cpu().numpy()
        over[r] = max(f.max() - max(vals), min(vals) - f.min()) / span
        gap[r] = np.sqrt(np.mean((f - exact) ** 2)) / span
    assert over[0.0] > 1.5 * over[0.55] and over[0.55] > 2.0 * over[1.0], over
    assert min((0.3, 0.55, 1.0, 1.5), key=lambda r: gap[r]) == 0.55, gap
