"""GPU parity of the modified discrete Green operator (the rotated finite-difference scheme; the
paper's introduction cites such operators, refs. [1, 11], as the second way to improve the basic
method): hom_solve with green = HOM_GREEN_ROTATED against the FP64 oracle run with the same scheme.

Bars as for the continuous operator: FP64 identical iteration counts and fields within 1e-10 of the
largest magnitude; FP32 C_eff within 1e-5."""
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


CASES = [
    ("disk45-2layer-c10", lambda: H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER), 10.0),
    ("disk27-voigt-c0.1", lambda: H.centred_disk_cell(27, rule=H.RULE_VOIGT), 0.1),
    ("disk16-none-c10", lambda: H.centred_disk_cell(16, rule=H.RULE_NONE), 10.0),
    ("sph15-2layer-c10", lambda: H.rsa_spheres_cell(15, seed=1015, vf=0.15, rmin=0.1, rmax=0.15, subgrid=6,
                                                    gap_voxels=1.0), 10.0),
]


@pytest.mark.parametrize("name,make,contrast", CASES, ids=[c[0] for c in CASES])
def test_rotated_fp64_matches_oracle(name, make, contrast):
    cell = make()
    phases = H.two_phases(contrast)
    c0 = H.mean_lame(phases)
    nc = O.nc_of(cell.dim)
    E = np.eye(nc)[:3]
    mat = hom.hom_filter_build([cell], phases)
    r = hom.hom_solve(mat, E, c0, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=1e-8, max_iter=3000,
                      green=hom.HOM_GREEN_ROTATED)
    assert (r["status"] == 0).all()
    fb = O.filter_build(cell, phases)
    ref = O.solve(fb["ctilde"], cell.dim, cell.n, c0[0], c0[1], E, tol=1e-8, max_iter=3000, criterion=O.CRIT_E,
                  scheme=O.SCHEME_ROTATED)
    np.testing.assert_array_equal(r["iterations"][0], ref["iterations"])
    for key, want in (("eps", ref["eps"]), ("sigma", ref["sigma"])):
        got = cell_fields(r, [cell], cell.dim, key)[0]
        assert float(np.abs(got - want).max() / np.abs(want).max()) < 1e-10
    # the continuous operator gives another discrete solution
    rc = hom.hom_solve(mat, E, c0, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=1e-8, max_iter=3000)
    assert float(np.abs(rc["mean_sigma"] - r["mean_sigma"]).max()) > 1e-6 * float(np.abs(r["mean_sigma"]).max())


def test_rotated_fp32_ceff_and_backward():
    """FP32 (generic passes) within 1e-5 of the oracle's C_eff; the adjoint derivative under the
    rotated operator keeps the energy identity dC_ij/dc~(x) = eps^(i)(x) eps^(j)(x) / N_v (the
    operator is still an orthogonal projection)."""
    cell = H.centred_disk_cell(45, rule=H.RULE_REUSS)
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    mat = hom.hom_filter_build([cell], phases)
    r = hom.hom_solve(mat, np.eye(3), c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-6,
                      max_iter=3000, green=hom.HOM_GREEN_ROTATED)
    assert (r["status"] == 0).all()
    fb = O.filter_build(cell, phases)
    ref = O.solve(fb["ctilde"], 2, 45, c0[0], c0[1], np.eye(3), tol=1e-10, max_iter=3000, scheme=O.SCHEME_ROTATED)
    C = hom.hom_effective_stiffness(np.eye(3), r["mean_sigma"], 2)[0]
    Cr = O.effective_stiffness(ref["mean_sigma"], np.eye(3))
    assert float(np.abs(C - Cr).max() / np.abs(Cr).max()) < 1e-5
    r64 = hom.hom_solve(mat, np.eye(3), c0, precision=hom.HOM_FP64, tol=1e-12, max_iter=3000,
                        green=hom.HOM_GREEN_ROTATED)
    G = np.zeros((1, 3, 3))
    G[0, 0, 1] = 1.0
    b = hom.hom_solve_backward(mat, r64, c0, dL_dC=G, precision=hom.HOM_FP64, green=hom.HOM_GREEN_ROTATED)
    got = b["dctilde"].cpu().numpy().reshape(-1, 6)
    e0 = ref["eps"][0].reshape(3, -1).T
    e1 = ref["eps"][1].reshape(3, -1).T
    A = e0[:, :, None] * e1[:, None, :] / 45 ** 2
    S = A + np.swapaxes(A, -1, -2)
    expect = np.stack([S[:, i, j] * (0.5 if i == j else 1.0) for i in range(3) for j in range(i, 3)], axis=-1)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-8 * np.abs(expect).max())


def test_rotated_rejected_by_cg():
    cell = H.centred_disk_cell(15, rule=H.RULE_VOIGT)
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    with pytest.raises(hom.HomError) as err:
        hom.hom_solve_cg(mat, np.eye(3), precision=hom.HOM_FP64, green=hom.HOM_GREEN_ROTATED)
    assert err.value.code == 9
