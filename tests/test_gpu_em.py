"""GPU tests of the Eyre-Milton scheme (hom_solve with scheme=HOM_SCHEME_EYRE_MILTON) against the
FP64 oracle's solve_em: the same iterate (iteration counts, mean stress, fields, compatibility
error) in FP64 on odd and even grids in 2D and 3D, FP32 to its rounding level, the graph path, a
batch of cells with their own reference media, and the sqrt(contrast) acceleration over the basic
scheme at contrast 1000."""
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


def _em(mat, E, c0, precision=hom.HOM_FP64, **kw):
    return hom.hom_solve(mat, E, c0, precision=precision, criterion=hom.HOM_CRIT_EN,
                         scheme=hom.HOM_SCHEME_EYRE_MILTON, **kw)


CASES = [
    # name, cell, contrast, tol
    ("disk27-2layer-c10", lambda: H.centred_disk_cell(27, rule=H.RULE_TWO_LAYER), 10.0, 1e-10),
    ("disk21-reuss-c1000", lambda: H.centred_disk_cell(21, rule=H.RULE_REUSS), 1e3, 1e-10),
    ("disk16-voigt-c0.01-even", lambda: H.centred_disk_cell(16, rule=H.RULE_VOIGT, radius_px=0.55), 0.01, 1e-10),
    ("sph9-2layer-c100", lambda: H.rsa_spheres_cell(9, seed=9, vf=0.12, rmin=0.12, rmax=0.16, subgrid=4,
                                                    gap_voxels=0.5), 100.0, 1e-10),
    ("sph10-voigt-c10-even", lambda: H.rsa_spheres_cell(10, seed=10, vf=0.2, rmin=0.12, rmax=0.2,
                                                        rule=H.RULE_VOIGT, subgrid=4, gap_voxels=0.5), 10.0, 1e-10),
]


@pytest.mark.parametrize("name,make,contrast,tol", CASES, ids=[c[0] for c in CASES])
def test_em_fp64_matches_oracle(name, make, contrast, tol):
    cell = make()
    dim = cell.dim
    nc = O.nc_of(dim)
    phases = H.two_phases(contrast)
    c0 = H.geometric_lame(phases, dim)
    E = np.eye(nc)
    mat = hom.hom_filter_build([cell], phases)
    res = _em(mat, E, [c0], tol=tol, max_iter=3000)
    fb = O.filter_build(cell, phases)
    ref = O.solve_em(fb["ctilde"], dim, cell.n, c0[0], c0[1], E, tol=tol, max_iter=3000)
    assert all(s == "converged" for s in ref["status"])
    assert (res["status"] == 0).all(), res["status"]
    # the same iterate: equal Green-operator counts (a stop decided within rounding may move one)
    assert np.abs(res["iterations"][0].astype(int) - ref["iterations"]).max() <= 1, (res["iterations"], ref["iterations"])
    C = hom.hom_effective_stiffness(E, res["mean_sigma"], dim)[0]
    Cr = O.effective_stiffness(ref["mean_sigma"], E)
    assert _rel(C, Cr) < 1e-9
    eps = cell_fields(res, [cell], dim, "eps")[0]
    sig = cell_fields(res, [cell], dim, "sigma")[0]
    assert _rel(eps, ref["eps"]) < 1e-8
    assert _rel(sig, ref["sigma"]) < 1e-8
    # reported errors: those of the returned iterate, below tol, matching the oracle's
    for l in range(nc):
        assert res["err_c"][0, l] < tol and res["err_n"][0, l] < tol
        if res["iterations"][0, l] == ref["iterations"][l]:
            assert abs(res["err_c"][0, l] - ref["errors_c"][l][-1]) <= 1e-3 * ref["errors_c"][l][-1] + 1e-15
            assert abs(res["err_n"][0, l] - ref["errors_n"][l][-1]) <= 1e-3 * ref["errors_n"][l][-1] + 1e-15


def test_em_fp32_matches_oracle():
    cell = H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(10.0)
    c0 = H.geometric_lame(phases, 2)
    E = np.eye(3)
    mat = hom.hom_filter_build([cell], phases)
    res = _em(mat, E, [c0], precision=hom.HOM_FP32, tol=1e-5, max_iter=2000)
    assert (res["status"] == 0).all()
    fb = O.filter_build(cell, phases)
    ref = O.solve_em(fb["ctilde"], 2, cell.n, c0[0], c0[1], E, tol=1e-10, max_iter=3000)
    C = hom.hom_effective_stiffness(E, res["mean_sigma"], 2)[0]
    assert _rel(C, O.effective_stiffness(ref["mean_sigma"], E)) < 2e-5
    eps = cell_fields(res, [cell], 2, "eps")[0]
    d = eps - ref["eps"]
    assert np.sqrt(np.mean(d ** 2)) / np.sqrt(np.mean(ref["eps"] ** 2)) < 5e-5
    ref5 = O.solve_em(fb["ctilde"], 2, cell.n, c0[0], c0[1], E, tol=1e-5, max_iter=3000)
    assert np.abs(res["iterations"][0].astype(int) - ref5["iterations"]).max() <= 2


def test_em_graph_equals_host_loop_and_batch():
    """Two cells with their own reference media and three loads: the whole-solve graph gives the
    host loop's result bit for bit, and each cell matches its own oracle solve."""
    cells = [H.centred_disk_cell(15, rule=H.RULE_TWO_LAYER), H.centred_disk_cell(21, rule=H.RULE_REUSS)]
    phases = H.two_phases(50.0)
    c0 = [H.geometric_lame(phases, 2), (1.3, 2.1)]
    E = np.array([[1.0, 0.0, 0.0], [0.2, -0.4, 0.1], [0.0, 0.0, 1.0]])
    mat = hom.hom_filter_build(cells, phases)
    a = _em(mat, E, c0, tol=1e-10, max_iter=4000)
    b = _em(mat, E, c0, tol=1e-10, max_iter=4000, use_graph=True)
    assert (a["status"] == 0).all()
    np.testing.assert_array_equal(a["iterations"], b["iterations"])
    np.testing.assert_array_equal(a["mean_sigma"], b["mean_sigma"])
    assert torch.equal(a["eps"], b["eps"])
    for ci, cell in enumerate(cells):
        fb = O.filter_build(cell, phases)
        ref = O.solve_em(fb["ctilde"], 2, cell.n, c0[ci][0], c0[ci][1], E, tol=1e-10, max_iter=4000)
        assert _rel(a["mean_sigma"][ci], ref["mean_sigma"]) < 1e-9
        assert np.abs(a["iterations"][ci].astype(int) - ref["iterations"]).max() <= 1


def test_em_accelerates_at_high_contrast():
    """Contrast 1000: the Eyre-Milton scheme converges in a small fraction of the basic scheme's
    iterations (sqrt(kappa) against kappa) to the same C_eff."""
    cell = H.centred_disk_cell(63, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(1e3)
    mat = hom.hom_filter_build([cell], phases)
    E = np.eye(3)
    em = _em(mat, E, [H.geometric_lame(phases, 2)], tol=1e-8, max_iter=5000)
    basic = hom.hom_solve(mat, E, [H.mean_lame(phases)], precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN,
                          tol=1e-8, max_iter=40000, fields=False)
    assert (em["status"] == 0).all() and (basic["status"] == 0).all()
    assert em["iterations"].max() * 8 < basic["iterations"].min(), (em["iterations"], basic["iterations"])
    assert _rel(hom.hom_effective_stiffness(E, em["mean_sigma"], 2), hom.hom_effective_stiffness(E, basic["mean_sigma"], 2)) < 1e-6


def test_em_rejects_unsupported_combinations():
    cell = H.centred_disk_cell(15)
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    for kw in (dict(green=hom.HOM_GREEN_ROTATED), dict(refine=2, precision=hom.HOM_FP32)):
        with pytest.raises(hom.HomError) as ei:
            hom.hom_solve(mat, np.eye(3), [H.geometric_lame(phases, 2)], scheme=hom.HOM_SCHEME_EYRE_MILTON,
                          allow_not_converged=True, **kw)
        assert ei.value.code == 9  # HOM_ERR_NOT_IMPL


def test_em_fp32_specialised_passes_match_generic_and_oracle():
    """The specialised FP32 2D passes run the scheme too (a per-phase W for pure voxels, the
    (c~ + c0)^-1 table for mixed ones, u_hat beside the Green tile): a batch of specialised sizes at
    contrasts 100 and 0.01 gives the generic passes' iterate (iteration counts within 2, C_eff and
    fields within FP32 rounding) and the oracle's C_eff."""
    cells = [H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER), H.centred_disk_cell(135, rule=H.RULE_VOIGT),
             H.centred_disk_cell(75, rule=H.RULE_REUSS)]
    contrasts = [100.0, 0.01, 10.0]
    phases, cs = [], []
    for cell, k in zip(cells, contrasts):
        cs.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(k))
    c0 = [H.geometric_lame(phases[2 * i:2 * i + 2], 2) for i in range(len(cs))]
    E = np.eye(3)
    mat = hom.hom_filter_build(cs, phases)
    fast = _em(mat, E, c0, precision=hom.HOM_FP32, tol=1e-6, max_iter=2000)
    gen = _em(mat, E, c0, precision=hom.HOM_FP32, tol=1e-6, max_iter=2000, passes=hom.HOM_PASSES_GENERIC)
    assert (fast["status"] == 0).all() and (gen["status"] == 0).all()
    # FP32 paths that round differently: near the floor (contrast 100) the counts may differ a little
    it_f, it_g = fast["iterations"].astype(int), gen["iterations"].astype(int)
    assert (np.abs(it_f - it_g) <= np.maximum(2, 0.15 * it_g)).all(), (it_f, it_g)
    Cf = hom.hom_effective_stiffness(E, fast["mean_sigma"], 2)
    Cg = hom.hom_effective_stiffness(E, gen["mean_sigma"], 2)
    for i, cell in enumerate(cs):
        assert _rel(Cf[i], Cg[i]) < 2e-6
        ph = phases[2 * i:2 * i + 2]
        fb = O.filter_build(H.remap_phases(cell, -2 * i), ph)
        ref = O.solve_em(fb["ctilde"], 2, cell.n, c0[i][0], c0[i][1], E, tol=1e-10, max_iter=3000)
        assert _rel(Cf[i], O.effective_stiffness(ref["mean_sigma"], E)) < 2e-5
    for key in ("eps", "sigma"):
        for a, b in zip(cell_fields(fast, cs, 2, key), cell_fields(gen, cs, 2, key)):
            assert np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)) < 2e-5


def test_em_fp32_specialised_3d_passes_match_generic_and_oracle():
    """The specialised FP32 3D passes (27^3 and 45^3 sphere cells, contrasts 100 and 0.1): the
    generic passes' iterate and the oracle's C_eff."""
    cells = [H.rsa_spheres_cell(27, seed=27, vf=0.2, rmin=0.1, rmax=0.15, subgrid=4, gap_voxels=1.0),
             H.rsa_spheres_cell(45, seed=45, vf=0.25, rmin=0.1, rmax=0.15, rule=H.RULE_VOIGT, subgrid=2,
                                gap_voxels=1.0)]
    contrasts = [100.0, 0.1]
    phases, cs = [], []
    for cell, k in zip(cells, contrasts):
        cs.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(k))
    c0 = [H.geometric_lame(phases[2 * i:2 * i + 2], 3) for i in range(len(cs))]
    E = np.eye(6)
    mat = hom.hom_filter_build(cs, phases)
    fast = _em(mat, E, c0, precision=hom.HOM_FP32, tol=1e-6, max_iter=2000)
    gen = _em(mat, E, c0, precision=hom.HOM_FP32, tol=1e-6, max_iter=2000, passes=hom.HOM_PASSES_GENERIC)
    assert (fast["status"] == 0).all() and (gen["status"] == 0).all()
    it_f, it_g = fast["iterations"].astype(int), gen["iterations"].astype(int)
    assert (np.abs(it_f - it_g) <= np.maximum(2, 0.15 * it_g)).all(), (it_f, it_g)
    Cf = hom.hom_effective_stiffness(E, fast["mean_sigma"], 3)
    Cg = hom.hom_effective_stiffness(E, gen["mean_sigma"], 3)
    for i, cell in enumerate(cs):
        assert _rel(Cf[i], Cg[i]) < 2e-6
    # the oracle on the 27^3 cell (the 45^3 one is checked through the generic passes)
    fb = O.filter_build(cells[0], phases[0:2])
    ref = O.solve_em(fb["ctilde"], 3, 27, c0[0][0], c0[0][1], E, tol=1e-7, max_iter=3000)
    assert _rel(Cf[0], O.effective_stiffness(ref["mean_sigma"], E)) < 2e-5
    for key in ("eps", "sigma"):
        for a, b in zip(cell_fields(fast, cs, 3, key), cell_fields(gen, cs, 3, key)):
            assert np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)) < 2e-5
