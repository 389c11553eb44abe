"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars: filter counts bit-exact, filtered stiffness within 1e-12 relative (FP64, different
formulas on each side for the 2-layer rule); FP64 solves within 1e-10 relative on C_eff and on
the local fields with identical iteration counts; FP32 solves within 1e-5 relative on C_eff."""
import math

import numpy as np
import pytest
import torch

import hom_inputs as H
import oracle as O

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")
from gpu_helpers import cell_fields, dense_ctilde, unpack  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


FILTER_CASES = [
    ("disk45-voigt", lambda: H.centred_disk_cell(45, rule=H.RULE_VOIGT), 10.0),
    ("disk45-reuss", lambda: H.centred_disk_cell(45, rule=H.RULE_REUSS), 0.1),
    ("disk45-2layer", lambda: H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER, radius_px=0.55), 10.0),
    ("disk45-none", lambda: H.centred_disk_cell(45, rule=H.RULE_NONE), 10.0),
    ("disk25-tie", lambda: H.centred_disk_cell(25, radius=0.2, rule=H.RULE_VOIGT, subgrid=5), 10.0),
    ("slab27-2layer", lambda: H.laminate_cell(27, 2, 0.37, axis=1, centre=0.43, rule=H.RULE_TWO_LAYER,
                                              subgrid=8), 0.1),
    ("sph15-2layer", lambda: H.rsa_spheres_cell(15, seed=1015, vf=0.15, rmin=0.1, rmax=0.15, subgrid=6, gap_voxels=1.0), 10.0),
    ("sph9-reuss", lambda: H.rsa_spheres_cell(9, seed=9, vf=0.15, rmin=0.12, rmax=0.18, rule=H.RULE_REUSS,
                                              subgrid=4, gap_voxels=1.0), 0.1),
    # disk across the periodic boundary (wrapped offsets)
    ("wrap-disk-2layer", lambda: H.Cell(2, 45, 0, [H.Primitive(H.PRIM_DISK, 1, (0.02, 0.97, 0.0), 0.3)],
                                        H.RULE_TWO_LAYER, 1.0, 16), 10.0),
    # overlapping disks of one phase: the owner of a sample is the first primitive containing it,
    # the 2-layer normal comes from the nearest surface, whichever primitive holds it
    ("overlap-2layer", lambda: H.Cell(2, 45, 0, [H.Primitive(H.PRIM_DISK, 1, (0.45, 0.5, 0.0), 0.2),
                                                 H.Primitive(H.PRIM_DISK, 1, (0.62, 0.52, 0.0), 0.15)],
                                      H.RULE_TWO_LAYER, 1.5, 8), 10.0),
    # many disks, larger filter radius and a coarse subgrid
    ("rdisks-voigt", lambda: H.random_disk_cell(7, sizes=(75,), kmin=30, kmax=30, radius_px=1.3, subgrid=7)[0], 0.1),
    ("sph21-voigt", lambda: H.rsa_spheres_cell(21, seed=21, vf=0.3, rmin=0.12, rmax=0.16, rule=H.RULE_VOIGT,
                                               subgrid=6, gap_voxels=0.1), 10.0),
]


@pytest.mark.parametrize("name,make,contrast", FILTER_CASES, ids=[c[0] for c in FILTER_CASES])
def test_filter_build_parity(name, make, contrast):
    cell = make()
    phases = H.two_phases(contrast)
    mat = hom.hom_filter_build([cell], phases)
    fb = O.filter_build(cell, phases)
    dim = cell.dim
    nc = O.nc_of(dim)
    got, mixed = dense_ctilde(mat, 0)
    ref = fb["ctilde"].reshape(-1, nc, nc)
    np.testing.assert_array_equal(mixed, fb["mixed"].ravel())
    assert _rel(unpack(got, nc), ref) < 1e-12
    # pure voxels carry the phase stiffness itself (the oracle forms shear terms as sqrt2*sqrt2*mu,
    # one rounding away from 2 mu)
    pure = ~mixed
    np.testing.assert_allclose(unpack(got, nc)[pure], ref[pure], rtol=4e-16, atol=0)
    if cell.rule != H.RULE_NONE and mat.mixed_count:
        # volume fractions are exact sample counts
        vox = mat.mixed_voxel[:mat.mixed_count].cpu().numpy()
        frac = mat.mixed_frac[:mat.mixed_count].cpu().numpy()
        ph = mat.mixed_phases[:2 * mat.mixed_count].cpu().numpy().reshape(-1, 2)
        counts = fb["counts"].reshape(-1, len(phases))
        np.testing.assert_array_equal(frac, counts[vox, ph[:, 1]] / fb["M"])
    # FP32 copy is the rounded FP64 value
    got32, _ = dense_ctilde(mat, 0, fp64=False)
    np.testing.assert_array_equal(got32, got.astype(np.float32))


def test_filter_build_three_phases():
    """Overlapping disks of two inclusion phases: counts per phase and the Voigt/Reuss averages of
    three phases match the oracle."""
    cell = H.Cell(2, 35, 0, [H.Primitive(H.PRIM_DISK, 1, (0.45, 0.5, 0.0), 0.2),
                             H.Primitive(H.PRIM_DISK, 2, (0.6, 0.55, 0.0), 0.15)], H.RULE_REUSS, 1.2, 12)
    phases = H.two_phases(10.0) + [H.lame_from_young(0.3, 0.3)]
    for rule in (H.RULE_VOIGT, H.RULE_REUSS):
        cell.rule = rule
        mat = hom.hom_filter_build([cell], phases)
        fb = O.filter_build(cell, phases)
        got, mixed = dense_ctilde(mat, 0)
        np.testing.assert_array_equal(mixed, fb["mixed"].ravel())
        assert _rel(unpack(got, 3), fb["ctilde"].reshape(-1, 3, 3)) < 1e-12


def _solve_both(cells, phases, E, precision, criterion, tol, max_iter=2000, c0=None):
    mat = hom.hom_filter_build(cells, phases)
    if c0 is None:
        c0 = [H.mean_lame(phases)] * len(cells)
    res = hom.hom_solve(mat, E, c0, precision=precision, criterion=criterion, tol=tol, max_iter=max_iter)
    refs = []
    for i, cell in enumerate(cells):
        fb = O.filter_build(cell, phases)
        refs.append(O.solve(fb["ctilde"], cell.dim, cell.n, c0[i][0], c0[i][1], np.asarray(E), tol=tol,
                            max_iter=max_iter, criterion=criterion))
    return mat, res, refs


SOLVE_FP64 = [
    ("disk45-voigt-c10", [lambda: H.centred_disk_cell(45, rule=H.RULE_VOIGT)], 10.0),
    ("disk45-2layer-c0.1", [lambda: H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER)], 0.1),
    ("disk27-none-c10", [lambda: H.centred_disk_cell(27, rule=H.RULE_NONE)], 10.0),
    ("disk75-reuss-c10", [lambda: H.centred_disk_cell(75, rule=H.RULE_REUSS)], 10.0),
]


@pytest.mark.parametrize("name,makers,contrast", SOLVE_FP64, ids=[c[0] for c in SOLVE_FP64])
def test_solve_fp64_2d_parity(name, makers, contrast):
    cells = [m() for m in makers]
    phases = H.two_phases(contrast)
    E = np.eye(3)
    mat, res, refs = _solve_both(cells, phases, E, hom.HOM_FP64, hom.HOM_CRIT_E, 1e-8)
    eps = cell_fields(res, cells, 2, "eps")
    sig = cell_fields(res, cells, 2, "sigma")
    for i, ref in enumerate(refs):
        assert list(res["iterations"][i]) == list(ref["iterations"])
        assert all(s == 0 for s in res["status"][i])
        C = hom.hom_effective_stiffness(E, res["mean_sigma"][i:i + 1], 2)[0]
        Cref = O.effective_stiffness(ref["mean_sigma"], E)
        assert _rel(C, Cref) < 1e-10
        assert _rel(eps[i], ref["eps"]) < 1e-10
        assert _rel(sig[i], ref["sigma"]) < 1e-10
        for l in range(3):
            assert abs(res["err"][i, l] - ref["errors"][l][-1]) < 1e-6 * ref["errors"][l][-1] + 1e-14


def test_solve_fp64_3d_parity():
    cell = H.rsa_spheres_cell(15, seed=1015, vf=0.15, rmin=0.1, rmax=0.15, subgrid=6, gap_voxels=1.0)
    phases = H.two_phases(10.0)
    E = np.eye(6)
    mat, res, refs = _solve_both([cell], phases, E, hom.HOM_FP64, hom.HOM_CRIT_E, 1e-8)
    ref = refs[0]
    assert list(res["iterations"][0]) == list(ref["iterations"])
    C = hom.hom_effective_stiffness(E, res["mean_sigma"], 3)[0]
    Cref = O.effective_stiffness(ref["mean_sigma"], E)
    assert _rel(C, Cref) < 1e-10
    assert _rel(cell_fields(res, [cell], 3, "eps")[0], ref["eps"]) < 1e-10
    assert _rel(cell_fields(res, [cell], 3, "sigma")[0], ref["sigma"]) < 1e-10


def test_solve_fp32_2d_parity():
    cells = [H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER), H.centred_disk_cell(45, rule=H.RULE_VOIGT)]
    phases = H.two_phases(10.0)
    E = np.eye(3)
    mat, res, refs = _solve_both(cells, phases, E, hom.HOM_FP32, hom.HOM_CRIT_EN, 1e-6)
    eps = cell_fields(res, cells, 2, "eps")
    for i, ref in enumerate(refs):
        C = hom.hom_effective_stiffness(E, res["mean_sigma"][i:i + 1], 2)[0]
        Cref = O.effective_stiffness(ref["mean_sigma"], E)
        assert _rel(C, Cref) < 1e-5
        assert all(abs(int(a) - int(b)) <= 2 for a, b in zip(res["iterations"][i], ref["iterations"]))
        # local fields: L2 and max errors relative to the field scale
        d = eps[i] - ref["eps"]
        assert np.sqrt(np.mean(d ** 2)) / np.sqrt(np.mean(ref["eps"] ** 2)) < 1e-5
        assert _rel(eps[i], ref["eps"]) < 1e-4


def test_solve_fp32_3d_parity():
    cell = H.rsa_spheres_cell(15, seed=1015, vf=0.15, rmin=0.1, rmax=0.15, subgrid=6, gap_voxels=1.0)
    phases = H.two_phases(0.1)
    E = np.eye(6)
    mat, res, refs = _solve_both([cell], phases, E, hom.HOM_FP32, hom.HOM_CRIT_EN, 1e-6)
    C = hom.hom_effective_stiffness(E, res["mean_sigma"], 3)[0]
    Cref = O.effective_stiffness(refs[0]["mean_sigma"], E)
    assert _rel(C, Cref) < 1e-5


def test_radix_11_and_13_grids():
    """Grids with prime factors 11 and 13 (11, 13, 65 = 5 x 13 -- the paper's 65-pixel cell of
    sections 4 to 6 -- and 143 = 11 x 13) in one batch, FP64 against the oracle (identical iteration
    counts, 1e-10 on C_eff and fields), then FP32 within 1e-5; and a 3D 39 = 3 x 13 cell."""
    cells = [H.centred_disk_cell(n, rule=rule, radius=math.pi / 15)
             for n, rule in ((11, H.RULE_VOIGT), (13, H.RULE_NONE), (65, H.RULE_TWO_LAYER), (143, H.RULE_REUSS))]
    phases = H.two_phases(10.0)
    E = np.eye(3)
    mat, res, refs = _solve_both(cells, phases, E, hom.HOM_FP64, hom.HOM_CRIT_E, 1e-8)
    eps = cell_fields(res, cells, 2, "eps")
    for i, ref in enumerate(refs):
        assert list(res["iterations"][i]) == list(ref["iterations"]), cells[i].n
        C = hom.hom_effective_stiffness(E, res["mean_sigma"][i:i + 1], 2)[0]
        assert _rel(C, O.effective_stiffness(ref["mean_sigma"], E)) < 1e-10
        assert _rel(eps[i], ref["eps"]) < 1e-10
    res32 = hom.hom_solve(mat, E, [H.mean_lame(phases)] * len(cells), precision=hom.HOM_FP32,
                          criterion=hom.HOM_CRIT_EN, tol=1e-6, max_iter=3000, fields=False)
    for i, cell in enumerate(cells):
        ref = O.solve(O.filter_build(cell, phases)["ctilde"], 2, cell.n, *H.mean_lame(phases), E, tol=1e-9,
                      max_iter=3000)
        C = hom.hom_effective_stiffness(E, res32["mean_sigma"][i:i + 1], 2)[0]
        assert _rel(C, O.effective_stiffness(ref["mean_sigma"], E)) < 1e-5, cell.n
    cell = H.rsa_spheres_cell(39, seed=39, vf=0.2, rmin=0.1, rmax=0.15, subgrid=4, gap_voxels=1.0)
    E = np.eye(6)[:2]
    mat, res, refs = _solve_both([cell], phases, E, hom.HOM_FP64, hom.HOM_CRIT_E, 1e-8)
    assert list(res["iterations"][0]) == list(refs[0]["iterations"])
    assert _rel(res["mean_sigma"][0], refs[0]["mean_sigma"]) < 1e-10
    assert _rel(cell_fields(res, [cell], 3, "eps")[0], refs[0]["eps"]) < 1e-10


def test_even_grids():
    """Even grids (Nyquist convention: zero strain at wave vectors with a Nyquist component, left out
    of e and e_n): 16, 30, 64 and 128 in one batch, FP64 against the oracle (identical iteration
    counts, 1e-10 on C_eff and fields), FP32 within 1e-5, conjugate gradients, and a 3D 16^3 cell."""
    cells = [H.centred_disk_cell(n, rule=rule, radius=math.pi / 15)
             for n, rule in ((16, H.RULE_VOIGT), (30, H.RULE_NONE), (64, H.RULE_TWO_LAYER), (128, H.RULE_REUSS))]
    phases = H.two_phases(10.0)
    E = np.eye(3)
    mat, res, refs = _solve_both(cells, phases, E, hom.HOM_FP64, hom.HOM_CRIT_E, 1e-8)
    eps = cell_fields(res, cells, 2, "eps")
    for i, ref in enumerate(refs):
        assert list(res["iterations"][i]) == list(ref["iterations"]), cells[i].n
        C = hom.hom_effective_stiffness(E, res["mean_sigma"][i:i + 1], 2)[0]
        assert _rel(C, O.effective_stiffness(ref["mean_sigma"], E)) < 1e-10
        assert _rel(eps[i], ref["eps"]) < 1e-10
    c0 = [H.mean_lame(phases)] * len(cells)
    res32 = hom.hom_solve(mat, E, c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-6, max_iter=3000,
                          fields=False)
    cg = hom.hom_solve_cg(mat, E, precision=hom.HOM_FP64, tol=1e-10, max_iter=3000, fields=False)
    for i, cell in enumerate(cells):
        ct = O.filter_build(cell, phases)["ctilde"]
        ref = O.solve(ct, 2, cell.n, *H.mean_lame(phases), E, tol=1e-10, max_iter=3000)
        Cref = O.effective_stiffness(ref["mean_sigma"], E)
        C = hom.hom_effective_stiffness(E, res32["mean_sigma"][i:i + 1], 2)[0]
        assert _rel(C, Cref) < 1e-5, cell.n
        Ccg = hom.hom_effective_stiffness(E, cg["mean_sigma"][i:i + 1], 2)[0]
        assert _rel(Ccg, Cref) < 1e-9, cell.n
    cell = H.rsa_spheres_cell(16, seed=16, vf=0.15, rmin=0.1, rmax=0.15, subgrid=4, gap_voxels=1.0)
    E = np.eye(6)[:2]
    mat, res, refs = _solve_both([cell], phases, E, hom.HOM_FP64, hom.HOM_CRIT_E, 1e-8)
    assert list(res["iterations"][0]) == list(refs[0]["iterations"])
    assert _rel(res["mean_sigma"][0], refs[0]["mean_sigma"]) < 1e-10
    assert _rel(cell_fields(res, [cell], 3, "eps")[0], refs[0]["eps"]) < 1e-10


def test_uneven_batch_matches_per_cell_oracle():
    """Cells of different sizes, rules and contrasts in one launch sequence."""
    base = [H.centred_disk_cell(15, rule=H.RULE_VOIGT), H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER),
            H.centred_disk_cell(27, rule=H.RULE_REUSS), H.centred_disk_cell(5, rule=H.RULE_NONE, radius=0.2)]
    contrasts = [10.0, 0.1, 3.0, 20.0]
    phases, cells = [], []
    for cell, c in zip(base, contrasts):
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(c))
    c0 = [H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(len(cells))]
    E = np.eye(3)
    mat = hom.hom_filter_build(cells, phases)
    res = hom.hom_solve(mat, E, c0, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=1e-9, max_iter=2000)
    eps = cell_fields(res, cells, 2, "eps")
    for i, cell in enumerate(cells):
        fb = O.filter_build(cell, phases)
        ref = O.solve(fb["ctilde"], 2, cell.n, c0[i][0], c0[i][1], E, tol=1e-9, max_iter=2000)
        assert list(res["iterations"][i]) == list(ref["iterations"])
        assert _rel(res["mean_sigma"][i], ref["mean_sigma"]) < 1e-10
        assert _rel(eps[i], ref["eps"]) < 1e-10


def test_homogeneous_and_laminate_edge_cases():
    phases = H.two_phases(10.0)
    # homogeneous cell: converged at iteration 0, eps = E
    for dim, n in [(2, 3), (3, 5)]:
        nc = O.nc_of(dim)
        cell = H.homogeneous_cell(n, dim)
        mat = hom.hom_filter_build([cell], phases)
        E = np.eye(nc)
        res = hom.hom_solve(mat, E, [3.0, 2.0], precision=hom.HOM_FP64, tol=1e-12, max_iter=5)
        assert (res["iterations"] == 0).all() and (res["status"] == 0).all()
        C = hom.hom_effective_stiffness(E, res["mean_sigma"], dim)[0]
        np.testing.assert_allclose(C, O.isotropic_mandel(*phases[0], dim), atol=1e-13)
    # grid-aligned laminate on the smallest grids is exact
    from closed_forms import backus
    for n, m in [(3, 1), (5, 2), (9, 5)]:
        centre = 0.5 if m % 2 == 1 else 0.5 + 0.5 / n
        cell = H.laminate_cell(n, 2, m / n, axis=0, centre=centre)
        mat = hom.hom_filter_build([cell], phases)
        res = hom.hom_solve(mat, np.eye(3), H.mean_lame(phases), precision=hom.HOM_FP64, tol=1e-13, max_iter=3000)
        C = hom.hom_effective_stiffness(np.eye(3), res["mean_sigma"], 2)[0]
        assert _rel(C, backus(2, m / n, phases)) < 1e-11


def test_max_iter_and_divergence_status():
    cell = H.centred_disk_cell(15, rule=H.RULE_VOIGT)
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    lam0, mu0 = H.mean_lame(phases)
    res = hom.hom_solve(mat, np.eye(3), [lam0, mu0], precision=hom.HOM_FP64, tol=1e-14, max_iter=3)
    assert res["code"] == hom.HOM_ERR_NOT_CONVERGED
    assert (res["status"] == 1).all() and (res["iterations"] == 3).all()
    ref = O.solve(O.filter_build(cell, phases)["ctilde"], 2, 15, lam0, mu0, np.eye(3), tol=1e-14, max_iter=3)
    assert _rel(res["mean_sigma"][0], ref["mean_sigma"]) < 1e-10
    # a reference medium far below the optimal one (alpha < 1) makes the basic scheme diverge
    res = hom.hom_solve(mat, np.eye(3), [0.05 * lam0, 0.05 * mu0], precision=hom.HOM_FP64, tol=1e-8,
                        max_iter=400, diverge_window=10)
    assert res["code"] == hom.HOM_ERR_DIVERGED
    assert (res["status"] == 2).any()


def test_host_outputs_graphs_and_repeatability():
    cells = [H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER)]
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build(cells, phases)
    c0 = H.mean_lame(phases)
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-6, max_iter=500)
    a = hom.hom_solve(mat, np.eye(3), c0, **kw)
    b = hom.hom_solve(mat, np.eye(3), c0, host_fields=True, **kw)
    c = hom.hom_solve(mat, np.eye(3), c0, use_graph=True, check_every=4, **kw)
    for r in (b, c):
        assert np.array_equal(r["mean_sigma"], a["mean_sigma"])
        assert np.array_equal(r["iterations"], a["iterations"])
        assert torch.equal(r["eps"].cpu(), a["eps"].cpu())
        assert torch.equal(r["sigma"].cpu(), a["sigma"].cpu())


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp64"])
def test_whole_solve_graph_matches_host_loop(precision):
    """use_graph runs the whole solve as one graph launch (a conditional WHILE node; the control
    kernel ends the loop).  On an uneven batch whose pairs stop at different iterations -- some
    converge, some reach max_iter -- it gives exactly the host loop's results, on repeated calls
    (the second and third replay the cached graph), and with a different max_iter (another graph)."""
    base = [(H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER), 10.0), (H.centred_disk_cell(27, rule=H.RULE_VOIGT), 100.0),
            (H.centred_disk_cell(75, rule=H.RULE_REUSS), 0.1)]
    phases, cells = [], []
    for cell, contrast in base:
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(contrast))
    c0 = [H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(len(cells))]
    mat = hom.hom_filter_build(cells, phases)
    crit = hom.HOM_CRIT_EN if precision == hom.HOM_FP32 else hom.HOM_CRIT_E
    for max_iter in (120, 33):
        kw = dict(precision=precision, criterion=crit, tol=1e-6, max_iter=max_iter)
        a = hom.hom_solve(mat, np.eye(3), c0, **kw)
        if max_iter == 120:
            assert len(np.unique(a["iterations"])) > 2
        for _ in range(3):
            g = hom.hom_solve(mat, np.eye(3), c0, use_graph=True, **kw)
            assert g["code"] == a["code"]
            assert np.array_equal(g["iterations"], a["iterations"])
            assert np.array_equal(g["status"], a["status"])
            assert np.array_equal(g["mean_sigma"], a["mean_sigma"])
            assert torch.equal(g["eps"].cpu(), a["eps"].cpu())
        if max_iter == 33:
            assert (a["status"] == 1).any() and (a["iterations"] <= 33).all()


def test_kernel_stats_count_the_work():
    cells = [H.centred_disk_cell(45, rule=H.RULE_VOIGT)]
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build(cells, phases)
    r = hom.hom_solve(mat, np.eye(3), H.mean_lame(phases), precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN,
                      tol=1e-6, max_iter=500, stats=True)
    st = r["stats"]
    total_it = int(r["iterations"].sum())
    assert st["row"]["launches"] >= r["iterations"].max() + 1
    assert st["green"]["ms"] > 0 and st["row"]["ms"] > 0
    n, H_ = 45, 23
    # Green pass: read + write of 3 complex FP32 components and of the 2-vector g per bin
    per_it = 2 * 45 * H_ * (3 + 2) * 8
    assert st["green"]["bytes"] == per_it * (total_it + 3)
    assert r["voxel_iterations"] == n * n * total_it


def test_stagnation_stop():
    """stall_window: an FP32 load case whose error floor (FP32 rounding, about 9e-8 x contrast) lies
    above the tolerance stops as HOM_STATUS_STALLED long before max_iter; a case that converges is
    unaffected, and the stalled pair's returned iterate is as accurate as the floor allows."""
    base = [(H.centred_disk_cell(45, rule=H.RULE_VOIGT), 100.0), (H.centred_disk_cell(45, rule=H.RULE_REUSS), 2.0)]
    phases, cells = [], []
    for cell, contrast in base:
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(H.two_phases(contrast))
    c0 = [H.mean_lame(phases[0:2]), H.mean_lame(phases[2:4])]
    mat = hom.hom_filter_build(cells, phases)
    r = hom.hom_solve(mat, np.eye(3), c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-8,
                      max_iter=5000, stall_window=40)
    assert r["code"] == hom.HOM_ERR_NOT_CONVERGED
    assert (r["status"][0] == 3).all() and (r["iterations"][0] < 5000).all()
    assert (r["err_n"][0] < 1e-4).all()
    easy = hom.hom_solve(mat, np.eye(3), c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-5,
                         max_iter=5000, stall_window=40)
    ref = hom.hom_solve(mat, np.eye(3), c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-5, max_iter=5000)
    assert (easy["status"][1] == 0).all()
    np.testing.assert_array_equal(easy["iterations"][1], ref["iterations"][1])


@pytest.mark.parametrize("contrast", [100.0, 0.01])
def test_fp32_high_contrast_ceff_matches_oracle(contrast):
    """FP32 at the ends of the ensemble's contrast range: the solve stops at e_n < 1e-6 or, where the
    FP32 floor lies above that, at the stagnation stop; either way C_eff is within 1e-5 of the
    oracle's (converged to e < 1e-10)."""
    cells = [H.centred_disk_cell(45, rule=H.RULE_VOIGT), H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER)]
    phases = H.two_phases(contrast)
    c0 = H.mean_lame(phases)
    mat = hom.hom_filter_build(cells, phases)
    r = hom.hom_solve(mat, np.eye(3), [c0, c0], precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-6,
                      max_iter=5000, stall_window=50)
    assert np.isin(r["status"], (0, 3)).all()
    C = hom.hom_effective_stiffness(np.eye(3), r["mean_sigma"], 2)
    for i, cell in enumerate(cells):
        fb = O.filter_build(cell, phases)
        ref = O.solve(fb["ctilde"], 2, 45, c0[0], c0[1], np.eye(3), tol=1e-10, max_iter=20000)
        Cr = O.effective_stiffness(ref["mean_sigma"], np.eye(3))
        assert _rel(C[i], Cr) < 1e-5
