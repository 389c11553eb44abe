"""GPU tests of the warm start (hom_solve(eps0=...): the initial strain field read from, and the
result written back to, the same device buffer) and of the residual history (history=True),
against the oracle run from the same start: identical iteration counts and fields in FP64, the
unchecked iterate 0 of a warm start, and the per-iterate errors of the basic and Eyre-Milton
schemes."""
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


def _dev(field):
    return torch.tensor(np.ascontiguousarray(field).ravel(), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,dim", [(21, 2), (16, 2), (9, 3)])
def test_warm_start_matches_oracle(n, dim):
    cell = H.centred_disk_cell(n, rule=H.RULE_TWO_LAYER) if dim == 2 else \
        H.rsa_spheres_cell(n, seed=n, vf=0.12, rmin=0.12, rmax=0.16, subgrid=4, gap_voxels=0.5)
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    nc = O.nc_of(dim)
    E = np.eye(nc)
    fb = O.filter_build(cell, phases)
    rng = np.random.default_rng(100 + n)
    eps0 = rng.standard_normal((nc, nc) + (n,) * dim)
    ref = O.solve(fb["ctilde"], dim, n, c0[0], c0[1], E, tol=1e-10, max_iter=2000, criterion=O.CRIT_EN, eps0=eps0)
    mat = hom.hom_filter_build([cell], phases)
    res = hom.hom_solve(mat, E, [c0], precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=1e-10,
                        max_iter=2000, eps0=_dev(eps0), history=True)
    assert (res["status"] == 0).all()
    assert np.abs(res["iterations"][0].astype(int) - ref["iterations"]).max() <= 1
    eps = cell_fields(res, [cell], dim, "eps")[0]
    assert _rel(eps, ref["eps"]) < 1e-8
    assert _rel(res["mean_sigma"][0], ref["mean_sigma"]) < 1e-9
    assert np.isnan(res["history"][0, :, 0]).all()  # iterate 0 of a warm start is not checked


def test_warm_start_at_the_solution_and_incompatible_start():
    cell = H.centred_disk_cell(21, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    fb = O.filter_build(cell, phases)
    ref = O.solve(fb["ctilde"], 2, 21, c0[0], c0[1], np.eye(3), tol=1e-12, max_iter=3000, criterion=O.CRIT_EN)
    mat = hom.hom_filter_build([cell], phases)
    res = hom.hom_solve(mat, np.eye(3), [c0], precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=1e-10,
                        max_iter=10, eps0=_dev(ref["eps"]))
    assert list(res["iterations"][0]) == [1, 1, 1]
    assert _rel(cell_fields(res, [cell], 2, "eps")[0], ref["eps"]) < 1e-10
    # equilibrated but incompatible start on a grid-aligned laminate (see the oracle's pin)
    n = 15
    ph = H.two_phases(100.0)
    lam = H.laminate_cell(n, 2, 5 / n, axis=0, centre=0.5)
    ct = O.filter_build(lam, ph)["ctilde"]
    l0, m0 = H.mean_lame(ph)
    x = (np.arange(n) + 0.5) / n
    e22 = np.broadcast_to(1.0 + 0.3 * np.cos(2 * np.pi * x)[None, :], (n, n))
    eps0 = np.zeros((1, 3, n, n))
    eps0[0, 1] = e22
    eps0[0, 0] = (2.0 - ct[..., 0, 1] * e22) / ct[..., 0, 0]
    E = np.array([[0.0, 1.0, 0.0]])
    cold = O.solve(ct, 2, n, l0, m0, E, tol=1e-12, max_iter=5000, criterion=O.CRIT_EN)
    m2 = hom.hom_filter_build([lam], ph)
    r2 = hom.hom_solve(m2, E, [(l0, m0)], precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=1e-12,
                       max_iter=5000, eps0=_dev(eps0))
    assert r2["iterations"][0, 0] >= 1 and r2["status"][0, 0] == 0
    assert _rel(r2["mean_sigma"][0], cold["mean_sigma"]) < 1e-9


def test_history_basic_and_em_match_oracle():
    cell = H.centred_disk_cell(27, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(10.0)
    fb = O.filter_build(cell, phases)
    mat = hom.hom_filter_build([cell], phases)
    E = np.eye(3)
    c0 = H.mean_lame(phases)
    ref = O.solve(fb["ctilde"], 2, 27, c0[0], c0[1], E, tol=1e-10, max_iter=500, criterion=O.CRIT_EN)
    res = hom.hom_solve(mat, E, [c0], precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=1e-10,
                        max_iter=500, history=True, fields=False)
    for l in range(3):
        k = int(res["iterations"][0, l])
        h = res["history"][0, l]
        assert k == ref["iterations"][l]
        np.testing.assert_allclose(h[:k + 1], ref["errors_n"][l], rtol=1e-6, atol=1e-14)
        assert np.isnan(h[k + 1:]).all()
        assert h[k] == res["err_n"][0, l]
    g = H.geometric_lame(phases, 2)
    rem = O.solve_em(fb["ctilde"], 2, 27, g[0], g[1], E, tol=1e-10, max_iter=500)
    em = hom.hom_solve(mat, E, [g], precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=1e-10, max_iter=500,
                       history=True, fields=False, scheme=hom.HOM_SCHEME_EYRE_MILTON)
    for l in range(3):
        k = int(em["iterations"][0, l])
        assert abs(k - rem["iterations"][l]) <= 1
        m = min(k, int(rem["iterations"][l])) + 1
        want = np.maximum(rem["errors_n"][l], rem["errors_c"][l])[:m]
        np.testing.assert_allclose(em["history"][0, l, :m], want, rtol=1e-6, atol=1e-14)


def test_history_on_the_specialised_fp32_passes():
    cell = H.centred_disk_cell(45, rule=H.RULE_VOIGT)
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    res = hom.hom_solve(mat, np.eye(3), [H.mean_lame(phases)], precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN,
                        tol=1e-5, max_iter=300, history=True, fields=False)
    assert (res["status"] == 0).all()
    for l in range(3):
        k = int(res["iterations"][0, l])
        h = res["history"][0, l, :k + 1]
        assert np.isfinite(h).all() and h[-1] < 1e-5 <= h[:-1].min()
        assert h[-1] == res["err_n"][0, l]
