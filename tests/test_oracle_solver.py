"""Pins of the oracle's fixed-point solver (section 2, eqs. 1-a, 1-b, 2) and of C_eff:
homogeneous cell, exact laminate solutions (Backus), the 2-layer filter reproducing a laminate,
variational bounds, symmetry and the energy identity."""
import math

import numpy as np
import pytest

import hom_inputs as H
import oracle as O
from closed_forms import axis_permutation, backus, hs_bulk_bounds_2d, isotropic_mandel


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_homogeneous_cell(dim, n):
    ph = H.two_phases(10.0)
    nc = O.nc_of(dim)
    cell = H.homogeneous_cell(n, dim)
    ct = O.filter_build(cell, ph)["ctilde"]
    lam0, mu0 = 3.0, 2.0
    r = O.solve(ct, dim, n, lam0, mu0, np.eye(nc), tol=1e-12, max_iter=10)
    assert list(r["iterations"]) == [0] * nc
    C = O.effective_stiffness(r["mean_sigma"], np.eye(nc))
    np.testing.assert_allclose(C, isotropic_mandel(*ph[0], dim), atol=1e-14)
    # one forced iteration keeps eps = E exactly (c0 != c)
    E = np.arange(1.0, nc + 1.0)
    r = O.solve(ct, dim, n, lam0, mu0, E[None], tol=-1.0, max_iter=1)
    assert r["iterations"][0] == 1 and r["status"][0] == "max_iter"
    np.testing.assert_allclose(r["eps"][0], np.broadcast_to(E.reshape((nc,) + (1,) * dim), r["eps"][0].shape),
                               atol=1e-13)


@pytest.mark.parametrize("dim,n,m,axis", [(2, 9, 5, 0), (2, 15, 4, 1), (2, 45, 17, 0),
                                          (3, 5, 2, 0), (3, 7, 3, 2), (3, 5, 3, 1)])
def test_grid_aligned_laminate_is_exact(dim, n, m, axis):
    """A slab of m whole voxel columns: the discrete solution is the continuum laminate."""
    ph = H.two_phases(10.0)
    nc = O.nc_of(dim)
    centre = 0.5 if m % 2 == 1 else 0.5 + 0.5 / n
    cell = H.laminate_cell(n, dim, m / n, axis=axis, centre=centre)
    ct = O.filter_build(cell, ph)["ctilde"]
    lam0, mu0 = O.default_reference(ph)
    r = O.solve(ct, dim, n, lam0, mu0, np.eye(nc), tol=1e-12, max_iter=3000)
    assert all(s == "converged" for s in r["status"])
    C = O.effective_stiffness(r["mean_sigma"], np.eye(nc))
    p = axis_permutation(dim, axis)
    expect = backus(dim, m / n, ph)[np.ix_(p, p)]
    np.testing.assert_allclose(C, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


@pytest.mark.parametrize("dim,n,axis", [(2, 15, 0), (2, 9, 1), (3, 7, 2)])
def test_two_layer_filter_reproduces_laminate(dim, n, axis):
    """Interfaces inside voxels + 2-layer filter: every voxel is a laminate with the slab normal,
    so C_eff is the laminate of the mean volume fraction (exact)."""
    ph = H.two_phases(0.1)
    nc = O.nc_of(dim)
    cell = H.laminate_cell(n, dim, 0.37, axis=axis, centre=0.43, rule=H.RULE_TWO_LAYER,
                           radius_px=1.0, subgrid=8)
    fb = O.filter_build(cell, ph)
    assert fb["mixed"].sum() > 0
    fmean = fb["counts"][..., 1].mean() / fb["M"]
    lam0, mu0 = O.default_reference(ph)
    r = O.solve(fb["ctilde"], dim, n, lam0, mu0, np.eye(nc), tol=1e-12, max_iter=3000)
    C = O.effective_stiffness(r["mean_sigma"], np.eye(nc))
    p = axis_permutation(dim, axis)
    expect = backus(dim, fmean, ph)[np.ix_(p, p)]
    np.testing.assert_allclose(C, expect, atol=1e-10 * np.abs(expect).max())


@pytest.fixture(scope="module")
def disk_solution():
    n = 45
    ph = H.two_phases(10.0)
    cell = H.centred_disk_cell(n, vf=0.2, rule=H.RULE_VOIGT, radius_px=1.0, subgrid=16)
    fb = O.filter_build(cell, ph)
    lam0, mu0 = O.default_reference(ph)
    r = O.solve(fb["ctilde"], 2, n, lam0, mu0, np.eye(3), tol=1e-10, max_iter=3000)
    return n, ph, fb, r


def test_disk_symmetry_and_bounds(disk_solution):
    n, ph, fb, r = disk_solution
    C = O.effective_stiffness(r["mean_sigma"], np.eye(3))
    sc = np.abs(C).max()
    # major symmetry and square symmetry of the centred disk
    np.testing.assert_allclose(C, C.T, atol=1e-8 * sc)
    assert abs(C[0, 0] - C[1, 1]) < 1e-8 * sc
    assert abs(C[0, 2]) < 1e-8 * sc and abs(C[1, 2]) < 1e-8 * sc
    # discrete Voigt / Reuss bounds of the grid field
    ct = fb["ctilde"].reshape(-1, 3, 3)
    voigt = ct.mean(axis=0)
    reuss = np.linalg.inv(np.linalg.inv(ct).mean(axis=0))
    assert np.linalg.eigvalsh(voigt - C).min() > -1e-8 * sc
    assert np.linalg.eigvalsh(C - reuss).min() > -1e-8 * sc
    # Hashin-Shtrikman bounds on the plane-strain bulk modulus (discretisation margin 2%)
    K = (C[0, 0] + C[0, 1] + C[1, 0] + C[1, 1]) / 4.0
    lo, hi = hs_bulk_bounds_2d(ph, 0.2)
    assert lo * 0.98 <= K <= hi * 1.02


def test_energy_identity(disk_solution):
    """C_ij = <eps^(i) : c : eps^(j)> at the discrete solution."""
    n, ph, fb, r = disk_solution
    C = O.effective_stiffness(r["mean_sigma"], np.eye(3))
    eps = r["eps"].reshape(3, 3, -1)
    sig = r["sigma"].reshape(3, 3, -1)
    W = np.einsum("iIx,jIx->ij", eps, sig) / eps.shape[-1]
    np.testing.assert_allclose(W, C, atol=1e-7 * np.abs(C).max())


def test_converged_error_below_tolerance(disk_solution):
    n, ph, fb, r = disk_solution
    for errs, it in zip(r["errors"], r["iterations"]):
        assert errs[-1] < 1e-10 and len(errs) == it + 1
        assert errs[0] > 1e-3


def test_filtering_leaves_iteration_count_alike():
    """Section 5: filtering has neither a positive nor a negative effect on the iteration count
    of the basic scheme (contrast 10, N = 45, tolerance 1e-4 on e)."""
    n = 45
    ph = H.two_phases(10.0)
    lam0, mu0 = O.default_reference(ph)
    its = {}
    for rule in (H.RULE_NONE, H.RULE_VOIGT, H.RULE_TWO_LAYER):
        cell = H.centred_disk_cell(n, rule=rule)
        fb = O.filter_build(cell, ph)
        its[rule] = O.solve(fb["ctilde"], 2, n, lam0, mu0, np.array([[0.01, 0, 0]]), tol=1e-4,
                            max_iter=1000)["iterations"][0]
    base = its[H.RULE_NONE]
    for v in its.values():
        assert abs(v - base) <= max(3, 0.25 * base), its


def test_effective_stiffness_general_loads():
    C = np.array([[3.0, 1.0, 0.2], [1.0, 4.0, 0.1], [0.2, 0.1, 2.0]])
    E = np.array([[1.0, 0.5, 0.0], [0.0, 2.0, 1.0], [0.3, 0.0, 1.0]])
    S = E @ C.T
    np.testing.assert_allclose(O.effective_stiffness(S, E), C, atol=1e-13)
