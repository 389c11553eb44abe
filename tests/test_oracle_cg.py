"""Pins of the oracle's conjugate-gradient solver (the accelerated scheme applied to the paper's
discrete problem) against facts that do not come from its own code:

* the discrete solution is unique, so CG must reach the fixed point's solution (section 2) on the
  same cell and filter;
* a homogeneous cell needs no step; a grid-aligned laminate reaches the exact Backus stiffness, and
  does so in a handful of steps (few distinct eigenvalues on fields that vary along one axis);
* the residuals are mutually orthogonal and the directions A-conjugate (what makes it CG);
* the stopping quantity e_G sits between e_n and sqrt(2) e_n of the same iterate;
* the paper's statement (section 5, after its ref. [12]) that Krylov schemes sharply reduce the
  contrast sensitivity of the basic scheme: at contrast 1e3 CG takes far fewer steps.
"""
import math

import numpy as np
import pytest

import hom_inputs as H
import oracle as O
from closed_forms import axis_permutation, backus


def test_same_solution_as_the_fixed_point():
    cell = H.centred_disk_cell(25, rule=H.RULE_TWO_LAYER)
    ph = H.two_phases(10.0)
    ct = O.filter_build(cell, ph)["ctilde"]
    lam0, mu0 = O.default_reference(ph)
    E = np.eye(3)
    fp = O.solve(ct, 2, 25, lam0, mu0, E, tol=1e-13, max_iter=5000)
    cg = O.solve_cg(ct, 2, 25, E, tol=1e-13, max_iter=500)
    assert all(s == "converged" for s in cg["status"])
    scale = np.abs(fp["eps"]).max()
    assert np.abs(cg["eps"] - fp["eps"]).max() < 1e-10 * scale
    assert np.abs(cg["mean_sigma"] - fp["mean_sigma"]).max() < 1e-10 * np.abs(fp["mean_sigma"]).max()


def test_homogeneous_cell_takes_no_step():
    ct = O.filter_build(H.homogeneous_cell(9, 2), H.two_phases(10.0))["ctilde"]
    r = O.solve_cg_one(ct, 2, 9, np.array([0.3, -0.1, 0.2]), tol=1e-12, max_iter=10)
    assert r["iterations"] == 0 and r["status"] == "converged"
    np.testing.assert_allclose(r["eps"][:, 2, 3], [0.3, -0.1, 0.2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,n,m,axis", [(2, 15, 6, 0), (2, 9, 4, 1), (3, 7, 3, 2)])
def test_grid_aligned_laminate_exact_in_few_steps(dim, n, m, axis):
    ph = H.two_phases(100.0)
    nc = O.nc_of(dim)
    centre = 0.5 if m % 2 == 1 else 0.5 + 0.5 / n
    cell = H.laminate_cell(n, dim, m / n, axis=axis, centre=centre)
    ct = O.filter_build(cell, ph)["ctilde"]
    r = O.solve_cg(ct, dim, n, np.eye(nc), tol=1e-12, max_iter=50)
    assert all(s == "converged" for s in r["status"])
    assert max(r["iterations"]) <= 4, r["iterations"]
    C = O.effective_stiffness(r["mean_sigma"], np.eye(nc))
    p = axis_permutation(dim, axis)
    expect = backus(dim, m / n, ph)[np.ix_(p, p)]
    np.testing.assert_allclose(C, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


def test_residuals_orthogonal_and_directions_conjugate():
    cell = H.centred_disk_cell(15, rule=H.RULE_VOIGT)
    ct = O.filter_build(cell, H.two_phases(50.0))["ctilde"]
    r = O.solve_cg_one(ct, 2, 15, np.array([1.0, 0.0, 0.0]), tol=1e-30, max_iter=8, history=True)
    R = r["residuals"]
    for i in range(len(R)):
        for j in range(i):
            cos = O._dot(R[i], R[j]) / math.sqrt(O._dot(R[i], R[i]) * O._dot(R[j], R[j]))
            assert abs(cos) < 1e-8, (i, j, cos)
    # directions rebuilt from the residuals: p_0 = r_0, p_k = r_k + beta_k p_{k-1}
    P = [R[0]]
    for k in range(1, len(R)):
        P.append(R[k] + O._dot(R[k], R[k]) / O._dot(R[k - 1], R[k - 1]) * P[-1])
    AP = [O.projection_G(O.constitutive(ct, p), 2, 15) for p in P]
    for i in range(len(P)):
        for j in range(i):
            c = O._dot(P[i], AP[j]) / math.sqrt(O._dot(P[i], AP[i]) * O._dot(P[j], AP[j]))
            assert abs(c) < 1e-8, (i, j, c)


def test_stopping_quantity_between_en_and_sqrt2_en():
    cell = H.centred_disk_cell(21, rule=H.RULE_REUSS)
    ct = O.filter_build(cell, H.two_phases(0.05))["ctilde"]
    for steps in (0, 3, 12):
        r = O.solve_cg_one(ct, 2, 21, np.array([0.0, 0.0, 1.0]), tol=1e-30, max_iter=steps)
        e, e_n = O.equilibrium_errors(np.fft.fftn(r["sigma"], axes=(-2, -1)), 2, 21)
        e_g = r["errors"][-1]
        assert e_n * (1 - 1e-9) <= e_g <= math.sqrt(2.0) * e_n * (1 + 1e-9), (steps, e_g, e_n)


def test_far_fewer_steps_than_the_basic_scheme_at_high_contrast():
    cell = H.centred_disk_cell(25, rule=H.RULE_TWO_LAYER, radius=math.pi / 15)
    ph = H.two_phases(1e3)
    ct = O.filter_build(cell, ph)["ctilde"]
    lam0, mu0 = O.default_reference(ph)
    E = np.array([1.0, 0.0, 0.0])
    fp = O.solve_one(ct, 2, 25, lam0, mu0, E, tol=1e-4, max_iter=20000, criterion=O.CRIT_EN)
    cg = O.solve_cg_one(ct, 2, 25, E, tol=1e-4, max_iter=2000)
    assert fp["status"] == "converged" and cg["status"] == "converged"
    assert 5 * cg["iterations"] < fp["iterations"], (cg["iterations"], fp["iterations"])
