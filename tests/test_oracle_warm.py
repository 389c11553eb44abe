"""Pins of the oracle's warm start (solve_one(eps0=...)): the fixed point of eqs. 1-a, 1-b, 2 is
unique, so any start reaches the cold start's solution; a start at that solution returns after one
Green-operator application with the same fields; and an incompatible start with an equilibrated
stress (the laminate case) is not returned as converged at iterate 0."""
import numpy as np

import hom_inputs as H
import oracle as O


def _cell(n=21, contrast=10.0):
    ph = H.two_phases(contrast)
    fb = O.filter_build(H.centred_disk_cell(n, rule=H.RULE_TWO_LAYER), ph)
    return fb["ctilde"], H.mean_lame(ph)


def test_any_start_reaches_the_cold_solution():
    ct, (l0, m0) = _cell()
    E = np.eye(3)
    cold = O.solve(ct, 2, 21, l0, m0, E, tol=1e-11, max_iter=2000, criterion=O.CRIT_EN)
    rng = np.random.default_rng(4)
    eps0 = rng.standard_normal((3, 3, 21, 21))
    warm = O.solve(ct, 2, 21, l0, m0, E, tol=1e-11, max_iter=2000, criterion=O.CRIT_EN, eps0=eps0)
    assert all(s == "converged" for s in warm["status"])
    np.testing.assert_allclose(warm["eps"], cold["eps"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(warm["mean_sigma"], cold["mean_sigma"], rtol=0, atol=1e-10)


def test_start_at_the_solution_returns_after_one_application():
    ct, (l0, m0) = _cell()
    E = np.eye(3)
    cold = O.solve(ct, 2, 21, l0, m0, E, tol=1e-12, max_iter=3000, criterion=O.CRIT_EN)
    warm = O.solve(ct, 2, 21, l0, m0, E, tol=1e-10, max_iter=10, criterion=O.CRIT_EN, eps0=cold["eps"])
    assert list(warm["iterations"]) == [1, 1, 1]
    np.testing.assert_allclose(warm["eps"], cold["eps"], rtol=0, atol=1e-10)


def test_incompatible_start_is_not_returned():
    """A grid-aligned laminate (pure voxels, stiffness varying along x only) and a start whose
    stress is in equilibrium although the strain is not compatible: eps_22(x) = 1 + 0.3 cos(2 pi x)
    (a function of x in eps_22 is not a symmetric gradient) with eps_11(x) chosen so that sigma_11 is
    uniform and eps_12 = 0.  Its equilibrium error is at rounding level, so iterate 0 would pass
    the test; the warm start skips it, and the returned iterate is the cold start's solution."""
    n = 15
    ph = H.two_phases(100.0)
    ct = O.filter_build(H.laminate_cell(n, 2, 5 / n, axis=0, centre=0.5), ph)["ctilde"]
    l0, m0 = H.mean_lame(ph)
    E = np.array([[0.0, 1.0, 0.0]])
    x = (np.arange(n) + 0.5) / n
    e22 = np.broadcast_to(1.0 + 0.3 * np.cos(2 * np.pi * x)[None, :], (n, n))
    eps0 = np.zeros((1, 3, n, n))
    eps0[0, 1] = e22
    eps0[0, 0] = (2.0 - ct[..., 0, 1] * e22) / ct[..., 0, 0]  # sigma_11 = 2 everywhere
    assert np.ptp(ct[..., 0, 0], axis=0).max() == 0.0  # the stiffness varies along x only
    cold = O.solve(ct, 2, n, l0, m0, E, tol=1e-12, max_iter=5000, criterion=O.CRIT_EN)
    warm = O.solve(ct, 2, n, l0, m0, E, tol=1e-12, max_iter=5000, criterion=O.CRIT_EN, eps0=eps0)
    assert warm["errors_n"][0][0] < 1e-13  # iterate 0 is in equilibrium ...
    assert warm["iterations"][0] >= 1      # ... and still not returned
    assert warm["status"][0] == "converged"
    np.testing.assert_allclose(warm["mean_sigma"], cold["mean_sigma"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(warm["eps"], cold["eps"], rtol=0, atol=1e-9)
