"""Pins of the oracle's defect correction of the basic scheme (solve_refined_one): an exact
reformulation of the fixed point of section 2 (eqs. 1-a, 1-b, 2) in which FP64 residuals drive
corrections computed by the same fixed point, so that a low-precision iteration reaches a
high-precision tolerance."""
import numpy as np

import hom_inputs as H
import oracle as O


def _cell(n, contrast):
    cell = H.centred_disk_cell(n, rule=H.RULE_VOIGT)
    ph = H.two_phases(contrast)
    lam0, mu0 = H.mean_lame(ph)
    return O.filter_build(cell, ph)["ctilde"], lam0, mu0


def _uniform(E, n):
    eps = np.empty((3, n, n))
    for I in range(3):
        eps[I] = E[I]
    return eps


def test_refined_solution_is_the_fixed_point_solution():
    n = 27
    ct, lam0, mu0 = _cell(n, 10.0)
    C = []
    for l in range(3):
        E = np.eye(3)[l]
        r = O.solve_refined_one(ct, 2, n, lam0, mu0, E, tol=1e-11, start=_uniform(E, n), inner_iters=20, max_outer=40)
        assert r["status"] == "converged"
        C.append(r["mean_sigma"])
    ref = O.solve(ct, 2, n, lam0, mu0, np.eye(3), tol=1e-12, max_iter=3000, criterion=O.CRIT_EN)
    np.testing.assert_allclose(O.effective_stiffness(np.array(C), np.eye(3)),
                               O.effective_stiffness(ref["mean_sigma"], np.eye(3)), rtol=0, atol=1e-9)


def test_one_step_with_a_converged_inner_solve_is_exact():
    """The problem is affine, so the correction's fixed point is the exact error: one outer step with
    the inner iteration run to convergence lands on the solution from any start."""
    n = 27
    ct, lam0, mu0 = _cell(n, 10.0)
    E = np.array([0.3, -0.2, 0.5])
    start = _uniform(E, n) + 0.01 * np.random.default_rng(1).standard_normal((3, n, n))
    r = O.solve_refined_one(ct, 2, n, lam0, mu0, E, tol=-1.0, start=start, inner_iters=400, max_outer=1)
    assert r["outer"] == 1
    sigma = O.constitutive(ct, r["eps"])
    e, e_n = O.equilibrium_errors(O._fft(sigma, 2), 2, n)
    assert e_n < 1e-12
    np.testing.assert_allclose(r["eps"].reshape(3, -1).mean(axis=1), E, atol=1e-14)


def test_fp32_storage_floor_is_removed():
    """Rounding the iterate to FP32 after every step stalls the basic scheme at e_n ~ 8e-7 at contrast
    100; the corrections, with their inner fields rounded to FP32 as well, go below 1e-9 in two outer
    steps, since the rounding is relative to the correction, not to the strain."""
    n = 27
    ct, lam0, mu0 = _cell(n, 100.0)
    E = np.array([1.0, 0.0, 0.0])
    eps = _uniform(E, n)
    errs = []
    for it in range(900):
        eps = O.fixed_point_map(ct, 2, n, lam0, mu0, E, eps).astype(np.float32).astype(np.float64)
        if it >= 700:
            errs.append(O.equilibrium_errors(O._fft(O.constitutive(ct, eps), 2), 2, n)[1])
    assert min(errs) > 1e-7
    r = O.solve_refined_one(ct, 2, n, lam0, mu0, E, tol=1e-9, start=eps, inner_iters=300, max_outer=4,
                            inner_dtype=np.float32)
    assert r["status"] == "converged" and r["outer"] <= 2
