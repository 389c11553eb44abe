"""Pins of the oracle's Eyre-Milton scheme (solve_em_one; an accelerated scheme the paper cites as
complementary to filtering): the same discrete solution as the basic scheme, exact laminates, the
reflection property its derivation rests on, and the sqrt(contrast) acceleration."""
import numpy as np
import pytest

import hom_inputs as H
import oracle as O
from closed_forms import axis_permutation, backus, isotropic_mandel


def _disk(n, contrast, rule=H.RULE_VOIGT):
    ph = H.two_phases(contrast)
    return O.filter_build(H.centred_disk_cell(n, rule=rule), ph)["ctilde"], ph


@pytest.mark.parametrize("contrast,n", [(10.0, 27), (1e3, 15)])
def test_em_solution_is_the_fixed_point_solution(contrast, n):
    """Same discrete solution as conjugate gradients on the projected equilibrium equation (a
    solver that shares no step with the scheme), in far fewer iterations than the basic scheme."""
    ct, ph = _disk(n, contrast, H.RULE_TWO_LAYER)
    l0, m0 = O.em_reference(ph, 2)
    r = O.solve_em(ct, 2, n, l0, m0, np.eye(3), tol=1e-11, max_iter=5000)
    assert all(s == "converged" for s in r["status"])
    rc = O.solve_cg(ct, 2, n, np.eye(3), tol=1e-10, max_iter=5000)
    assert all(s == "converged" for s in rc["status"])
    C = O.effective_stiffness(r["mean_sigma"], np.eye(3))
    Cc = O.effective_stiffness(rc["mean_sigma"], np.eye(3))
    np.testing.assert_allclose(C, Cc, rtol=0, atol=1e-9 * np.abs(Cc).max())
    np.testing.assert_allclose(r["eps"], rc["eps"], rtol=0, atol=1e-8 * np.abs(rc["eps"]).max())
    if contrast > 100:
        # sqrt(kappa) against kappa: the basic scheme is still far from tol after 10x the count
        lb, mb = H.mean_lame(ph)
        k = 10 * int(r["iterations"].max())
        rb = O.solve_one(ct, 2, n, lb, mb, np.eye(3)[0], tol=1e-11, max_iter=k, criterion=O.CRIT_EN)
        assert rb["status"] == "max_iter" and rb["errors_n"][-1] > 1e-9


def test_em_homogeneous_cell_with_c0_equal_c():
    ph = H.two_phases(10.0)
    ct = O.filter_build(H.homogeneous_cell(9, 2), ph)["ctilde"]
    E = np.array([0.3, -0.1, 0.2])
    r = O.solve_em_one(ct, 2, 9, ph[0][0], ph[0][1], E, tol=1e-14, max_iter=10)
    assert r["iterations"] == 0
    np.testing.assert_allclose(r["eps"].reshape(3, -1), np.repeat(E[:, None], 81, axis=1), atol=1e-15)


@pytest.mark.parametrize("dim,n,m,axis", [(2, 15, 4, 1), (3, 7, 3, 2)])
def test_em_grid_aligned_laminate_is_exact(dim, n, m, axis):
    ph = H.two_phases(100.0)
    nc = O.nc_of(dim)
    centre = 0.5 if m % 2 == 1 else 0.5 + 0.5 / n
    ct = O.filter_build(H.laminate_cell(n, dim, m / n, axis=axis, centre=centre), ph)["ctilde"]
    l0, m0 = O.em_reference(ph, dim)
    r = O.solve_em(ct, dim, n, l0, m0, np.eye(nc), tol=1e-12, max_iter=5000)
    C = O.effective_stiffness(r["mean_sigma"], np.eye(nc))
    p = axis_permutation(dim, axis)
    expect = backus(dim, m / n, ph)[np.ix_(p, p)]
    np.testing.assert_allclose(C, expect, rtol=0, atol=1e-9 * np.abs(expect).max())


def test_reflection_is_an_isometry_for_the_c0_inverse_inner_product():
    """R = I - 2 c0 Gamma0 preserves <w, c0^-1 w> on zero-mean fields (and R R = I): the identity
    that makes the scheme's map a contraction."""
    n, dim = 11, 2
    rng = np.random.default_rng(4)
    l0, m0 = 0.8, 1.3
    C0 = isotropic_mandel(l0, m0, dim)
    iC0 = np.linalg.inv(C0)
    w = rng.standard_normal((3, n, n))
    w -= w.reshape(3, -1).mean(axis=1)[:, None, None]
    w_hat = O._fft(w, dim)

    def R(x_hat):
        return x_hat - 2.0 * np.einsum("IJ,J...->I...", C0, -O.apply_gamma0(x_hat, dim, n, l0, m0))
    Rw = np.real(O._ifft(R(w_hat), dim))
    q = lambda f: float(np.sum(f * np.einsum("IJ,J...->I...", iC0, f)))
    assert abs(q(Rw) - q(w)) < 1e-12 * q(w)
    np.testing.assert_allclose(np.real(O._ifft(R(R(w_hat)), dim)), w, atol=1e-12)



@pytest.mark.parametrize("lam0,mu0", [(1.1, 0.9), (3.0, 0.2)])
def test_compatibility_error_closed_forms(lam0, mu0):
    """Fields of one wave along x (the last numpy axis) in 2D, Mandel order (11, 22, sqrt2 12).
    eps_22(x) = f(x) is not compatible (eps_22'' along x must vanish): the c0-orthogonal split keeps
    the part with the same divergence of c0 eps, u_1 from (lam0 + 2 mu0) u_1'' = lam0 f', i.e. a
    compatible eps_11 = r f, r = lam0 / (lam0 + 2 mu0); the remainder (-r f, f, 0) has RMS
    a sqrt((1 + r^2) / 2).  eps_12(x), eps_11(x) and eps_22(y) are symmetric gradients: e_c = 0.
    A wrong mean at k = 0 counts fully."""
    n, dim = 16, 2
    x = (np.arange(n) + 0.5) / n
    f = np.cos(2 * np.pi * x)
    E = np.array([0.4, -0.2, 0.3])
    a = 0.3
    r = lam0 / (lam0 + 2 * mu0)

    def field(comp, along_x):
        eps = np.broadcast_to(E[:, None, None], (3, n, n)).copy()
        eps[comp] += a * (f[None, :] if along_x else f[:, None])
        return eps

    ne = np.linalg.norm(E)
    got = O.compatibility_error(field(1, True), dim, n, lam0, mu0, E)
    assert abs(got - a * np.sqrt((1 + r * r) / 2) / ne) < 1e-12
    for comp, along_x in ((2, True), (0, True), (1, False)):
        assert O.compatibility_error(field(comp, along_x), dim, n, lam0, mu0, E) < 1e-14
    shifted = np.broadcast_to((E + [0.0, 0.1, 0.0])[:, None, None], (3, n, n))
    assert abs(O.compatibility_error(shifted, dim, n, lam0, mu0, E) - 0.1 / ne) < 1e-14


def test_basic_scheme_iterates_are_compatible():
    """The basic scheme's iterates are compatible by construction (section 2): e_c of its solution
    is at rounding level, while the Eyre-Milton solution reaches e_c < tol only at convergence."""
    cell = H.centred_disk_cell(15, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(10.0)
    fb = O.filter_build(cell, phases)
    l0, m0 = O.em_reference(phases, 2)
    E = np.eye(3)
    lb, mb = H.mean_lame(phases)
    b = O.solve(fb["ctilde"], 2, 15, lb, mb, E, tol=1e-6, max_iter=2000)
    for i in range(3):
        # being a symmetric gradient does not depend on the c0 that defines the split
        assert O.compatibility_error(b["eps"][i], 2, 15, l0, m0, E[i]) < 1e-13
    em = O.solve_em(fb["ctilde"], 2, 15, l0, m0, E, tol=1e-8, max_iter=2000)
    for i in range(3):
        assert em["errors_c"][i][-1] < 1e-8 and em["errors_c"][i][0] > 1e-4


def test_em_reference_media_agree():
    """The input generators' reference medium for the scheme and the oracle's are the same
    geometric means (written independently on each side)."""
    for contrast in (0.01, 10.0, 1e3):
        ph = H.two_phases(contrast)
        for dim in (2, 3):
            np.testing.assert_allclose(H.geometric_lame(ph, dim), O.em_reference(ph, dim), rtol=1e-14)


def test_em_on_an_even_grid_reaches_the_cg_solution():
    """Even grids (the Nyquist convention: Gamma0 left out at bins with a Nyquist component): the
    scheme's fixed point has zero Nyquist strain, so it is the same discrete solution as conjugate
    gradients on the projected equilibrium equation."""
    n = 16
    ct, ph = _disk(n, 10.0, H.RULE_TWO_LAYER)
    l0, m0 = O.em_reference(ph, 2)
    r = O.solve_em(ct, 2, n, l0, m0, np.eye(3), tol=1e-11, max_iter=3000)
    assert all(s == "converged" for s in r["status"])
    rc = O.solve_cg(ct, 2, n, np.eye(3), tol=1e-11, max_iter=3000)
    np.testing.assert_allclose(r["mean_sigma"], rc["mean_sigma"], rtol=0, atol=1e-9 * np.abs(rc["mean_sigma"]).max())
    np.testing.assert_allclose(r["eps"], rc["eps"], rtol=0, atol=1e-8 * np.abs(rc["eps"]).max())
    eps_hat = np.fft.fft2(r["eps"])
    assert np.abs(eps_hat[:, :, n // 2, :]).max() < 1e-8 * n * n and np.abs(eps_hat[:, :, :, n // 2]).max() < 1e-8 * n * n
