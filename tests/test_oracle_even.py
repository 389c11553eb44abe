"""Pins of the oracle on even grids, which the paper does not define (its J is for odd N).  Reading:
a wave vector with a Nyquist component (bin n/2) gets zero strain from the Green operator and is
left out of the equilibrium errors.  Checked against facts that do not depend on that code:

* the Green operator of c0 = identity stays an L2-orthogonal projection (idempotent, self-adjoint)
  and its output has no Nyquist content;
* the equilibrium errors of a closed-form cosine field; a field whose only variation sits at the
  Nyquist frequency counts as equilibrated;
* a homogeneous cell needs no iteration; fixed point and conjugate gradients reach one solution;
* the 2-layer filter's smooth spatial convergence (section 3): C_11 at n = 32 lies between its values
  at the odd neighbours 31 and 33.
"""
import math

import numpy as np
import pytest

import hom_inputs as H
import oracle as O

RNG = np.random.default_rng(2024)


@pytest.mark.parametrize("dim,n", [(2, 8), (2, 12), (3, 6)])
def test_projection_on_even_grids(dim, n):
    nc = O.nc_of(dim)
    f = RNG.standard_normal((nc,) + (n,) * dim)
    g = RNG.standard_normal((nc,) + (n,) * dim)
    Gf, Gg = O.projection_G(f, dim, n), O.projection_G(g, dim, n)
    scale = np.abs(Gf).max()
    assert np.abs(O.projection_G(Gf, dim, n) - Gf).max() < 1e-12 * scale
    assert abs(np.sum(Gf * g) - np.sum(f * Gg)) < 1e-10 * np.sqrt(np.sum(f * f) * np.sum(g * g))
    spec = np.fft.fftn(Gf, axes=tuple(range(-dim, 0)))
    assert np.abs(spec[:, O.nyquist_mask(dim, n)]).max() < 1e-11 * np.abs(spec).max()
    assert np.abs(spec[(slice(None),) + (0,) * dim]).max() < 1e-11 * np.abs(spec).max()


def test_equilibrium_errors_on_even_grids():
    n, A = 16, 0.3
    x = (np.arange(n) + 0.5) / n
    s = np.zeros((3, n, n))
    s[0] = 1.0 + A * np.cos(2 * math.pi * x)[None, :]
    e, e_n = O.equilibrium_errors(np.fft.fftn(s, axes=(-2, -1)), 2, n)
    assert abs(e - math.sqrt(2) * math.pi * A) < 1e-12
    assert abs(e_n - A / math.sqrt(2)) < 1e-12
    # variation only at the Nyquist frequency along x (sin(pi n x) = +-1 at the voxel centres): left
    # out, so e = e_n = 0
    s2 = np.zeros((3, n, n))
    s2[0] = 1.0 + A * np.sin(math.pi * n * x)[None, :]
    assert np.abs(np.fft.fft(s2[0, 0])[n // 2]) > 0.1 * n
    e, e_n = O.equilibrium_errors(np.fft.fftn(s2, axes=(-2, -1)), 2, n)
    assert e < 1e-13 and e_n < 1e-13


def test_homogeneous_even_cell():
    ct = O.filter_build(H.homogeneous_cell(8, 2), H.two_phases(10.0))["ctilde"]
    lam0, mu0 = O.default_reference(H.two_phases(10.0))
    r = O.solve_one(ct, 2, 8, lam0, mu0, np.array([0.2, 0.1, -0.3]), tol=1e-12, max_iter=10)
    assert r["iterations"] == 0
    np.testing.assert_allclose(r["eps"][:, 3, 5], [0.2, 0.1, -0.3], atol=1e-15)


def test_fixed_point_and_cg_agree_on_an_even_grid():
    cell = H.centred_disk_cell(16, rule=H.RULE_VOIGT)
    ph = H.two_phases(20.0)
    ct = O.filter_build(cell, ph)["ctilde"]
    lam0, mu0 = O.default_reference(ph)
    fp = O.solve(ct, 2, 16, lam0, mu0, np.eye(3), tol=1e-12, max_iter=5000)
    cg = O.solve_cg(ct, 2, 16, np.eye(3), tol=1e-12, max_iter=500)
    assert np.abs(fp["eps"] - cg["eps"]).max() < 1e-10 * np.abs(fp["eps"]).max()


def test_two_layer_c11_at_32_between_odd_neighbours():
    ph = H.two_phases(10.0)
    lam0, mu0 = O.default_reference(ph)
    c11 = {}
    for n in (31, 32, 33):
        cell = H.centred_disk_cell(n, rule=H.RULE_TWO_LAYER, radius=math.pi / 15)
        ct = O.filter_build(cell, ph)["ctilde"]
        r = O.solve_one(ct, 2, n, lam0, mu0, np.array([1.0, 0.0, 0.0]), tol=1e-10, max_iter=3000)
        c11[n] = r["mean_sigma"][0]
    assert min(c11[31], c11[33]) < c11[32] < max(c11[31], c11[33]), c11
