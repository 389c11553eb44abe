"""Pins of the oracle's modified discrete Green operator (the "rotated" finite-difference scheme; the
paper's introduction names such operators, refs. [1, 11], as the second way to improve the basic
method).  The wave vector it substitutes for xi is pinned against a real-space construction of the
scheme written out independently here: strains are symmetric finite differences of a displacement
held at the voxel corners, each derivative averaged over the cell edges along its axis."""
import itertools

import numpy as np
import pytest

import hom_inputs as H
import oracle as O
from closed_forms import axis_permutation, backus, isotropic_mandel

ROT = O.SCHEME_ROTATED


def _fd_strain(u, n):
    """Rotated finite-difference strain at the voxel centres of a periodic n^d grid from the corner
    displacement u [d, *grid] (numpy axis order (z,) y, x; corner b of voxel a is node a + b).
    d_j u_i at voxel a = mean over the 2^(d-1) edges of the voxel along axis j of
    (u_i(end) - u_i(start)) / h.  Returns the Mandel strain [nc, *grid]."""
    d = u.shape[0]
    h = 1.0 / n
    grad = np.zeros((d, d) + u.shape[1:])  # grad[i, j] = d_j u_i

    def shift(f, offs):  # f at node a + offs (component j of offs moves axis j; numpy axis d-1-j)
        for j, o in enumerate(offs):
            if o:
                f = np.roll(f, -o, axis=d - 1 - j)
        return f

    for j in range(d):
        others = [m for m in range(d) if m != j]
        for corner in itertools.product((0, 1), repeat=d - 1):
            start = [0] * d
            for m, c in zip(others, corner):
                start[m] = c
            end = list(start)
            end[j] = 1
            for i in range(d):
                grad[i, j] += (shift(u[i], end) - shift(u[i], start)) / h
        grad[:, j] /= 2 ** (d - 1)
    eps = 0.5 * (grad + np.swapaxes(grad, 0, 1))
    return O.tensor2_to_mandel(np.moveaxis(eps, (0, 1), (-2, -1)), d).transpose((d,) + tuple(range(d)))


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 8), (3, 5), (3, 6)])
def test_rotated_operator_reproduces_finite_difference_strains(dim, n):
    """Gamma0 at the rotated wave vector maps c0 : eps back to eps (minus its mean) for every strain
    that is a rotated finite-difference gradient, and the continuous operator does not (at n = 4 the
    two coincide on the non-Nyquist bins, where every q is parallel to xi, so n >= 5 here)."""
    rng = np.random.default_rng(dim * 100 + n)
    u = rng.standard_normal((dim,) + (n,) * dim)
    eps = _fd_strain(u, n)
    lam0, mu0 = 1.3, 0.7
    nc = O.nc_of(dim)
    C0 = isotropic_mandel(lam0, mu0, dim)
    tau_hat = O._fft(np.einsum("IJ,J...->I...", C0, eps), dim)
    keep = ~O.nyquist_mask(dim, n)  # even grids: the operator zeroes the Nyquist bins
    want = O._fft(eps, dim)
    zero = (slice(None),) + (0,) * dim
    want[zero] = 0.0
    for scheme, agrees in ((ROT, True), (O.SCHEME_CONTINUOUS, False)):
        got = -O.apply_gamma0(tau_hat, dim, n, lam0, mu0, scheme=scheme)
        diff = np.abs(got - want)[:, keep].max() / np.abs(want).max()
        assert (diff < 1e-12) == agrees, (scheme, diff)
        assert nc == got.shape[0]


@pytest.mark.parametrize("dim,n", [(2, 11), (3, 5)])
def test_rotated_operator_is_an_orthogonal_projection(dim, n):
    """Gamma0(q) : c0 is idempotent on random fields and self-adjoint for the c0 inner product."""
    rng = np.random.default_rng(n)
    nc = O.nc_of(dim)
    lam0, mu0 = 0.9, 1.1
    C0 = isotropic_mandel(lam0, mu0, dim)
    a = O._fft(rng.standard_normal((nc,) + (n,) * dim), dim)
    b = O._fft(rng.standard_normal((nc,) + (n,) * dim), dim)

    def P(x):  # eps_hat -> Gamma0 : c0 : eps_hat
        return -O.apply_gamma0(np.einsum("IJ,J...->I...", C0, x), dim, n, lam0, mu0, scheme=ROT)
    Pa = P(a)
    np.testing.assert_allclose(P(Pa), Pa, atol=1e-12 * np.abs(Pa).max())
    lhs = np.sum(np.conj(np.einsum("IJ,J...->I...", C0, P(a))) * b)
    rhs = np.sum(np.conj(np.einsum("IJ,J...->I...", C0, a)) * P(b))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_rotated_wave_vector_closed_form_points():
    """q at a few bins, written out: 2D n = 9, a = (1, 2): q_x = 18 sin(pi/9) cos(2 pi/9),
    q_y = 18 cos(pi/9) sin(2 pi/9); axis bins reduce to the one-sided difference 2n sin(pi a / n)."""
    q = O.wave_vectors(2, 9, ROT)
    s, c = np.sin, np.cos
    np.testing.assert_allclose(q[2, 1], [18 * s(np.pi / 9) * c(2 * np.pi / 9), 18 * c(np.pi / 9) * s(2 * np.pi / 9)],
                               rtol=1e-15)
    np.testing.assert_allclose(q[0, 3], [18 * s(3 * np.pi / 9), 0.0], atol=1e-14)
    np.testing.assert_allclose(q[7, 0], [0.0, 18 * s(-2 * np.pi / 9)], atol=1e-14)  # bin 7 = a -2


@pytest.mark.parametrize("dim,n,m,axis", [(2, 15, 4, 1), (2, 9, 5, 0), (3, 7, 3, 2)])
def test_rotated_scheme_grid_aligned_laminate_is_exact(dim, n, m, axis):
    """Piecewise-constant strains along the laminate normal are finite-difference compatible and
    the stress is equilibrated, so the rotated scheme solves the grid-aligned laminate exactly."""
    ph = H.two_phases(10.0)
    nc = O.nc_of(dim)
    centre = 0.5 if m % 2 == 1 else 0.5 + 0.5 / n
    cell = H.laminate_cell(n, dim, m / n, axis=axis, centre=centre)
    ct = O.filter_build(cell, ph)["ctilde"]
    lam0, mu0 = O.default_reference(ph)
    r = O.solve(ct, dim, n, lam0, mu0, np.eye(nc), tol=1e-12, max_iter=3000, scheme=ROT)
    assert all(st == "converged" for st in r["status"])
    C = O.effective_stiffness(r["mean_sigma"], np.eye(nc))
    p = axis_permutation(dim, axis)
    expect = backus(dim, m / n, ph)[np.ix_(p, p)]
    np.testing.assert_allclose(C, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


def test_rotated_scheme_disk_between_bounds_and_symmetric():
    """The disk cell under the rotated scheme: C_eff symmetric and between the grid-field bounds
    <c~^-1>^-1 <= C_eff <= <c~>, like the continuous scheme's (same discrete energy principle)."""
    cell = H.centred_disk_cell(21, rule=H.RULE_VOIGT)
    ph = H.two_phases(10.0)
    ct = O.filter_build(cell, ph)["ctilde"]
    lam0, mu0 = O.default_reference(ph)
    r = O.solve(ct, 2, 21, lam0, mu0, np.eye(3), tol=1e-11, max_iter=3000, scheme=ROT)
    C = O.effective_stiffness(r["mean_sigma"], np.eye(3))
    assert np.abs(C - C.T).max() < 1e-9 * np.abs(C).max()
    cv = ct.reshape(-1, 3, 3)
    upper = cv.mean(axis=0)
    lower = np.linalg.inv(np.linalg.inv(cv).mean(axis=0))
    assert np.linalg.eigvalsh(upper - C).min() > -1e-9
    assert np.linalg.eigvalsh(C - lower).min() > -1e-9
