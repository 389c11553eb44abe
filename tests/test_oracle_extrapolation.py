"""Pins of the oracle's Fourier extrapolation of c~ (section 6, Fig. 4) against facts fixed by the
mathematics and by the paper, none of which re-types the oracle's FFT-and-series formula:

* the Dirichlet-kernel interpolation sum, evaluated point by point on tiny grids;
* interpolation: where a fine point coincides with a grid point, the series returns the grid value;
* a single Fourier mode of J is reproduced everywhere (closed form);
* the fine-grid mean equals the grid mean (every non-zero frequency of J sums to zero on the finer
  grid);
* the exact (point-sampled) property of a slab, closed form at every fine point;
* Fig. 4's statement for the Voigt filter: the extrapolated property overshoots the phase range less
  as the radius grows (none > 0.55 > 1.0), and the gap to the exact microstructure is smallest at
  0.55 among the radii 0.3, 0.55, 1.0, 1.5.
"""
import math

import numpy as np
import pytest

import hom_inputs as H
import oracle as O


def dirichlet_sum(field, dim, n, m):
    """f(y) = sum_a c(x_a) prod_d sin(n pi t_d) / (n sin(pi t_d)), t = y - x_a, by brute force."""
    x = (np.arange(n) + 0.5) / n
    y = (np.arange(m) + 0.5) / m

    def D(t):
        s = np.sin(np.pi * t)
        with np.errstate(invalid="ignore", divide="ignore"):
            v = np.sin(n * np.pi * t) / (n * s)
        return np.where(np.abs(s) < 1e-14, 1.0, v)

    out = np.zeros((m,) * dim)
    for a in np.ndindex(*((n,) * dim)):
        w = np.ones((m,) * dim)
        for ax in range(dim):
            shape = [1] * dim
            shape[ax] = m
            w = w * D(y - x[a[ax]]).reshape(shape)
        out += field[a] * w
    return out


@pytest.mark.parametrize("dim,n,m", [(2, 5, 15), (2, 7, 11), (2, 9, 4), (3, 3, 7), (3, 5, 5)])
def test_matches_dirichlet_interpolation_sum(dim, n, m):
    rng = np.random.default_rng(100 * dim + n + m)
    field = rng.standard_normal((n,) * dim)
    got = O.fourier_extrapolate(field, dim, n, m)
    want = dirichlet_sum(field, dim, n, m)
    assert np.abs(got - want).max() < 1e-12 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("dim,n,k", [(2, 9, 3), (2, 15, 5), (3, 5, 3)])
def test_interpolates_grid_values(dim, n, k):
    rng = np.random.default_rng(n * k)
    field = rng.uniform(1.0, 2.0, (n,) * dim)
    f = O.fourier_extrapolate(field, dim, n, k * n)
    # y_b = x_a for b = k a + (k - 1)/2 (k odd)
    sl = tuple(slice((k - 1) // 2, None, k) for _ in range(dim))
    assert np.abs(f[sl] - field).max() < 1e-12


def test_same_grid_is_identity():
    rng = np.random.default_rng(3)
    field = rng.standard_normal((25, 25))
    assert np.abs(O.fourier_extrapolate(field, 2, 25, 25) - field).max() < 1e-12


@pytest.mark.parametrize("k1,k2,phi", [(0, 0, 0.3), (3, 0, 0.0), (-2, 4, 1.1), (4, -4, -0.7)])
def test_single_mode_is_reproduced(k1, k2, phi):
    n, m = 9, 31
    x = (np.arange(n) + 0.5) / n
    y = (np.arange(m) + 0.5) / m
    X, Y = np.meshgrid(x, x, indexing="xy")     # numpy order [y][x]
    field = np.cos(2 * np.pi * (k1 * X + k2 * Y) + phi)
    FX, FY = np.meshgrid(y, y, indexing="xy")
    want = np.cos(2 * np.pi * (k1 * FX + k2 * FY) + phi)
    assert np.abs(O.fourier_extrapolate(field, 2, n, m) - want).max() < 1e-12


@pytest.mark.parametrize("dim,n,m", [(2, 15, 16), (2, 15, 47), (3, 5, 6)])
def test_fine_mean_equals_grid_mean(dim, n, m):
    rng = np.random.default_rng(m)
    field = rng.uniform(0.0, 1.0, (n,) * dim)
    assert abs(O.fourier_extrapolate(field, dim, n, m).mean() - field.mean()) < 1e-13


def test_exact_property_area():
    """The point-sampled disk covers pi r^2 of the cell up to the fine grid's resolution."""
    cell = H.centred_disk_cell(25, radius=0.21)
    ex = O.exact_property(cell, [0.0, 1.0], 25 * 9)
    assert abs(ex.mean() - math.pi * 0.21 ** 2) < 4.0 * 2 * math.pi * 0.21 / (25 * 9)
    assert set(np.unique(ex)) == {0.0, 1.0}


@pytest.mark.parametrize("axis,centre,thickness", [(0, 0.43, 0.37), (1, 0.05, 0.3)])
def test_exact_property_of_a_slab_point_by_point(axis, centre, thickness):
    """The slab holds the fine voxel centres y = (b + 1/2)/m within thickness/2 of its centre
    (periodic distance): closed form at every point."""
    n, m = 9, 27
    cell = H.laminate_cell(n, 2, thickness, axis=axis, centre=centre)
    ex = O.exact_property(cell, [0.0, 1.0], m)
    y = (np.arange(m) + 0.5) / m
    d = np.abs(y - centre)
    inside = (np.minimum(d, 1.0 - d) <= thickness / 2).astype(float)
    want = inside[None, :] if axis == 0 else inside[:, None]
    np.testing.assert_array_equal(ex, np.broadcast_to(want, (m, m)))


def test_fig4_voigt_filter_reduces_oscillations():
    """Section 6, Fig. 4 (65^2 grid, disk of radius pi/15, contrast 1e-3): the overshoot of the
    extrapolated stiffness beyond the phase range decreases from no filter to radius 0.55 to radius
    1.0, and the L2 gap to the exact microstructure is smallest at radius 0.55 of (0.3, 0.55, 1.0, 1.5)."""
    n, m = 65, 325
    phases = H.two_phases(1e-3)
    vals = [lam + 2 * mu for lam, mu in phases]          # c_11 of each phase (Mandel)
    span = max(vals) - min(vals)
    over, gap = {}, {}
    for rule, r in [(H.RULE_NONE, 0.0), (H.RULE_VOIGT, 0.3), (H.RULE_VOIGT, 0.55), (H.RULE_VOIGT, 1.0),
                    (H.RULE_VOIGT, 1.5)]:
        cell = H.centred_disk_cell(n, rule=rule, radius_px=r if r else 1.0, subgrid=16, radius=math.pi / 15)
        c11 = O.filter_build(cell, phases)["ctilde"][..., 0, 0]
        f = O.fourier_extrapolate(c11, 2, n, m)
        over[r] = max(f.max() - max(vals), min(vals) - f.min()) / span
        gap[r] = np.sqrt(np.mean((f - O.exact_property(cell, vals, m)) ** 2)) / span
    assert over[0.0] > 1.5 * over[0.55] and over[0.55] > 2.0 * over[1.0], over
    assert min((0.3, 0.55, 1.0, 1.5), key=lambda r: gap[r]) == 0.55, gap
