"""Pins of the oracle's filter layer: refined-grid volume fractions (section 2) and the Voigt,
Reuss and 2-layer homogenisation rules (eqs. 3, 4, 5).  Expected values are closed forms
(Backus laminate averages, circular-segment and lens areas, Loewner bounds) or brute force."""
import math

import numpy as np
import pytest

import hom_inputs as H
import oracle as O

RNG = np.random.default_rng(777)


def test_sample_count_close_to_ball_volume():
    for dim, S, r in [(2, 16, 1.0), (2, 16, 0.55), (3, 8, 1.0), (2, 8, 1.5)]:
        M = O.sample_offsets(dim, r, S).shape[0]
        vol = math.pi * (S * r) ** 2 if dim == 2 else 4.0 / 3.0 * math.pi * (S * r) ** 3
        surf = 2 * math.pi * S * r if dim == 2 else 4 * math.pi * (S * r) ** 2
        assert abs(M - vol) < surf, (dim, S, r, M, vol)
    # 2D, r = 1, S = 16: the ball holds about 804 fine points
    assert abs(O.sample_offsets(2, 1.0, 16).shape[0] - 804) <= 20


def test_sample_offsets_are_symmetric():
    for dim, S, r in [(2, 16, 1.0), (3, 8, 0.55), (2, 5, 1.0)]:
        t = O.sample_offsets(dim, r, S)
        D = 2 * t + 1 - S
        s = set(map(tuple, D.tolist()))
        assert all(tuple(-d for d in v) in s for v in s)


def _lens_area(R, r, d):
    """Area of the intersection of disks of radii R, r with centre distance d."""
    if d >= R + r:
        return 0.0
    if d <= abs(R - r):
        return math.pi * min(R, r) ** 2
    a = r * r * math.acos((d * d + r * r - R * R) / (2 * d * r))
    b = R * R * math.acos((d * d + R * R - r * r) / (2 * d * R))
    c = 0.5 * math.sqrt((-d + r + R) * (d + r - R) * (d - r + R) * (d + r + R))
    return a + b - c


def test_disk_fractions_match_lens_area():
    """Sampled inclusion fraction of every mixed voxel vs the exact disk-ball lens area."""
    n, S, rpx = 15, 16, 1.0
    cell = H.centred_disk_cell(n, radius=0.31, rule=H.RULE_VOIGT, radius_px=rpx, subgrid=S)
    counts, M = O.volume_fraction_counts(cell, 2)
    h = 1.0 / n
    worst = 0.0
    for iy in range(n):
        for ix in range(n):
            c = counts[iy, ix]
            x = np.array([(ix + 0.5) * h, (iy + 0.5) * h])
            d = float(np.linalg.norm(x - 0.5))
            exact = _lens_area(0.31, rpx * h, d) / (math.pi * (rpx * h) ** 2)
            worst = max(worst, abs(c[1] / M - exact))
    assert worst < 4.0 / S, worst


def test_slab_fraction_matches_segment_area():
    """A slab face crossing the ball at signed distance delta from its centre: the fraction on
    the far side is the circular segment (2D) / spherical cap (3D) volume fraction."""
    for dim, S in [(2, 16), (3, 8)]:
        n = 9
        for off in [0.13, 0.37, 0.5, 0.71]:
            # slab from the cell centre plane + off*h to far away: face crossing voxel (4, ...)
            thick = 0.4
            centre = (4 + 0.5 + off) / n + thick / 2
            cell = H.laminate_cell(n, dim, thick, axis=0, centre=centre, rule=H.RULE_VOIGT,
                                   radius_px=1.0, subgrid=S)
            counts, M = O.volume_fraction_counts(cell, 2)
            frac = counts[(0,) * (dim - 1) + (4,)][1] / M
            u = off  # distance of the face from the voxel centre in units of the ball radius
            if dim == 2:
                exact = (math.acos(u) - u * math.sqrt(1 - u * u)) / math.pi
            else:
                exact = (1 - u) ** 2 * (2 + u) / 4.0
            assert abs(frac - exact) < 0.25 / S, (dim, off, frac, exact)


@pytest.mark.parametrize("dim,n,cellmaker", [
    (2, 9, lambda: H.centred_disk_cell(9, radius=0.23, rule=H.RULE_REUSS, radius_px=1.0, subgrid=6)),
    (2, 7, lambda: H.laminate_cell(7, 2, 0.33, axis=1, centre=0.41, rule=H.RULE_VOIGT, radius_px=0.55, subgrid=5)),
    (3, 5, lambda: H.rsa_spheres_cell(5, seed=3, vf=0.1, rmin=0.12, rmax=0.16, radius_px=1.0, subgrid=4, gap_voxels=0.2)),
])
def test_pruned_counts_equal_brute_force(dim, n, cellmaker):
    cell = cellmaker()
    a, Ma = O.volume_fraction_counts(cell, 2, brute_force=False)
    b, Mb = O.volume_fraction_counts(cell, 2, brute_force=True)
    assert Ma == Mb
    np.testing.assert_array_equal(a, b)


def test_point_sample_ties_count_inside():
    """Grid points exactly on a slab face or a circle belong to the inclusion; a hair less
    thickness drops them."""
    n = 9
    ph = H.two_phases(10.0)
    C1 = O.isotropic_mandel(*ph[1], 2)
    for half, expect in [(2.0 / n, 5), ((2.0 - 1e-9) / n, 3), (2.5 / n, 5)]:
        cell = H.laminate_cell(n, 2, 2 * half, axis=0, centre=0.5, rule=H.RULE_NONE)
        ct = O.filter_build(cell, ph)["ctilde"]
        inside = np.all(ct[0] == C1, axis=(-1, -2))
        assert inside.sum() == expect, (half, inside)
    # disk of radius 0.2 centred at 0.5 on a 5-grid: the 4 axis neighbours sit on the circle
    cell = H.centred_disk_cell(5, radius=0.2, rule=H.RULE_NONE)
    ct = O.filter_build(cell, ph)["ctilde"]
    inside = np.all(ct == C1, axis=(-1, -2))
    assert inside.sum() == 5 and inside[2, 1] and inside[1, 2] and not inside[1, 1]


def test_point_sample_inclusion_area():
    n = 135
    R = math.sqrt(0.2 / math.pi)
    cell = H.centred_disk_cell(n, radius=R, rule=H.RULE_NONE)
    fb = O.filter_build(cell, H.two_phases(10.0))
    C1 = O.isotropic_mandel(*H.two_phases(10.0)[1], 2)
    inside = np.all(np.isclose(fb["ctilde"], C1), axis=(-1, -2))
    assert abs(inside.mean() - 0.2) < 2 * math.pi * R / n


# ---------------------------------------------------------------------------- rules


def _phases(dim, contrast=10.0):
    return [O.isotropic_mandel(*p, dim) for p in H.two_phases(contrast)]


def _backus(dim, f, contrast=10.0):
    """Closed-form laminate stiffness (normal e1) of two isotropic phases (Backus averages)."""
    ph = H.two_phases(contrast)
    lam = np.array([p[0] for p in ph])
    mu = np.array([p[1] for p in ph])
    M = lam + 2 * mu
    w = np.array([1 - f, f])
    av = lambda a: float(np.sum(w * a))  # noqa: E731
    c11 = 1 / av(1 / M)
    c12 = av(lam / M) / av(1 / M)
    c22 = av(M - lam ** 2 / M) + av(lam / M) ** 2 / av(1 / M)
    gout = 2 / av(1 / mu)      # Mandel shear with one index along the normal
    if dim == 2:
        return np.array([[c11, c12, 0], [c12, c22, 0], [0, 0, gout]])
    c23 = av(lam - lam ** 2 / M) + av(lam / M) ** 2 / av(1 / M)
    gin = 2 * av(mu)           # Mandel in-plane shear (23)
    C = np.zeros((6, 6))
    C[0, 0] = c11
    C[0, 1] = C[1, 0] = C[0, 2] = C[2, 0] = c12
    C[1, 1] = C[2, 2] = c22
    C[1, 2] = C[2, 1] = c23
    C[3, 3] = gin
    C[4, 4] = C[5, 5] = gout
    return C


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("f", [0.0, 0.2, 0.5, 0.93, 1.0])
def test_two_layer_normal_e1_is_backus(dim, f):
    C0, C1 = _phases(dim)
    got = O.hr_two_layer(C0, C1, 1 - f, f, np.eye(dim)[0], dim)
    np.testing.assert_allclose(got, _backus(dim, f), atol=1e-12)


def test_two_layer_axis_permutation():
    """Normal e2 (2D) / e3 (3D) is the normal-e1 laminate with the axes relabelled."""
    f = 0.37
    C0, C1 = _phases(2)
    a = O.hr_two_layer(C0, C1, 1 - f, f, np.array([0.0, 1.0]), 2)
    p = [1, 0, 2]
    np.testing.assert_allclose(a, _backus(2, f)[np.ix_(p, p)], atol=1e-12)
    C0, C1 = _phases(3)
    b = O.hr_two_layer(C0, C1, 1 - f, f, np.array([0.0, 0.0, 1.0]), 3)
    # axes (x, y, z) -> (z, y, x): Mandel (11,22,33,23,13,12) -> (33,22,11,21,31,32)
    p3 = [2, 1, 0, 5, 4, 3]
    np.testing.assert_allclose(b, _backus(3, f)[np.ix_(p3, p3)], atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_rules_pure_and_equal_phases(dim):
    C0, C1 = _phases(dim)
    nrm = RNG.standard_normal(dim)
    for rule in (O.hr_voigt, O.hr_reuss):
        np.testing.assert_allclose(rule([C0, C1], [1.0, 0.0]), C0, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(rule([C1, C1], [0.3, 0.7]), C1, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(O.hr_two_layer(C0, C1, 0.0, 1.0, nrm, dim), C1, atol=1e-12)
    np.testing.assert_allclose(O.hr_two_layer(C1, C1, 0.4, 0.6, nrm, dim), C1, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_loewner_order_reuss_two_layer_voigt(dim):
    for contrast in (1e-3, 0.1, 10.0, 1e3):
        C0, C1 = _phases(dim, contrast)
        for _ in range(10):
            f = float(RNG.uniform(0.01, 0.99))
            nrm = RNG.standard_normal(dim)
            v = O.hr_voigt([C0, C1], [1 - f, f])
            r = O.hr_reuss([C0, C1], [1 - f, f])
            t = O.hr_two_layer(C0, C1, 1 - f, f, nrm, dim)
            sc = np.abs(v).max()
            assert np.linalg.eigvalsh(v - t).min() > -1e-11 * sc
            assert np.linalg.eigvalsh(t - r).min() > -1e-11 * sc
            np.testing.assert_allclose(t, t.T, atol=1e-12 * sc)


def test_two_layer_satisfies_interface_conditions():
    """For a random macroscopic strain the 2-layer stiffness has phase strains that are
    continuous in-plane with continuous traction (eqs. 5-a/5-b) -- checked in the global
    frame through the Hadamard jump form: eps1 - eps2 = sym(n (x) a), (sig1 - sig2) n = 0."""
    dim = 3
    C0, C1 = _phases(dim)
    nrm = RNG.standard_normal(3)
    nrm /= np.linalg.norm(nrm)
    f = 0.3
    Ct = O.hr_two_layer(C0, C1, 1 - f, f, nrm, dim)
    T0, T1 = O.mandel_to_tensor4(C0, 3), O.mandel_to_tensor4(C1, 3)
    E = RNG.standard_normal((3, 3))
    E = E + E.T
    def sym(a):
        return 0.5 * (np.outer(nrm, a) + np.outer(a, nrm))
    # phase 1 (fraction f) strain = E + (1-f) sym(n a), phase 0 = E - f sym(n a): the mean is E
    # and the in-plane strain is continuous; traction continuity (s1 - s0) n = 0 fixes a.
    rhs = -(np.einsum("ijkl,kl->ij", T1 - T0, E) @ nrm)
    K = np.zeros((3, 3))
    for m in range(3):
        a = np.eye(3)[m]
        s1 = np.einsum("ijkl,kl->ij", T1, (1 - f) * sym(a))
        s0 = np.einsum("ijkl,kl->ij", T0, -f * sym(a))
        K[:, m] = (s1 - s0) @ nrm
    a = np.linalg.solve(K, rhs)
    e1 = E + (1 - f) * sym(a)
    e0 = E - f * sym(a)
    sig = f * np.einsum("ijkl,kl->ij", T1, e1) + (1 - f) * np.einsum("ijkl,kl->ij", T0, e0)
    got = O.mandel_to_tensor2(Ct @ O.tensor2_to_mandel(E, 3), 3)
    np.testing.assert_allclose(got, sig, atol=1e-11)


def test_filter_build_pure_voxels_are_exact():
    cell = H.centred_disk_cell(45, rule=H.RULE_REUSS, radius_px=1.0, subgrid=16)
    ph = H.two_phases(10.0)
    fb = O.filter_build(cell, ph)
    Cs = [O.isotropic_mandel(*p, 2) for p in ph]
    ct = fb["ctilde"].reshape(-1, 3, 3)
    mixed = fb["mixed"].ravel()
    for v in np.nonzero(~mixed)[0][::37]:
        assert any(np.array_equal(ct[v], C) for C in Cs)
    # mixed voxels lie within one filter radius of the circle
    n = 45
    ys, xs = np.nonzero(fb["mixed"])
    d = np.hypot((xs + 0.5) / n - 0.5, (ys + 0.5) / n - 0.5) - math.sqrt(0.2 / math.pi)
    assert np.all(np.abs(d) <= 1.0 / n + 1e-9)
    assert mixed.sum() > 0


def test_n_within_picks_the_first_resolution_that_stays_in_band():
    """N_1% logic of the resolution study (section 3): the smallest n after which every larger
    resolution stays within 1 % of the converged value."""
    from paper_1412_3228_gb300.experiments import n_within
    sizes = [9, 15, 21, 27, 45]
    assert n_within(sizes, [1.5, 1.0, 1.02, 0.995, 1.001], 1.0) == 27   # 21 is outside the band
    assert n_within(sizes, [1.005, 0.995, 1.0, 1.0, 1.0], 1.0) == 9
    assert n_within(sizes, [1.0, 1.0, 1.0, 1.0, 1.2], 1.0) is None     # the last point misses
    assert n_within(list(reversed(sizes)), [1.001, 0.995, 1.02, 1.0, 1.5], 1.0) == 27  # order-free
