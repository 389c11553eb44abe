"""Pins of the oracle's transform, Mandel and Green-operator layers (section 2, eq. 2 and the
odd frequency set J).  Every expected value here is a closed form or an identity of the
continuum operator, not a re-run of the oracle's own formula."""
import math

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(12345)


@pytest.mark.parametrize("n", [3, 5, 9, 15, 25, 27, 45])
def test_naive_dft_matches_fft_1d(n):
    x = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    X = O.naive_dft(x, axes=[0])
    np.testing.assert_allclose(X, np.fft.fft(x), rtol=0, atol=1e-12 * n)
    # inverse direction and round trip
    y = O.naive_dft(X, axes=[0], sign=+1) / n
    np.testing.assert_allclose(y, x, atol=1e-12 * n)


@pytest.mark.parametrize("shape", [(5, 9), (3, 5, 7), (9, 9, 9)])
def test_naive_dft_matches_fft_nd(shape):
    x = RNG.standard_normal(shape)
    X = O.naive_dft(x, axes=range(len(shape)))
    np.testing.assert_allclose(X, np.fft.fftn(x), atol=1e-10)
    # Hermitian symmetry of a real input (what the half-spectrum storage relies on)
    flip = X[np.ix_(*[(-np.arange(s)) % s for s in shape])]
    np.testing.assert_allclose(X, np.conj(flip), atol=1e-10)
    # Parseval
    assert abs(np.sum(np.abs(X) ** 2) / x.size - np.sum(x ** 2)) < 1e-9 * np.sum(x ** 2)


def test_signed_frequencies():
    for n in [3, 5, 45, 1215]:
        a = O.signed_frequencies(n)
        assert sorted(a.tolist()) == list(range(-(n - 1) // 2, (n - 1) // 2 + 1))
        # bin m and bin n-m are opposite frequencies (conjugate pairs)
        assert np.all(a[1:] == -a[1:][::-1])
        assert not O.nyquist_mask(2, n).any()
    for n in [4, 8, 30]:
        a = O.signed_frequencies(n)
        assert sorted(a.tolist()) == list(range(-n // 2 + 1, n // 2 + 1))
        m = O.nyquist_mask(2, n)
        assert m.sum() == 2 * n - 1 and m[n // 2, 0] and m[0, n // 2] and not m[1, 1]


@pytest.mark.parametrize("dim", [2, 3])
def test_mandel_round_trip_and_inner_product(dim):
    nc = O.nc_of(dim)
    A = RNG.standard_normal((4, dim, dim))
    A = A + np.swapaxes(A, -1, -2)
    B = RNG.standard_normal((4, dim, dim))
    B = B + np.swapaxes(B, -1, -2)
    a, b = O.tensor2_to_mandel(A, dim), O.tensor2_to_mandel(B, dim)
    assert a.shape == (4, nc)
    np.testing.assert_allclose(O.mandel_to_tensor2(a, dim), A, atol=1e-14)
    # Mandel vectors preserve the double contraction A:B
    np.testing.assert_allclose(np.sum(a * b, -1), np.einsum("pij,pij->p", A, B), atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_isotropic_mandel_closed_form(dim):
    lam, mu = 1.7, 0.9
    C = O.isotropic_mandel(lam, mu, dim)
    nc = O.nc_of(dim)
    expect = 2.0 * mu * np.eye(nc)
    expect[:dim, :dim] += lam
    np.testing.assert_allclose(C, expect, atol=1e-14)
    # Mandel matrix <-> tensor round trip keeps minor symmetries
    T = O.mandel_to_tensor4(C, dim)
    np.testing.assert_allclose(T, O.isotropic_tensor(lam, mu, dim), atol=1e-14)


def _ddot(A, B):
    """(A:B)_ijkl = A_ijmn B_mnkl."""
    return np.einsum("ijmn,mnkl->ijkl", A, B)


@pytest.mark.parametrize("dim", [2, 3])
def test_gamma0_identities(dim):
    lam0, mu0 = 2.3, 0.7
    C0 = O.isotropic_tensor(lam0, mu0, dim)
    for _ in range(10):
        xi = RNG.standard_normal(dim) * 7.0
        G = O.gamma0_tensor(xi, lam0, mu0)
        # projection: Gamma0 : c0 : Gamma0 = Gamma0
        np.testing.assert_allclose(_ddot(_ddot(G, C0), G), G, atol=1e-12)
        # compatible strains are reproduced: Gamma0 : c0 : sym(xi (x) v) = sym(xi (x) v)
        v = RNG.standard_normal(dim)
        e = 0.5 * (np.outer(xi, v) + np.outer(v, xi))
        np.testing.assert_allclose(np.einsum("khij,ij->kh", _ddot(G, C0), e), e, atol=1e-12)
        # equilibrium: xi . (c0 : Gamma0 : tau) = xi . tau  for every symmetric tau
        tau = RNG.standard_normal((dim, dim))
        tau = tau + tau.T
        s = np.einsum("ijkl,kl->ij", C0, np.einsum("khij,ij->kh", G, tau))
        np.testing.assert_allclose(s @ xi, tau @ xi, atol=1e-12)
        # tau with tau.xi = 0 is annihilated
        if dim == 2:
            t = np.array([-xi[1], xi[0]])
        else:
            t = np.cross(xi, RNG.standard_normal(3))
        tau0 = np.outer(t, t)
        np.testing.assert_allclose(np.einsum("khij,ij->kh", G, tau0), 0.0, atol=1e-12)
        # major and minor symmetries
        np.testing.assert_allclose(G, np.transpose(G, (2, 3, 0, 1)), atol=1e-14)
        np.testing.assert_allclose(G, np.transpose(G, (1, 0, 2, 3)), atol=1e-14)
        np.testing.assert_allclose(G, np.transpose(G, (0, 1, 3, 2)), atol=1e-14)
        # homogeneous of degree 0 and even in xi
        np.testing.assert_allclose(O.gamma0_tensor(3.1 * xi, lam0, mu0), G, atol=1e-13)
        np.testing.assert_allclose(O.gamma0_tensor(-xi, lam0, mu0), G, atol=1e-13)


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_apply_gamma0_on_compatible_fields(dim, n):
    """-Gamma0 : (c0 : eps_hat) = -eps_hat for compatible eps_hat = sym(xi (x) u), k != 0."""
    lam0, mu0 = 1.3, 0.6
    xi = O.wave_vectors(dim, n)
    u = RNG.standard_normal(xi.shape) + 1j * RNG.standard_normal(xi.shape)
    e = 0.5 * (xi[..., :, None] * u[..., None, :] + u[..., :, None] * xi[..., None, :])
    C0 = O.isotropic_mandel(lam0, mu0, dim)
    em = np.moveaxis(O.tensor2_to_mandel(e, dim), -1, 0)
    s = np.einsum("IJ,J...->I...", C0, em)
    out = O.apply_gamma0(s, dim, n, lam0, mu0)
    zero = (slice(None),) + (0,) * dim
    em[zero] = 0.0
    np.testing.assert_allclose(out, -em, atol=1e-10)


def test_equilibrium_error_closed_form():
    """sigma_11(x) = 1 + A cos(2 pi x): ||div sigma||_L2 = sqrt(2) pi A, <sigma> = e1 (x) e1, so
    e = sqrt(2) pi A; with the unit wave vector, e_n = A / sqrt(2)."""
    n, A = 15, 0.3
    x = (np.arange(n) + 0.5) / n
    s = np.zeros((3, n, n))
    s[0] = 1.0 + A * np.cos(2 * math.pi * x)[None, :]
    e, e_n = O.equilibrium_errors(np.fft.fftn(s, axes=(-2, -1)), 2, n)
    assert abs(e - math.sqrt(2) * math.pi * A) < 1e-12
    assert abs(e_n - A / math.sqrt(2)) < 1e-12
    # an equilibrated field: sigma_12 depends on nothing, sigma_11 varies only along y
    s2 = np.zeros((3, n, n))
    s2[0] = 1.0 + np.sin(2 * math.pi * x)[:, None]
    e, e_n = O.equilibrium_errors(np.fft.fftn(s2, axes=(-2, -1)), 2, n)
    assert e < 1e-13 and e_n < 1e-13
