"""Closed-form expected values used by the tests (independent of the oracle's code)."""
import numpy as np


def backus(dim, f, phases):
    """Stiffness (Mandel) of a laminate with normal e1 made of two isotropic phases
    [(lam, mu), (lam, mu)] with fraction f of the second one (Backus averages)."""
    lam = np.array([p[0] for p in phases])
    mu = np.array([p[1] for p in phases])
    M = lam + 2 * mu
    w = np.array([1 - f, f])

    def av(a):
        return float(np.sum(w * a))
    c11 = 1 / av(1 / M)
    c12 = av(lam / M) / av(1 / M)
    c22 = av(M - lam ** 2 / M) + av(lam / M) ** 2 / av(1 / M)
    gout = 2 / av(1 / mu)
    if dim == 2:
        return np.array([[c11, c12, 0], [c12, c22, 0], [0, 0, gout]])
    c23 = av(lam - lam ** 2 / M) + av(lam / M) ** 2 / av(1 / M)
    gin = 2 * av(mu)
    C = np.zeros((6, 6))
    C[0, 0] = c11
    C[0, 1] = C[1, 0] = C[0, 2] = C[2, 0] = c12
    C[1, 1] = C[2, 2] = c22
    C[1, 2] = C[2, 1] = c23
    C[3, 3] = gin
    C[4, 4] = C[5, 5] = gout
    return C


def axis_permutation(dim, axis):
    """Mandel index permutation that relabels axis `axis` as axis 0 (swap of two axes)."""
    if dim == 2:
        return [0, 1, 2] if axis == 0 else [1, 0, 2]
    if axis == 0:
        return list(range(6))
    if axis == 1:   # swap x <-> y: (11,22,33,23,13,12) -> (22,11,33,13,23,12)
        return [1, 0, 2, 4, 3, 5]
    return [2, 1, 0, 5, 4, 3]   # swap x <-> z


def isotropic_mandel(lam, mu, dim):
    nc = 3 if dim == 2 else 6
    C = 2.0 * mu * np.eye(nc)
    C[:dim, :dim] += lam
    return C


def hs_bulk_bounds_2d(phases, f):
    """Hashin-Shtrikman bounds on the plane-strain bulk modulus K = lam + mu of a two-phase
    2D composite (fraction f of phase 1), phases well ordered."""
    K = [p[0] + p[1] for p in phases]
    G = [p[1] for p in phases]
    fr = [1 - f, f]

    def hs(a, b):
        return K[a] + fr[b] / (1.0 / (K[b] - K[a]) + fr[a] / (K[a] + G[a]))
    soft, stiff = (0, 1) if K[0] < K[1] else (1, 0)
    return hs(soft, stiff), hs(stiff, soft)
