"""Plain, slow FP64 CPU oracle for FFT-based homogenisation with filtered material properties
(L. Gélébart and F. Ouaki, "Filtering material properties to improve FFT-based methods for
numerical homogenization", arXiv 1412.3228).

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA implementation.  Only the
test-suite, the smoke check and the CPU-baseline leg of the benchmark may import it; the
product library never calls it and has no CPU fallback.  It shares no code with the CUDA path:
the only module both sides import is `hom_inputs` (seeded geometry, no method arithmetic).

What it computes, in the paper's order:
  * section 2, eqs. (1-a)/(1-b): the Lippmann-Schwinger fixed point eps = -Gamma0 * tau + E,
    tau = (c - c0) : eps, iterated in the literal "tau form";
  * section 2, eq. (2): the Green operator applied in Fourier space on the truncated odd
    frequency set J, with eps_hat(0) = E;
  * section 2, eqs. (3), (4), (5-a), (5-b): the Voigt, Reuss and 2-layer homogenisation rules
    applied to phase volume fractions obtained by averaging indicator functions on a refined
    grid inside a ball of radius r pixels centred on each grid point;
  * the stress-equilibrium stopping criterion of Moulinec & Suquet (ref. [9] of the paper).

Readings where the paper is silent or garbled (each is listed in the design notes):
  * J is the integer range -(N-1)/2 .. (N-1)/2 per axis for odd N; on even grids (which the paper
    does not define) the Nyquist bins get zero strain and are left out of the equilibrium errors;
  * grid points are voxel centres x_a = (a + 1/2) h, h = 1/N, cell side 1;
  * eq. (5-b) reads f1 sigma1^P + f2 sigma2^P = sigma^P and f1 eps1^OP + f2 eps2^OP = eps^OP;
  * 2D is plane strain, all rules act on the 3x3 in-plane Mandel matrices;
  * the equilibrium error is e = sqrt(sum_k |xi_k . sigma_hat(k)|^2) / ||sigma_hat(0)||
    (unnormalised DFT, xi = 2 pi a); its normalised variant e_n uses xi/|xi| instead of xi;
  * filter samples sit on the global fine lattice (j + 1/2) h / S and a sample belongs to
    the ball when its distance to x_a is <= r h (ties inside).

Precision: float64 throughout.  The filter sampling uses the exact integer/FP64 recipe of
`_inside_primitive` so that an implementation following the same arithmetic gets identical
counts.

Parity status: every function is pinned by tests in tests/test_oracle_*.py (naive DFT,
Green-operator projection identities, Backus laminate closed forms, exact laminate solution,
homogeneous cell, Loewner ordering of the rules, analytic areas, bounds).  The disk/sphere
cells have no closed form: their solutions are pinned only through the invariants above.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

from hom_inputs import (PRIM_DISK, PRIM_SLAB, PRIM_SPHERE, RULE_NONE, RULE_REUSS, RULE_TWO_LAYER,
                        RULE_VOIGT, Cell)

SQRT2 = math.sqrt(2.0)

# =============================================================================================
# Mandel notation.  Strain/stress vectors hold (11, 22, sqrt2*12) in 2D and
# (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12) in 3D; stiffnesses are nc x nc Mandel matrices.


def mandel_pairs(dim: int) -> List[Tuple[int, int]]:
    if dim == 2:
        return [(0, 0), (1, 1), (0, 1)]
    return [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def mandel_weights(dim: int) -> np.ndarray:
    return np.array([1.0 if i == j else SQRT2 for (i, j) in mandel_pairs(dim)])


def nc_of(dim: int) -> int:
    return 3 if dim == 2 else 6


def tensor2_to_mandel(t: np.ndarray, dim: int) -> np.ndarray:
    """[..., d, d] symmetric tensor -> [..., nc] Mandel vector."""
    w = mandel_weights(dim)
    return np.stack([w[I] * t[..., i, j] for I, (i, j) in enumerate(mandel_pairs(dim))], axis=-1)


def mandel_to_tensor2(v: np.ndarray, dim: int) -> np.ndarray:
    """[..., nc] Mandel vector -> [..., d, d] symmetric tensor."""
    w = mandel_weights(dim)
    t = np.zeros(v.shape[:-1] + (dim, dim), dtype=v.dtype)
    for I, (i, j) in enumerate(mandel_pairs(dim)):
        t[..., i, j] = v[..., I] / w[I]
        t[..., j, i] = v[..., I] / w[I]
    return t


def tensor4_to_mandel(C: np.ndarray, dim: int) -> np.ndarray:
    """[..., d, d, d, d] tensor with minor symmetries -> [..., nc, nc] Mandel matrix."""
    w = mandel_weights(dim)
    P = mandel_pairs(dim)
    nc = len(P)
    M = np.zeros(C.shape[:-4] + (nc, nc), dtype=C.dtype)
    for I, (i, j) in enumerate(P):
        for J, (k, l) in enumerate(P):
            M[..., I, J] = w[I] * w[J] * C[..., i, j, k, l]
    return M


def mandel_to_tensor4(M: np.ndarray, dim: int) -> np.ndarray:
    w = mandel_weights(dim)
    P = mandel_pairs(dim)
    C = np.zeros(M.shape[:-2] + (dim,) * 4, dtype=M.dtype)
    for I, (i, j) in enumerate(P):
        for J, (k, l) in enumerate(P):
            val = M[..., I, J] / (w[I] * w[J])
            for (a, b) in {(i, j), (j, i)}:
                for (c, d) in {(k, l), (l, k)}:
                    C[..., a, b, c, d] = val
    return C


def isotropic_tensor(lam: float, mu: float, dim: int) -> np.ndarray:
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk); in 2D the indices run over the
    plane (plane strain)."""
    d = np.eye(dim)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def isotropic_mandel(lam: float, mu: float, dim: int) -> np.ndarray:
    return tensor4_to_mandel(isotropic_tensor(lam, mu, dim), dim)


def rotate_tensor4(C: np.ndarray, R: np.ndarray) -> np.ndarray:
    """C'_ijkl = R_ip R_jq R_kr R_ls C_pqrs."""
    return np.einsum("ip,jq,kr,ls,pqrs->ijkl", R, R, R, R, C)


# =============================================================================================
# Grid, frequencies and the discrete Green operator (section 2, eq. 2 and the set J)


def signed_frequencies(n: int) -> np.ndarray:
    """DFT bin m -> signed frequency a: J = {-(n-1)/2, ..., (n-1)/2} for odd n (section 2).  The
    paper defines J for odd grids only; for even n the bins run -n/2+1 ... n/2, the last being the
    Nyquist frequency, which `nyquist_mask` singles out."""
    m = np.arange(n)
    return np.where(m <= n // 2, m, m - n)


def nyquist_mask(dim: int, n: int) -> np.ndarray:
    """[*grid] True at the DFT bins with a Nyquist component (bin n/2 along some axis) of an even
    grid; all False for odd n.  A real field's spectrum has no conjugate partner there, so on even
    grids the Green operator gives zero strain at those bins and the equilibrium errors leave them
    out (a reading: the paper does not define even grids)."""
    if n % 2:
        return np.zeros((n,) * dim, dtype=bool)
    nyq = np.arange(n) == n // 2
    grids = np.meshgrid(*([nyq] * dim), indexing="ij")
    out = grids[0].copy()
    for g in grids[1:]:
        out |= g
    return out


SCHEME_CONTINUOUS = 0  # eq. (2): the wave vector xi = 2 pi a of the continuous Green operator
SCHEME_ROTATED = 1     # a modified discrete Green operator (the paper's second category, refs. [1, 11])


def wave_vectors(dim: int, n: int, scheme: int = SCHEME_CONTINUOUS) -> np.ndarray:
    """The wave vector the Green operator and the equilibrium check use at every DFT bin of an
    n^dim grid, numpy axis order (z,) y, x.  Returns [*grid, dim] with component 0 = x, 1 = y, 2 = z.

    SCHEME_CONTINUOUS: xi_k = 2 pi a (section 2, eq. 2).
    SCHEME_ROTATED: the modified discrete Green operator of the "rotated" finite-difference scheme
    (one of the modified operators the paper's introduction cites as the second way to improve the
    method).  There, strains are symmetric finite-difference gradients of a displacement held at
    the voxel corners, each derivative averaged over the 2^(d-1) cell edges along its axis, and
    equilibrium is the adjoint difference of the stress.  The symbol of the derivative along axis
    j is k_j = (1/(2^(d-1) h)) (e^(i t_j) - 1) prod_{m != j} (e^(i t_m) + 1), t = 2 pi a / n; all d
    components share the phase i exp(i sum_m t_m / 2), which cancels in the operator, leaving the
    real vector
        q_j = (2/h) sin(t_j / 2) prod_{m != j} cos(t_m / 2)        (h = 1/n)
    in place of xi everywhere: compatible fields are sym(q (x) u_hat), equilibrium is q . sigma_hat
    = 0, and the Green operator is eq. (2)'s formula evaluated at q."""
    a = signed_frequencies(n).astype(np.float64)
    grids = np.meshgrid(*([a] * dim), indexing="ij")  # axis order (z,) y, x
    comps = [grids[dim - 1 - c] for c in range(dim)]  # x is the last numpy axis
    if scheme == SCHEME_CONTINUOUS:
        return np.stack([2.0 * math.pi * g for g in comps], axis=-1)
    half = [math.pi * g / n for g in comps]  # t_j / 2
    out = []
    for j in range(dim):
        q = 2.0 * n * np.sin(half[j])
        for m in range(dim):
            if m != j:
                q = q * np.cos(half[m])
        out.append(q)
    return np.stack(out, axis=-1)


def gamma0_tensor(xi: np.ndarray, lam0: float, mu0: float) -> np.ndarray:
    """Periodic Green operator of the isotropic reference medium c0 = (lam0, mu0), written out
    as the fourth-order tensor of Moulinec & Suquet:
        G_khij = (d_ki x_h x_j + d_hi x_k x_j + d_kj x_h x_i + d_hj x_k x_i) / (4 mu0 |x|^2)
                 - (lam0 + mu0) / (mu0 (lam0 + 2 mu0)) x_i x_j x_k x_h / |x|^4.
    xi: [..., d] nonzero wave vectors.  Returns [..., d, d, d, d] indexed (k, h, i, j)."""
    d = xi.shape[-1]
    q2 = np.sum(xi * xi, axis=-1)[..., None, None, None, None]
    I = np.eye(d)
    t1 = (np.einsum("ki,...h,...j->...khij", I, xi, xi) + np.einsum("hi,...k,...j->...khij", I, xi, xi)
          + np.einsum("kj,...h,...i->...khij", I, xi, xi) + np.einsum("hj,...k,...i->...khij", I, xi, xi))
    t2 = np.einsum("...i,...j,...k,...h->...khij", xi, xi, xi, xi)
    return t1 / (4.0 * mu0 * q2) - (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0)) * t2 / (q2 * q2)


def apply_gamma0(tau_hat: np.ndarray, dim: int, n: int, lam0: float, mu0: float,
                 chunk: int = 1 << 17, scheme: int = SCHEME_CONTINUOUS) -> np.ndarray:
    """eq. (2): eps_hat(k) = -Gamma0(k) : tau_hat(k) for k != 0 on J (at the scheme's wave vector).
    tau_hat: complex Mandel field [nc, *grid].  Returns -Gamma0:tau_hat with the k = 0 entry
    left at zero (the caller sets eps_hat(0))."""
    nc = nc_of(dim)
    shape = tau_hat.shape[1:]
    npts = int(np.prod(shape))
    xi = wave_vectors(dim, n, scheme).reshape(npts, dim)
    t = mandel_to_tensor2(np.moveaxis(tau_hat.reshape(nc, npts), 0, -1), dim)  # [npts, d, d]
    out = np.zeros((npts, dim, dim), dtype=np.complex128)
    for s in range(0, npts, chunk):
        e = min(npts, s + chunk)
        x = xi[s:e]
        nz = np.sum(x * x, axis=-1) > 0.0
        if not np.any(nz):
            continue
        G = gamma0_tensor(x[nz], lam0, mu0)
        out[s:e][nz] = -np.einsum("pkhij,pij->pkh", G, t[s:e][nz])
    out[nyquist_mask(dim, n).reshape(npts)] = 0.0  # even grids only
    v = tensor2_to_mandel(out, dim)  # [npts, nc]
    return np.moveaxis(v, -1, 0).reshape((nc,) + shape)


def naive_dft(x: np.ndarray, axes: Sequence[int], sign: int = -1) -> np.ndarray:
    """O(n^2)-per-axis DFT by explicit summation: X[k] = sum_m x[m] exp(sign 2 pi i k m / n)."""
    X = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        n = X.shape[ax]
        k = np.arange(n)
        W = np.exp(sign * 2j * math.pi * np.outer(k, k) / n)
        X = np.moveaxis(np.tensordot(W, np.moveaxis(X, ax, 0), axes=(1, 0)), 0, ax)
    return X


def _fft(f: np.ndarray, dim: int) -> np.ndarray:
    return np.fft.fftn(f, axes=tuple(range(-dim, 0)))


def _ifft(f: np.ndarray, dim: int) -> np.ndarray:
    return np.fft.ifftn(f, axes=tuple(range(-dim, 0)))


def equilibrium_errors(sig_hat: np.ndarray, dim: int, n: int, scheme: int = SCHEME_CONTINUOUS) -> Tuple[float, float]:
    """Stress-equilibrium criterion of Moulinec & Suquet (ref. [9] of the paper):
        e   = sqrt(sum_{k in J} |xi_k . sigma_hat(k)|^2) / ||sigma_hat(0)||
        e_n = sqrt(sum_{k in J, k != 0} |(xi_k/|xi_k|) . sigma_hat(k)|^2) / ||sigma_hat(0)||
    with xi the scheme's wave vector (wave_vectors).
    sig_hat: complex Mandel field [nc, *grid] (unnormalised DFT)."""
    nc = nc_of(dim)
    shape = sig_hat.shape[1:]
    npts = int(np.prod(shape))
    xi = wave_vectors(dim, n, scheme).reshape(npts, dim)
    t = mandel_to_tensor2(np.moveaxis(sig_hat.reshape(nc, npts), 0, -1), dim)  # [npts, d, d]
    div = np.einsum("pij,pj->pi", t, xi)
    q2 = np.sum(xi * xi, axis=-1)
    d2 = np.sum(np.abs(div) ** 2, axis=-1)
    d2[nyquist_mask(dim, n).reshape(npts)] = 0.0  # even grids: Nyquist bins left out
    nz = q2 > 0
    den = math.sqrt(float(np.sum(np.abs(t[0]) ** 2)))  # k = 0 is the first bin
    e = math.sqrt(float(np.sum(d2))) / den
    e_n = math.sqrt(float(np.sum(d2[nz] / q2[nz]))) / den
    return e, e_n


# =============================================================================================
# Lippmann-Schwinger fixed point (section 2, eqs. 1-a, 1-b, 2), literal "tau form"

CRIT_E = 0    # e of ref. [9]
CRIT_EN = 1   # normalised variant e_n


def constitutive(ctilde: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """sigma(x) = c(x) : eps(x) in Mandel form.  ctilde [*grid, nc, nc], eps [nc, *grid]."""
    return np.einsum("...IJ,J...->I...", ctilde, eps)


def solve_one(ctilde: np.ndarray, dim: int, n: int, lam0: float, mu0: float, E: np.ndarray,
              tol: float, max_iter: int, criterion: int = CRIT_E, scheme: int = SCHEME_CONTINUOUS,
              eps0: np.ndarray = None) -> Dict:
    """Basic fixed-point scheme for one macroscopic strain E (Mandel [nc]):
        eps^0 = E  (or the given field eps0 [nc, *grid]: a warm start)
        repeat i = 0, 1, ...:
            sigma^i = c : eps^i ; evaluate the equilibrium error of sigma^i; stop if < tol
                (a warm start's eps^0 need not be compatible, so iterate 0 is then never returned:
                the first Green-operator application makes the iterate compatible with mean E)
            tau^i = sigma^i - c0 : eps^i
            eps_hat^{i+1}(k) = -Gamma0(k) : tau_hat^i(k)   (k in J, k != 0)
            eps_hat^{i+1}(0) = E (times N_v for the unnormalised DFT)
            eps^{i+1} = inverse DFT
    (Gamma0 and the error at the scheme's wave vector; SCHEME_CONTINUOUS is eq. 2 itself.)
    Returns the iterate that passed (iterations = number of Green-operator applications)."""
    nc = nc_of(dim)
    grid = (n,) * dim
    nv = n ** dim
    C0 = isotropic_mandel(lam0, mu0, dim)
    eps = np.empty((nc,) + grid)
    for I in range(nc):
        eps[I] = E[I]
    if eps0 is not None:
        eps = np.array(eps0, dtype=np.float64).reshape((nc,) + grid)
    errs, errs_n = [], []
    status = "max_iter"
    it = 0
    while True:
        sigma = constitutive(ctilde, eps)
        e, e_n = equilibrium_errors(_fft(sigma, dim), dim, n, scheme)
        errs.append(e)
        errs_n.append(e_n)
        err = e if criterion == CRIT_E else e_n
        if not math.isfinite(err):
            status = "diverged"
            break
        if err < tol and not (eps0 is not None and it == 0):
            status = "converged"
            break
        if it >= max_iter:
            break
        tau = sigma - constitutive(np.broadcast_to(C0, grid + (nc, nc)), eps)
        eps_hat = apply_gamma0(_fft(tau, dim), dim, n, lam0, mu0, scheme=scheme)
        zero = (slice(None),) + (0,) * dim
        eps_hat[zero] = nv * np.asarray(E, dtype=np.float64)
        eps = np.real(_ifft(eps_hat, dim))
        it += 1
    mean_sigma = np.array([math.fsum(sigma[I].ravel()) for I in range(nc)]) / nv
    return dict(eps=eps, sigma=sigma, mean_sigma=mean_sigma, iterations=it, status=status,
                errors=np.array(errs), errors_n=np.array(errs_n))


def solve(ctilde: np.ndarray, dim: int, n: int, lam0: float, mu0: float, E: np.ndarray,
          tol: float = 1e-8, max_iter: int = 1000, criterion: int = CRIT_E, scheme: int = SCHEME_CONTINUOUS,
          eps0: np.ndarray = None) -> Dict:
    """Solve every load case (rows of E, Mandel [L, nc]) independently; eps0 [L, nc, *grid]
    optionally warm-starts each."""
    E = np.atleast_2d(np.asarray(E, dtype=np.float64))
    runs = [solve_one(ctilde, dim, n, lam0, mu0, E[l], tol, max_iter, criterion, scheme,
                      None if eps0 is None else eps0[l]) for l in range(E.shape[0])]
    return dict(eps=np.stack([r["eps"] for r in runs]), sigma=np.stack([r["sigma"] for r in runs]),
                mean_sigma=np.stack([r["mean_sigma"] for r in runs]),
                iterations=np.array([r["iterations"] for r in runs]),
                status=[r["status"] for r in runs], errors=[r["errors"] for r in runs],
                errors_n=[r["errors_n"] for r in runs])


def fixed_point_map(ctilde: np.ndarray, dim: int, n: int, lam0: float, mu0: float, E: np.ndarray,
                    eps: np.ndarray) -> np.ndarray:
    """F(eps) = E - Gamma0 * ((c - c0) : eps), the map the basic scheme iterates (eqs. 1-a, 1-b, 2):
    eps_hat(k) = -Gamma0(k) : tau_hat(k) for k != 0, eps_hat(0) = E, tau = (c - c0) : eps."""
    nc = nc_of(dim)
    grid = (n,) * dim
    C0 = isotropic_mandel(lam0, mu0, dim)
    tau = constitutive(ctilde, eps) - constitutive(np.broadcast_to(C0, grid + (nc, nc)), eps)
    eps_hat = apply_gamma0(_fft(tau, dim), dim, n, lam0, mu0)
    zero = (slice(None),) + (0,) * dim
    eps_hat[zero] = n ** dim * np.asarray(E, dtype=np.float64)
    return np.real(_ifft(eps_hat, dim))


def solve_refined_one(ctilde: np.ndarray, dim: int, n: int, lam0: float, mu0: float, E: np.ndarray,
                      tol: float, start: np.ndarray, inner_iters: int, max_outer: int,
                      criterion: int = CRIT_EN, inner_dtype=np.float64) -> Dict:
    """Defect correction of the fixed point of section 2 (mixed-precision iterative refinement; the
    paper works in one precision, this is how a low-precision iteration reaches a high-precision
    tolerance).  The discrete problem is eps = F(eps) with F the affine map of eqs. 1-a, 1-b, 2
    (fixed_point_map).  From a start eps_0 (an iterate of the basic scheme), for m = 0, 1, ...:
        evaluate the equilibrium error of eps_m (FP64); stop if below tol;
        r_m = F(eps_m) - eps_m                                  (FP64 residual)
        delta^0 = r_m;  delta^{k+1} = r_m - Gamma0 * ((c - c0) : delta^k), k < inner_iters
                                                                (the same fixed point for the
                                                                 correction, zero mean strain)
        eps_{m+1} = eps_m + delta                               (FP64 update)
    Since F is affine, the exact correction solves delta = F(eps_m + delta) - eps_m, i.e. that inner
    fixed point, so each outer step shrinks the error by the inner iteration's contraction (to the
    inner precision's rounding floor relative to |delta|, not to |eps|).  inner_dtype = float32
    rounds the inner fields to FP32 after every step (an emulation of FP32 storage).
    Returns the final iterate, its errors, the outer steps and the inner iterations performed."""
    nc = nc_of(dim)
    E = np.asarray(E, dtype=np.float64)
    zeroE = np.zeros(nc)
    eps = np.array(start, dtype=np.float64)
    outer = inner = 0
    hist = []
    while True:
        sigma = constitutive(ctilde, eps)
        e, e_n = equilibrium_errors(_fft(sigma, dim), dim, n)
        hist.append((e, e_n))
        err = e if criterion == CRIT_E else e_n
        if err < tol or outer >= max_outer:
            break
        r = fixed_point_map(ctilde, dim, n, lam0, mu0, E, eps) - eps
        r_low = r.astype(inner_dtype).astype(np.float64)
        delta = r_low
        for _ in range(inner_iters):
            delta = (r_low + (fixed_point_map(ctilde, dim, n, lam0, mu0, zeroE, delta))).astype(inner_dtype)
            delta = delta.astype(np.float64)
            inner += 1
        eps = eps + delta
        outer += 1
    mean_sigma = np.array([math.fsum(sigma[I].ravel()) for I in range(nc)]) / n ** dim
    return dict(eps=eps, sigma=sigma, mean_sigma=mean_sigma, outer=outer, inner=inner,
                status="converged" if hist[-1][1 if criterion == CRIT_EN else 0] < tol else "max_outer",
                errors=np.array([h[0] for h in hist]), errors_n=np.array([h[1] for h in hist]))


def compatibility_error(eps: np.ndarray, dim: int, n: int, lam0: float, mu0: float, E: np.ndarray) -> float:
    """e_c = RMS(eps - P eps) / |E| for a strain field eps [nc, *grid] (Mandel), P the projection
    onto compatible fields of mean E that is orthogonal in the energy product of the isotropic c0
    (section 2): (P eps)_hat(k) = Gamma0(k) : c0 : eps_hat(k) for k != 0 and the mean E at k = 0.
    Zero exactly when eps is a symmetric gradient plus E; the basic scheme's iterates are of that
    form by construction, the Eyre-Milton scheme's only at convergence."""
    nv = n ** dim
    C0 = isotropic_mandel(lam0, mu0, dim)
    eps_hat = _fft(eps, dim)
    res = eps_hat + apply_gamma0(np.einsum("IJ,J...->I...", C0, eps_hat), dim, n, lam0, mu0)
    zero = (slice(None),) + (0,) * dim
    res[zero] = eps_hat[zero] - nv * np.asarray(E, dtype=np.float64)
    return math.sqrt(float(np.sum(np.abs(res) ** 2))) / (nv * float(np.linalg.norm(E)))


def solve_em_one(ctilde: np.ndarray, dim: int, n: int, lam0: float, mu0: float, E: np.ndarray,
                 tol: float, max_iter: int, criterion: int = CRIT_EN) -> Dict:
    """Eyre-Milton accelerated scheme (one of the accelerated schemes the paper's introduction and
    section 5 cite as complementary to filtering) for one macroscopic strain E, written from the
    discrete problem: with u = sigma + c0 : eps and v = sigma - c0 : eps, the constitutive law reads
    v = W u, W = (c - c0)(c + c0)^-1 (local, a contraction), and compatibility of eps (mean E) with
    equilibrium of sigma reads v = R u - 2 c0 : E, R = I - 2 c0 Gamma0 (a reflection: c0 Gamma0 is the
    projection onto compatible zero-mean fields for the c0^-1 inner product).  So u = R(W u + 2 c0:E),
    iterated from the uniform u^0 = 2 c0 : E:
        eps^i = (c + c0)^-1 : u^i ;  sigma^i = c : eps^i ; evaluate the equilibrium error of sigma^i
        and the compatibility error e_c of eps^i; stop if both < tol
        w^i = (c - c0) : eps^i + 2 c0 : E
        u_hat^{i+1}(k) = w_hat^i(k) - 2 c0 : Gamma0(k) : w_hat^i(k)  (k != 0),  u_hat^{i+1}(0) = w_hat^i(0)
    The contraction factor is that of W, (sqrt(kappa) - 1) / (sqrt(kappa) + 1) for a contrast kappa
    with c0 the geometric mean of the phase moduli, against (kappa - 1) / (kappa + 1) for the basic
    scheme.  Unlike the basic scheme's, these iterates are not compatible before convergence (a
    laminate's stress can be equilibrated while its strain is not compatible), so the stopping rule
    also bounds e_c = RMS(eps - P eps) / |E|, P the projection onto compatible fields of mean E:
    (P eps)_hat(k) = Gamma0(k) : c0 : eps_hat(k) for k != 0, N_v E at k = 0.
    Returns the iterate that passed (iterations = Green-operator applications) and its e_c."""
    nc = nc_of(dim)
    grid = (n,) * dim
    nv = n ** dim
    C0 = isotropic_mandel(lam0, mu0, dim)
    E = np.asarray(E, dtype=np.float64)
    two_c0E = 2.0 * (C0 @ E)
    cp = ctilde + C0  # c + c0 per voxel
    cm = ctilde - C0
    u = np.empty((nc,) + grid)
    for I in range(nc):
        u[I] = two_c0E[I]
    errs, errs_n, errs_c = [], [], []
    status = "max_iter"
    it = 0
    while True:
        eps = np.moveaxis(np.linalg.solve(cp, np.moveaxis(u, 0, -1)[..., None])[..., 0], -1, 0)
        sigma = constitutive(ctilde, eps)
        e, e_n = equilibrium_errors(_fft(sigma, dim), dim, n)
        e_c = compatibility_error(eps, dim, n, lam0, mu0, E)
        errs.append(e)
        errs_n.append(e_n)
        errs_c.append(e_c)
        err = max(e if criterion == CRIT_E else e_n, e_c)
        if not math.isfinite(err):
            status = "diverged"
            break
        if err < tol:
            status = "converged"
            break
        if it >= max_iter:
            break
        w = constitutive(cm, eps)
        for I in range(nc):
            w[I] += two_c0E[I]
        w_hat = _fft(w, dim)
        gw = -apply_gamma0(w_hat, dim, n, lam0, mu0)  # Gamma0 : w_hat (k != 0), zero at k = 0
        u_hat = w_hat - 2.0 * np.einsum("IJ,J...->I...", C0, gw)
        u = np.real(_ifft(u_hat, dim))
        it += 1
    mean_sigma = np.array([math.fsum(sigma[I].ravel()) for I in range(nc)]) / nv
    return dict(eps=eps, sigma=sigma, mean_sigma=mean_sigma, iterations=it, status=status,
                errors=np.array(errs), errors_n=np.array(errs_n), errors_c=np.array(errs_c))


def solve_em(ctilde: np.ndarray, dim: int, n: int, lam0: float, mu0: float, E: np.ndarray,
             tol: float = 1e-8, max_iter: int = 1000, criterion: int = CRIT_EN) -> Dict:
    """solve_em_one for every load case (rows of E)."""
    E = np.atleast_2d(np.asarray(E, dtype=np.float64))
    runs = [solve_em_one(ctilde, dim, n, lam0, mu0, E[l], tol, max_iter, criterion) for l in range(E.shape[0])]
    return dict(eps=np.stack([r["eps"] for r in runs]), sigma=np.stack([r["sigma"] for r in runs]),
                mean_sigma=np.stack([r["mean_sigma"] for r in runs]),
                iterations=np.array([r["iterations"] for r in runs]), status=[r["status"] for r in runs],
                errors=[r["errors"] for r in runs], errors_n=[r["errors_n"] for r in runs],
                errors_c=[r["errors_c"] for r in runs])


def em_reference(phases: Sequence[Tuple[float, float]], dim: int) -> Tuple[float, float]:
    """Reference medium of the Eyre-Milton scheme: the geometric means of the extreme phase shear
    and bulk moduli (bulk lam + 2 mu / d), returned as Lame constants (lam0, mu0)."""
    mus = [mu for (_, mu) in phases]
    ks = [lam + 2.0 * mu / dim for (lam, mu) in phases]
    mu0 = math.sqrt(min(mus) * max(mus))
    k0 = math.sqrt(min(ks) * max(ks))
    return k0 - 2.0 * mu0 / dim, mu0


def effective_stiffness(mean_sigma: np.ndarray, E: np.ndarray) -> np.ndarray:
    """C_eff from the mean stresses of linearly independent load cases:
    <sigma^(l)> = C_eff E^(l) for every l, i.e. C_eff = S^T (E^T)^-1 with rows of S, E per load."""
    S = np.atleast_2d(mean_sigma)
    E = np.atleast_2d(E)
    return np.linalg.solve(E, S).T


# =============================================================================================
# Filtered stiffness (section 2, eqs. 3, 4, 5): volume fractions on a refined grid


def sample_offsets(dim: int, radius_px: float, S: int) -> np.ndarray:
    """Fine-lattice offsets inside the filter ball.

    The refined grid has spacing h/S with points at (j + 1/2) h / S (j integer, per axis).
    Measured in units of h/(2S) a fine point sits at 2j + 1 and the centre of voxel a at
    (2a + 1) S, so with j = a S + t the separation is D = 2t + 1 - S (an exact integer).
    A fine point is in the ball of radius r h when sum D^2 <= (2 S r)^2.
    Returns the integer offsets t [M, dim] (the same for every voxel)."""
    two_s_r = (2.0 * S) * radius_px
    R2 = two_s_r * two_s_r
    K = int(math.ceil(S * radius_px)) + S
    t = np.arange(-K, K + S + 1)
    D = 2 * t + 1 - S
    grids = np.meshgrid(*([D] * dim), indexing="ij")
    q = sum(g.astype(np.int64) ** 2 for g in grids)
    keep = q.astype(np.float64) <= R2
    tg = np.meshgrid(*([t] * dim), indexing="ij")
    return np.stack([g[keep] for g in tg], axis=-1)


def _inside_primitive(prim, su: np.ndarray, S: int, n: int, dim: int) -> np.ndarray:
    """Exact membership test of fine points in one primitive (periodic).

    su: [..., dim] sample coordinates in units of h/(2S) (odd integers stored as float64,
    component 0 = x).  The recipe fixes every IEEE operation so that an independent
    implementation doing the same operations gets the same answer:
      cu = c * (2 S n);  du = su - cu;  du -= 2 S n if du > S n;  du += 2 S n if du < -S n
      disk/sphere: inside iff ((du_x^2 + du_y^2) + du_z^2) <= (R * 2 S n)^2
      slab (normal axis a, thickness T): inside iff |du_a| <= T * (S n)."""
    P2 = float(2 * S * n)
    half = float(S * n)

    def wrapped(axis):
        cu = prim.centre[axis] * P2
        du = su[..., axis] - cu
        du = np.where(du > half, du - P2, du)
        du = np.where(du < -half, du + P2, du)
        return du

    if prim.kind == PRIM_SLAB:
        return np.abs(wrapped(prim.axis)) <= prim.radius * half
    Ru = prim.radius * P2
    Ru2 = Ru * Ru
    q = wrapped(0) * wrapped(0)
    for axis in range(1, dim):
        w = wrapped(axis)
        q = q + w * w
    return q <= Ru2


def phase_at(cell: Cell, su: np.ndarray, S: int) -> np.ndarray:
    """Phase of fine points: the first primitive (list order) containing the point, else the
    matrix phase."""
    out = np.full(su.shape[:-1], cell.matrix_phase, dtype=np.int64)
    decided = np.zeros(su.shape[:-1], dtype=bool)
    for prim in cell.prims:
        inside = _inside_primitive(prim, su, S, cell.n, cell.dim) & ~decided
        out[inside] = prim.phase
        decided |= inside
    return out


def _voxel_centres(dim: int, n: int) -> np.ndarray:
    """[*grid, dim] voxel-centre coordinates (component 0 = x), numpy axis order (z,) y, x."""
    a = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([a] * dim), indexing="ij")
    return np.stack([grids[dim - 1 - c] for c in range(dim)], axis=-1)


def _voxel_index(dim: int, n: int) -> np.ndarray:
    a = np.arange(n)
    grids = np.meshgrid(*([a] * dim), indexing="ij")
    return np.stack([grids[dim - 1 - c] for c in range(dim)], axis=-1)


def surface_distance(prim, x: np.ndarray, dim: int) -> Tuple[np.ndarray, np.ndarray]:
    """Distance from points x [..., dim] to the primitive's surface (periodic minimum image)
    and the unit vector from the centre (disk/sphere) or the slab normal."""
    c = np.array(prim.centre[:dim])
    if prim.kind == PRIM_SLAB:
        d = x[..., prim.axis] - c[prim.axis]
        d = d - np.round(d)
        dist = np.abs(np.abs(d) - 0.5 * prim.radius)
        nrm = np.zeros(x.shape)
        nrm[..., prim.axis] = 1.0
        return dist, nrm
    v = x - c
    v = v - np.round(v)
    r = np.sqrt(np.sum(v * v, axis=-1))
    with np.errstate(invalid="ignore", divide="ignore"):
        nrm = v / r[..., None]
    return np.abs(r - prim.radius), nrm


def volume_fraction_counts(cell: Cell, phases_count: int, brute_force: bool = False):
    """Per-voxel counts of fine-lattice samples of each phase inside the filter ball
    (section 2: "averaging indicator functions evaluated on a refined grid").

    Returns counts [*grid, phases_count] (int64) and the number of samples M per ball.
    Unless brute_force, voxels whose ball cannot reach any primitive surface (distance from the
    voxel centre to every surface > r h + 1e-9) are not sampled: all their samples share the
    phase of the voxel centre, which is exact."""
    dim, n, S, r = cell.dim, cell.n, cell.subgrid, cell.radius_px
    offs = sample_offsets(dim, r, S)
    M = offs.shape[0]
    idx = _voxel_index(dim, n).reshape(-1, dim)
    nv = idx.shape[0]
    counts = np.zeros((nv, phases_count), dtype=np.int64)
    centre_su = (2 * idx + 1).astype(np.float64) * S
    centre_phase = phase_at(cell, centre_su, S)
    if brute_force:
        near = np.ones(nv, dtype=bool)
    else:
        x = _voxel_centres(dim, n).reshape(-1, dim)
        near = np.zeros(nv, dtype=bool)
        for prim in cell.prims:
            dist, _ = surface_distance(prim, x, dim)
            near |= dist <= r / n + 1e-9
    far = ~near
    counts[far, centre_phase[far]] = M
    sel = np.nonzero(near)[0]
    chunk = max(1, (1 << 22) // max(M, 1))
    for s in range(0, sel.size, chunk):
        v = sel[s:s + chunk]
        j = idx[v][:, None, :] * S + offs[None, :, :]
        su = (2 * j + 1).astype(np.float64)
        ph = phase_at(cell, su, S)
        for p in range(phases_count):
            counts[v, p] = np.sum(ph == p, axis=1)
    shape = (n,) * dim + (phases_count,)
    return counts.reshape(shape), M


def hr_voigt(Cs: Sequence[np.ndarray], fs: Sequence[float]) -> np.ndarray:
    """eq. (3): c_tilde = sum_i f_i c_i."""
    return sum(f * C for f, C in zip(fs, Cs))


def hr_reuss(Cs: Sequence[np.ndarray], fs: Sequence[float]) -> np.ndarray:
    """eq. (4): c_tilde = (sum_i f_i c_i^-1)^-1."""
    return np.linalg.inv(sum(f * np.linalg.inv(C) for f, C in zip(fs, Cs)))


def interface_frame(normal: np.ndarray) -> np.ndarray:
    """Orthonormal rows (t1[, t2], n): the interface normal is the last local axis."""
    nrm = np.asarray(normal, dtype=np.float64)
    nrm = nrm / np.linalg.norm(nrm)
    if nrm.size == 2:
        return np.array([[nrm[1], -nrm[0]], [nrm[0], nrm[1]]])
    e = np.zeros(3)
    e[int(np.argmin(np.abs(nrm)))] = 1.0
    t1 = np.cross(nrm, e)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(nrm, t1)
    return np.array([t1, t2, nrm])


def _in_plane_components(dim: int) -> Tuple[List[int], List[int]]:
    """Local Mandel components split into in-plane (P: both indices tangential) and
    out-of-plane (OP: at least one index along the normal, the last local axis)."""
    P, O = [], []
    for I, (i, j) in enumerate(mandel_pairs(dim)):
        (O if (i == dim - 1 or j == dim - 1) else P).append(I)
    return P, O


def hr_two_layer(C1: np.ndarray, C2: np.ndarray, f1: float, f2: float, normal: np.ndarray,
                 dim: int) -> np.ndarray:
    """eqs. (5-a), (5-b): two-phase laminate with planar interface of the given normal.

    In the interface frame, for each unit macroscopic strain eps (local Mandel basis) the
    phase strains eps1, eps2 satisfy
        eps1^P = eps2^P = eps^P                    (5-a, in-plane strain continuous)
        (C1 eps1)^OP = (C2 eps2)^OP                (5-a, out-of-plane stress continuous)
        f1 eps1^OP + f2 eps2^OP = eps^OP           (5-b)
    which is solved as one dense 2nc x 2nc linear system; the homogenised stress is
    sigma^OP = (C1 eps1)^OP and sigma^P = f1 (C1 eps1)^P + f2 (C2 eps2)^P (5-b)."""
    nc = nc_of(dim)
    R = interface_frame(normal)
    L1 = tensor4_to_mandel(rotate_tensor4(mandel_to_tensor4(C1, dim), R), dim)
    L2 = tensor4_to_mandel(rotate_tensor4(mandel_to_tensor4(C2, dim), R), dim)
    P, O = _in_plane_components(dim)
    A = np.zeros((2 * nc, 2 * nc))
    row = 0
    rows_rhs = []
    for I in P:
        A[row, I] = 1.0
        rows_rhs.append(("P", I))
        row += 1
    for I in P:
        A[row, nc + I] = 1.0
        rows_rhs.append(("P", I))
        row += 1
    for I in O:
        A[row, I] = f1
        A[row, nc + I] = f2
        rows_rhs.append(("O", I))
        row += 1
    for I in O:
        A[row, :nc] = L1[I]
        A[row, nc:] = -L2[I]
        rows_rhs.append(("Z", I))
        row += 1
    Cloc = np.zeros((nc, nc))
    for J in range(nc):
        b = np.array([1.0 if (kind != "Z" and I == J) else 0.0 for (kind, I) in rows_rhs])
        x = np.linalg.solve(A, b)
        e1, e2 = x[:nc], x[nc:]
        s1, s2 = L1 @ e1, L2 @ e2
        sig = np.empty(nc)
        for I in P:
            sig[I] = f1 * s1[I] + f2 * s2[I]
        for I in O:
            sig[I] = s1[I]
        Cloc[:, J] = sig
    return tensor4_to_mandel(rotate_tensor4(mandel_to_tensor4(Cloc, dim), R.T), dim)


def filter_build(cell: Cell, phases: Sequence[Tuple[float, float]], brute_force: bool = False) -> Dict:
    """c_tilde(x_a) = HR(c, omega(x_a)) for every grid point (section 2).

    RULE_NONE samples the phase at the grid point itself.  Otherwise the filter counts
    fine-lattice samples per phase; a voxel whose samples all share one phase keeps that
    phase's stiffness exactly, otherwise the rule is applied to the volume fractions
    f_i = count_i / M.  The 2-layer normal is the unit vector from the centre of the
    primitive whose surface is nearest to x_a (periodic image) to x_a, or the slab normal.
    The 2-layer rule takes the two phases present; with a degenerate normal it falls back to
    Voigt.  Returns ctilde [*grid, nc, nc], counts, M, mixed mask, fraction of the second
    phase and normals."""
    dim, n = cell.dim, cell.n
    nc = nc_of(dim)
    Cs = [isotropic_mandel(lam, mu, dim) for (lam, mu) in phases]
    grid = (n,) * dim
    nphase = len(phases)
    idx = _voxel_index(dim, n).reshape(-1, dim)
    nv = idx.shape[0]
    ctilde = np.empty((nv, nc, nc))
    mixed = np.zeros(nv, dtype=bool)
    normals = np.zeros((nv, dim))
    if cell.rule == RULE_NONE:
        ph = phase_at(cell, (2 * idx + 1).astype(np.float64) * cell.subgrid, cell.subgrid)
        for v in range(nv):
            ctilde[v] = Cs[ph[v]]
        return dict(ctilde=ctilde.reshape(grid + (nc, nc)), mixed=mixed.reshape(grid), counts=None,
                    M=1, normals=normals.reshape(grid + (dim,)))
    counts, M = volume_fraction_counts(cell, nphase, brute_force)
    counts = counts.reshape(nv, nphase)
    x = _voxel_centres(dim, n).reshape(-1, dim)
    best = np.full(nv, np.inf)
    for prim in cell.prims:
        dist, nrm = surface_distance(prim, x, dim)
        better = dist < best
        best = np.where(better, dist, best)
        normals[better] = nrm[better]
    for v in range(nv):
        present = np.nonzero(counts[v])[0]
        if present.size == 1:
            ctilde[v] = Cs[present[0]]
            continue
        mixed[v] = True
        fs = counts[v, present] / M
        cs = [Cs[p] for p in present]
        if cell.rule == RULE_VOIGT:
            ctilde[v] = hr_voigt(cs, fs)
        elif cell.rule == RULE_REUSS:
            ctilde[v] = hr_reuss(cs, fs)
        elif cell.rule == RULE_TWO_LAYER:
            if present.size != 2:
                raise ValueError("the 2-layer rule needs exactly two phases in the filter")
            nv_ = normals[v]
            if not np.all(np.isfinite(nv_)) or np.linalg.norm(nv_) < 0.5:
                ctilde[v] = hr_voigt(cs, fs)
            else:
                ctilde[v] = hr_two_layer(cs[0], cs[1], fs[0], fs[1], nv_, dim)
        else:
            raise ValueError("unknown rule")
    return dict(ctilde=ctilde.reshape(grid + (nc, nc)), mixed=mixed.reshape(grid),
                counts=counts.reshape(grid + (nphase,)), M=M, normals=normals.reshape(grid + (dim,)))


def default_reference(phases: Sequence[Tuple[float, float]]) -> Tuple[float, float]:
    """Reference medium (lam0, mu0) = means of the extreme phase Lamé constants."""
    lams = [p[0] for p in phases]
    mus = [p[1] for p in phases]
    return 0.5 * (min(lams) + max(lams)), 0.5 * (min(mus) + max(mus))


# =============================================================================================
# Fourier extrapolation of the filtered stiffness (section 6, Fig. 4)


def fourier_extrapolate(field: np.ndarray, dim: int, n: int, m: int) -> np.ndarray:
    """Truncated Fourier series of a real grid field, evaluated on a finer grid (section 6, Fig. 4).

    The Fourier coefficients are the FFT of the values at the grid points x_a = (a + 1/2)/n; the
    series keeps the frequencies of J (-(n-1)/2 .. (n-1)/2 per axis) and is evaluated at the voxel
    centres y_b = (b + 1/2)/m of an m^dim grid:
        f(y) = n^-dim sum_{k in J} f_hat(k) exp(2 pi i k . (y - x_0)),   x_0 = 1/(2n) per axis,
    the shift making f(x_a) reproduce the field's value at x_a.  field: [(n,) n, n] (numpy axis
    order (z,) y, x).  Returns [(m,) m, m] float64 (J is symmetric for odd n, so the series is
    real; the imaginary part of the sum is rounding and is dropped)."""
    if n % 2 == 0:
        raise ValueError("the truncated series on J is real for odd grids only")
    fh = _fft(np.asarray(field, dtype=np.float64).reshape((n,) * dim), dim)
    k = signed_frequencies(n)
    y = (np.arange(m) + 0.5) / m
    W = np.exp(2j * np.pi * np.outer(y - 0.5 / n, k))     # [m, n] over (fine point, FFT index)
    out = fh
    for ax in range(dim):
        out = np.moveaxis(np.tensordot(W, out, axes=([1], [ax])), 0, ax)
    return out.real / float(n) ** dim


def exact_property(cell: Cell, values: Sequence[float], m: int) -> np.ndarray:
    """A per-phase scalar (values[phase]) at the voxel centres of an m^dim grid, m a multiple of
    the cell's n: the unfiltered microstructure that Fig. 4-A shows, point-sampled by the same
    exact membership recipe as the filter."""
    if m % cell.n:
        raise ValueError("m must be a multiple of n")
    k = m // cell.n
    b = np.arange(m)
    grids = np.meshgrid(*([b] * cell.dim), indexing="ij")
    su = np.stack([2.0 * grids[cell.dim - 1 - c] + 1.0 for c in range(cell.dim)], axis=-1)
    return np.asarray(values, dtype=np.float64)[phase_at(cell, su, k)]


# =============================================================================================
# Conjugate gradients on the same discrete problem (an accelerated scheme of the kind the
# paper's introduction and section 5 call complementary to filtering)


def projection_G(f: np.ndarray, dim: int, n: int) -> np.ndarray:
    """G f: the compatible, zero-mean part of a real Mandel field f [nc, *grid].  G is eq. (2)'s
    Green operator for the reference medium c0 = identity (lam0 = 0, mu0 = 1/2), for which
    Gamma0 : c0 = Gamma0 is the L2-orthogonal projection onto compatible zero-mean strain fields."""
    return -np.real(_ifft(apply_gamma0(_fft(f, dim), dim, n, 0.0, 0.5), dim))


def _dot(a: np.ndarray, b: np.ndarray) -> float:
    """L2 inner product of two real Mandel fields (Mandel components make it the tensor product)."""
    return math.fsum((a * b).ravel())


def solve_cg_one(ctilde: np.ndarray, dim: int, n: int, E: np.ndarray, tol: float, max_iter: int,
                 history: bool = False) -> Dict:
    """Conjugate gradients for the strain eps = E + x, x compatible with zero mean, such that the
    stress c : eps is in equilibrium, i.e. G(c : eps) = 0:
        A x = b   with  A x = G(c : x),  b = -G(c : E)
    A is symmetric positive definite on compatible zero-mean fields (G is an orthogonal projection,
    c is symmetric positive definite at every grid point), so plain CG applies:
        x = 0, r = b, p = r
        repeat k = 0, 1, ...:
            sigma = c : (E + x);  e_G = sqrt(<r, r> / N_v) / |<sigma>|
            if e_G < tol: recompute the true residual r_t = -G(sigma); stop if e_G(r_t) < tol,
                          else restart from it (r = p = r_t)
            q = A p;  alpha = <r, r> / <p, q>
            x += alpha p;  r -= alpha q
            beta = <r, r>_new / <r, r>_old;  p = r + beta p
    The recursion r -= alpha q drifts from the true residual in finite precision; the check makes
    the stopping rule hold for the returned iterate itself.  r = -G sigma is the projected stress,
    so e_G lies between e_n and sqrt(2) e_n (per frequency, |G s|^2 = 2 |s n|^2 - (n.s n)^2 for
    the unit wave vector n).  iterations = CG steps taken (x updates)."""
    nc = nc_of(dim)
    grid = (n,) * dim
    nv = n ** dim
    Ef = np.empty((nc,) + grid)
    for I in range(nc):
        Ef[I] = E[I]
    x = np.zeros((nc,) + grid)
    r = -projection_G(constitutive(ctilde, Ef), dim, n)
    p = r.copy()
    rr = _dot(r, r)
    errs, res = [], []
    status = "max_iter"
    it = 0
    while True:
        sigma = constitutive(ctilde, Ef + x)
        mean_sigma = np.array([math.fsum(sigma[I].ravel()) for I in range(nc)]) / nv
        e_g = math.sqrt(rr / nv) / float(np.linalg.norm(mean_sigma))
        errs.append(e_g)
        if history:
            res.append(r.copy())
        if not math.isfinite(e_g):
            status = "diverged"
            break
        if e_g < tol:
            r_t = -projection_G(sigma, dim, n)
            rr_t = _dot(r_t, r_t)
            e_t = math.sqrt(rr_t / nv) / float(np.linalg.norm(mean_sigma))
            errs[-1] = e_t
            if e_t < tol:
                status = "converged"
                break
            r, p, rr = r_t, r_t.copy(), rr_t
        if it >= max_iter:
            break
        q = projection_G(constitutive(ctilde, p), dim, n)
        pq = _dot(p, q)
        if not pq > 0.0:
            status = "diverged"
            break
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = _dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    out = dict(eps=Ef + x, sigma=sigma, mean_sigma=mean_sigma, iterations=it, status=status,
               errors=np.array(errs))
    if history:
        out["residuals"] = res
    return out


def solve_cg(ctilde: np.ndarray, dim: int, n: int, E: np.ndarray, tol: float = 1e-8,
             max_iter: int = 1000) -> Dict:
    """solve_cg_one for every load case (rows of E, Mandel [L, nc])."""
    E = np.atleast_2d(np.asarray(E, dtype=np.float64))
    runs = [solve_cg_one(ctilde, dim, n, E[l], tol, max_iter) for l in range(E.shape[0])]
    return dict(eps=np.stack([r["eps"] for r in runs]), sigma=np.stack([r["sigma"] for r in runs]),
                mean_sigma=np.stack([r["mean_sigma"] for r in runs]),
                iterations=np.array([r["iterations"] for r in runs]),
                status=[r["status"] for r in runs], errors=[r["errors"] for r in runs])
